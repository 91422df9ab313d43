"""Parity at the full size of the preferential-attachment configuration, PA(n = 2^24, k = 16).

The oracle cannot run NodeIterator++ on 268M edges within a test, so the
checks are: the whole oriented CSR (the oracle's orientation is one linear
pass), T_v and C_v on sampled vertices (T_v by its definition, one vertex at a
time), the sparsified count and kept-edge count (the oracle counts the small
kept graph), and properties that hold at any size.  The calls are the ones
bench.py times, with the same launch configuration.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

N = 1 << 24


@pytest.fixture(scope="module")
def run():
    from paper_1706_05151_gb300 import build
    build.build()
    import paper_1706_05151_gb300 as tc
    e = synth.ba(N, 16, 1)
    g = tc.orient(torch.from_numpy(e).cuda(), N)
    T, tv, cc, tri = tc.analyze(g)
    return tc, e, g, T, tv, cc, tri


def test_fullsize_orientation_is_exact(run):
    tc, e, g, *_ = run
    adj = oracle.Adjacency(N, e)
    off, cols, dhat = adj.orient()
    assert np.array_equal(g.offsets.cpu().numpy(), off)
    assert np.array_equal(g.dhat.cpu().numpy(), dhat)
    assert np.array_equal(g.deg.cpu().numpy(), adj.deg)
    assert np.array_equal(g.cols.cpu().numpy(), cols)
    run_cache["adj"] = adj


run_cache = {}


def test_fullsize_sampled_vertex_counts(run):
    tc, e, g, T, tv, cc, tri = run
    adj = run_cache.get("adj") or oracle.Adjacency(N, e)
    deg = adj.deg
    rng = np.random.default_rng(5)
    sample = rng.choice(N, 400, replace=False)
    sample = np.concatenate([sample, np.arange(0, 64)])            # the oldest, highest-degree vertices
    sample = [int(v) for v in sample if deg[v] <= 4000]
    tv_h = tv.cpu().numpy()
    cc_h = cc.cpu().numpy()
    ref_tv = np.array([adj.vertex_triangles(v) for v in sample], dtype=np.int64)
    assert np.array_equal(tv_h[sample], ref_tv)
    ref_cc = oracle.clustering(deg[sample], ref_tv)
    assert np.array_equal(cc_h[sample].view(np.uint64), ref_cc.view(np.uint64))


def test_fullsize_invariants(run):
    tc, e, g, T, tv, cc, tri = run
    assert int(tv.sum().item()) == 3 * T
    assert tc.count(g) == T
    assert len(tri) == T
    # every listed triple is a triangle, listed once
    assert int(torch.unique(tri, dim=0).shape[0]) == T
    adj = run_cache.get("adj") or oracle.Adjacency(N, e)
    idx = np.random.default_rng(6).choice(T, min(T, 20000), replace=False)
    th = tri[idx].cpu().numpy()

    def has(a, b):
        lo, hi = adj.off[a], adj.off[a + 1]
        j = np.searchsorted(adj.adj[lo:hi], b)
        return j < hi - lo and adj.adj[lo + j] == b
    assert all(has(a, b) and has(b, c) and has(a, c) for a, b, c in th)


def test_fullsize_sparsified_count(run):
    tc, e, g, *_ = run
    t, mk, est = tc.sparsify_count(g, 0.1, 1)
    rt, rmk, rest = oracle.sparsify_count(N, e, 1, 0.1)
    assert (t, mk) == (rt, rmk)
    assert est == rest
