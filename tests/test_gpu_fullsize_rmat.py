"""Parity at the full size of the listing configuration: R-MAT scale 24, edge
factor 16 -- T, T_v, C_v, the two-pass triangle list (about 10^10 triples)
and the sparsified count at q = 0.1, with the thresholds bench.py picks.

The oracle cannot run NodeIterator++ on 260M edges of R-MAT within a test, so
the checks are T_v and C_v on sampled vertices (by their definition, one vertex
at a time), the sparsified count (the oracle counts the kept graph), and
properties that hold at any size: sum T_v = 3T, the listing has T rows,
strictly increasing (so no triangle repeats), and sampled rows are triangles.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import synth
from tests.test_gpu_fullsize import occurrences, rows_oriented, rows_strictly_increasing

pytestmark = pytest.mark.gpu

SCALE = 24
N = 1 << SCALE


@pytest.fixture(scope="module")
def run():
    from paper_1706_05151_gb300 import build
    build.build()
    import paper_1706_05151_gb300 as tc
    from paper_1706_05151_gb300 import autotune
    e = synth.rmat(SCALE, 16, 1)
    g = tc.orient(torch.from_numpy(e).cuda(), N)
    autotune.tune(g, record=False)
    T, tv, cc, tri = tc.analyze(g)
    yield tc, e, g, T, tv, cc, tri
    tc.default_context().set_tuning(0, 1)
    tc.default_context().set_hub_min(0)


@pytest.fixture(scope="module")
def adj(run):
    return oracle.Adjacency(N, run[1])


def test_rmat24_sampled_vertex_counts(run, adj):
    tc, e, g, T, tv, cc, tri = run
    deg = adj.deg
    rng = np.random.default_rng(11)
    cand = np.flatnonzero((deg >= 2) & (deg <= 3000))
    sample = [int(v) for v in rng.choice(cand, 300, replace=False)]
    sample += [int(v) for v in np.argsort(deg)[-200:] if deg[v] <= 3000][:20]  # some of the largest lists too
    ref_tv = np.array([adj.vertex_triangles(v) for v in sample], dtype=np.int64)
    assert np.array_equal(tv.cpu().numpy()[sample], ref_tv)
    ref_cc = oracle.clustering(deg[sample], ref_tv)
    assert np.array_equal(cc.cpu().numpy()[sample].view(np.uint64), ref_cc.view(np.uint64))


def test_rmat24_listing_and_invariants(run, adj):
    tc, e, g, T, tv, cc, tri = run
    assert T > 10 ** 9  # about 1.03e10: the listing is ~123 GB on the device
    assert int(tv.sum().item()) == 3 * T
    assert tri.shape[0] == T
    assert rows_strictly_increasing(tri)
    assert rows_oriented(tri, g.deg)
    idx = torch.from_numpy(np.random.default_rng(12).choice(T, 20000, replace=False)).cuda()
    th = tri[idx].cpu().numpy()

    def has(a, b):
        lo, hi = adj.off[a], adj.off[a + 1]
        j = np.searchsorted(adj.adj[lo:hi], b)
        return j < hi - lo and adj.adj[lo + j] == b
    assert all(has(a, b) and has(b, c) and has(a, c) for a, b, c in th)
    # a vertex's triangles in the listing are its T_v (one full pass over the list per vertex)
    for v in (int(np.argmax(adj.deg)), int(th[0][1]), int(th[1][2])):
        assert occurrences(tri, v) == int(tv[v].item())


def test_rmat24_sparsified_count(run):
    tc, e, g, *_ = run
    t, mk, est = tc.sparsify_count(g, 0.1, 1)
    rt, rmk, rest = oracle.sparsify_count(N, e, 1, 0.1)
    assert (t, mk) == (rt, rmk)
    assert est == rest
