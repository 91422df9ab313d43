"""Exact parity at the full size of the listing configuration: R-MAT scale 24,
edge factor 16 -- T, T_v, C_v, the two-pass triangle list (about 10^10
triples, 123 GB on the device) and the sparsified count at q = 0.1, with the
thresholds bench.py picks.

The oracle result is complete, computed on the host's cores by the parallel
oracle (NodeIteratorN, Figure 2, pinned to the serial NodeIterator++): the
whole oriented CSR, T, every T_v and C_v, and, since the listing does not fit
in host memory, the listing compared as a set: the same number of rows, no
row repeated (strictly increasing), every row in the order, the same count of
triangles for every first vertex, and the same pair of hash sums over all
rows (tests/fingerprint.py).
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import par
from tests.fingerprint import listing_fingerprint
from tests.test_gpu_fullsize import apex_counts, equal_on_device, rows_oriented, rows_strictly_increasing

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
    tc.default_context().set_kernel_shape(0, 0, 0, 0)
    tc.default_context().release_workspace()
    del g, tv, cc, tri
    torch.cuda.empty_cache()


@pytest.fixture(scope="module")
def ref(run):
    e = run[1]
    adj = par.adjacency(N, e)
    deg = adj.deg
    off, cols, dhat = par.orient(adj)
    r = par.count(N, off, cols, local=True, fingerprint=True)
    r.update(off=off, cols=cols, dhat=dhat, deg=deg, adj=adj)
    return r


def test_rmat24_orientation_is_exact(run, ref):
    tc, e, g, *_ = run
    assert equal_on_device(g.offsets, ref["off"])
    assert equal_on_device(g.dhat, ref["dhat"])
    assert equal_on_device(g.deg, ref["deg"])
    assert equal_on_device(g.cols, ref["cols"])


def test_rmat24_counts_are_exact(run, ref):
    tc, e, g, T, tv, cc, tri = run
    assert T == ref["T"] > 10 ** 9  # about 1.03e10
    assert np.array_equal(tv.cpu().numpy(), ref["tv"])
    ref_cc = oracle.clustering(ref["deg"], ref["tv"])
    assert np.array_equal(cc.cpu().numpy().view(np.uint64), ref_cc.view(np.uint64))


def test_rmat24_listing_equals_the_oracle_set(run, ref):
    tc, e, g, T, tv, cc, tri = run
    assert tri.shape[0] == ref["T"]
    assert rows_strictly_increasing(tri)
    assert rows_oriented(tri, g.deg)
    assert np.array_equal(apex_counts(tri, N).cpu().numpy(), ref["apex"])
    assert listing_fingerprint(tri) == ref["fp"]
    # and sampled rows are triangles of the input graph
    adj = ref["adj"]
    idx = torch.from_numpy(np.random.default_rng(12).choice(T, 20000, replace=False)).cuda()
    th = tri[idx].cpu().numpy()

    def has(a, b):
        lo, hi = adj.off[a], adj.off[a + 1]
        j = np.searchsorted(adj.adj[lo:hi], b)
        return j < hi - lo and adj.adj[lo + j] == b
    assert all(has(a, b) and has(b, c) and has(a, c) for a, b, c in th)


def test_rmat24_sparsified_count(run, ref):
    tc, e, g, *_ = run
    t, mk, est = tc.sparsify_count(g, 0.1, 1)
    rt, rmk, rest = par.sparsify_count(N, e, ref["deg"], 1, 0.1)
    assert (t, mk) == (rt, rmk)
    assert est == rest
