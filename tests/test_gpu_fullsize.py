"""Exact parity at the full size of the preferential-attachment configuration, PA(n = 2^24, k = 16).

Everything is compared with a complete oracle result, computed on the host's
cores by the parallel oracle (oracle/par.py: NodeIteratorN, Figure 2, pinned
to the serial NodeIterator++ of Figure 1): the whole oriented CSR, T, the
whole T_v and C_v vectors, the whole triangle list (343,808 triples) and the
sparsified count.  The calls are the ones bench.py times, with the thresholds
it picks.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import par

pytestmark = pytest.mark.gpu

N = 1 << 24


@pytest.fixture(scope="module")
def run():
    from paper_1706_05151_gb300 import build
    build.build()
    import paper_1706_05151_gb300 as tc
    from paper_1706_05151_gb300 import autotune
    e = synth.ba(N, 16, 1)
    g = tc.orient(torch.from_numpy(e).cuda(), N)
    autotune.tune(g, record=False)  # the thresholds bench.py picks before it times
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
    """The oracle's full result on the same edge list."""
    e = run[1]
    adj = par.adjacency(N, e)
    deg = adj.deg
    off, cols, dhat = par.orient(adj)
    del adj
    r = par.count(N, off, cols, local=True, fingerprint=True)
    r.update(off=off, cols=cols, dhat=dhat, deg=deg)
    return r


def equal_on_device(dev: torch.Tensor, host: np.ndarray, chunk: int = 1 << 28) -> bool:
    """dev == host element by element, copying the host array up in chunks."""
    if dev.numel() != host.size:
        return False
    flat = dev.reshape(-1)
    h = host.reshape(-1)
    for s in range(0, h.size, chunk):
        if not torch.equal(flat[s:s + chunk], torch.from_numpy(np.ascontiguousarray(h[s:s + chunk])).to(dev.device)):
            return False
    return True


def rows_strictly_increasing(tri: torch.Tensor, chunk: int = 1 << 27) -> bool:
    """Each triple (v, u, w) is lexicographically below the next (on the device, in chunks):
    the listing is in oriented-edge order with ascending w, so no triple repeats."""
    T = tri.shape[0]
    for s in range(0, max(T - 1, 0), chunk):
        e = min(s + chunk, T - 1)
        a, b = tri[s:e], tri[s + 1:e + 1]
        lt = (a[:, 0] < b[:, 0]) | ((a[:, 0] == b[:, 0]) & ((a[:, 1] < b[:, 1]) |
                                                          ((a[:, 1] == b[:, 1]) & (a[:, 2] < b[:, 2]))))
        if not bool(lt.all()):
            return False
    return True


def rows_oriented(tri: torch.Tensor, deg: torch.Tensor, chunk: int = 1 << 27) -> bool:
    """Every triple (v, u, w) has v before u before w in the order of Eq. (1) (degree, then id)."""
    def before(x, y):
        dx, dy = deg[x], deg[y]
        return (dx < dy) | ((dx == dy) & (x < y))
    for s in range(0, tri.shape[0], chunk):
        t = tri[s:s + chunk].to(torch.int64)
        if not bool((before(t[:, 0], t[:, 1]) & before(t[:, 1], t[:, 2])).all()):
            return False
    return True


def apex_counts(tri: torch.Tensor, n: int, chunk: int = 1 << 27) -> torch.Tensor:
    """Triangles per first vertex of the listing (bincount of column 0, in chunks, on the device)."""
    c = torch.zeros(n, dtype=torch.int64, device=tri.device)
    for s in range(0, tri.shape[0], chunk):
        c += torch.bincount(tri[s:s + chunk, 0].to(torch.int64), minlength=n)
    return c


def test_fullsize_orientation_is_exact(run, ref):
    tc, e, g, *_ = run
    assert equal_on_device(g.offsets, ref["off"])
    assert equal_on_device(g.dhat, ref["dhat"])
    assert equal_on_device(g.deg, ref["deg"])
    assert equal_on_device(g.cols, ref["cols"])


def test_fullsize_counts_are_exact(run, ref):
    tc, e, g, T, tv, cc, tri = run
    assert T == ref["T"]
    assert tc.count(g) == ref["T"]
    assert np.array_equal(tv.cpu().numpy(), ref["tv"])
    # C_v for every vertex, bit for bit (one correctly rounded division on both sides)
    ref_cc = oracle.clustering(ref["deg"], ref["tv"])
    assert np.array_equal(cc.cpu().numpy().view(np.uint64), ref_cc.view(np.uint64))


def test_fullsize_listing_is_exact(run, ref):
    tc, e, g, T, tv, cc, tri = run
    assert len(tri) == ref["T"]
    assert rows_strictly_increasing(tri)
    assert rows_oriented(tri, g.deg)
    ref_tri = par.listing(N, ref["off"], ref["cols"], ref["apex"])
    got = tri.cpu().numpy()
    rows = lambda t: t[np.lexsort((t[:, 2], t[:, 1], t[:, 0]))]
    assert np.array_equal(rows(got), rows(ref_tri))


def test_fullsize_sparsified_count(run, ref):
    tc, e, g, *_ = run
    t, mk, est = tc.sparsify_count(g, 0.1, 1)
    rt, rmk, rest = par.sparsify_count(N, e, ref["deg"], 1, 0.1)
    assert (t, mk) == (rt, rmk)
    assert est == rest
