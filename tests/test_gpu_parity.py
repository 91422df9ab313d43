"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by element.

Every count here is an exact integer and must match bit for bit; C_v is one
IEEE division of exact operands on both sides and must match bit for bit too.
"""
from __future__ import annotations

import math

import numpy as np
import pytest
import torch

import oracle
import synth
from tests import brute

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    from paper_1706_05151_gb300 import build
    build.build()
    import paper_1706_05151_gb300 as lib
    return lib


def to_dev(e: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(e, dtype=np.int32)).cuda()


def check_orient(tc, n, e, g=None):
    adj = oracle.Adjacency(n, e)
    off, cols, dhat = adj.orient()
    g = g or tc.orient(to_dev(e), n)
    assert np.array_equal(g.offsets.cpu().numpy(), off)
    assert np.array_equal(g.cols.cpu().numpy(), cols)
    assert np.array_equal(g.deg.cpu().numpy(), adj.deg)
    assert np.array_equal(g.dhat.cpu().numpy(), dhat)
    return adj, g


def check_all(tc, n, e, listing=True):
    """Orientation, T, T_v, C_v and listing against the oracle."""
    adj, g = check_orient(tc, n, e)
    ref = adj.count(local=True, listing=listing)
    assert tc.count(g) == ref["T"]
    T, tv, cc = tc.count_local(g)
    assert T == ref["T"]
    assert np.array_equal(tv.cpu().numpy(), ref["tv"])
    ref_cc = oracle.clustering(adj.deg, ref["tv"])
    assert np.array_equal(cc.cpu().numpy().view(np.uint64), ref_cc.view(np.uint64))
    T2, tv2, cc2, tri2 = tc.analyze(g)
    assert T2 == ref["T"]
    assert np.array_equal(tv2.cpu().numpy(), ref["tv"])
    assert np.array_equal(cc2.cpu().numpy().view(np.uint64), ref_cc.view(np.uint64))
    assert len(tri2) == ref["T"]
    if listing:
        tri = tc.list_triangles(g).cpu().numpy()
        assert len(tri) == ref["T"]
        t2 = tri2.cpu().numpy()
        assert np.array_equal(t2[np.lexsort((t2[:, 2], t2[:, 1], t2[:, 0]))] if len(t2) else t2,
                              tri[np.lexsort((tri[:, 2], tri[:, 1], tri[:, 0]))] if len(tri) else tri)
        # both sides emit (v, u, w) with v < u < w in the order: compare the row sets
        a = tri[np.lexsort((tri[:, 2], tri[:, 1], tri[:, 0]))] if len(tri) else tri
        r = ref["tri"]
        b = r[np.lexsort((r[:, 2], r[:, 1], r[:, 0]))] if len(r) else r
        assert np.array_equal(a, b)
    return g, ref


# ---- closed forms and degenerate inputs -------------------------------------------

@pytest.mark.parametrize("n", [3, 4, 5, 17, 40, 300, 700])
def test_complete(tc, n):
    g, ref = check_all(tc, n, synth.complete(n), listing=n <= 300)
    assert ref["T"] == math.comb(n, 3)


@pytest.mark.parametrize("make,n", [
    (lambda: synth.cycle(1000), 1000), (lambda: synth.wheel(3), 4), (lambda: synth.wheel(1000), 1001),
    (lambda: synth.star(5000), 5001), (lambda: synth.complete_bipartite(40, 60), 100),
    (lambda: synth.random_tree(20000, 5), 20000),
])
def test_closed_forms(tc, make, n):
    check_all(tc, n, make())


def test_empty_graphs(tc):
    for n in [0, 1, 7]:
        e = np.zeros((0, 2), np.int32)
        g = tc.orient(torch.zeros((0, 2), dtype=torch.int32, device="cuda"), n)
        assert tc.count(g) == 0
        T, tv, _ = tc.count_local(g)
        assert T == 0 and (n == 0 or int(tv.abs().sum()) == 0)
        assert len(tc.list_triangles(g)) == 0
        assert tc.sparsify_count(g, 0.5, 1)[:2] == (0, 0)


def test_ids_beyond_one_degree_pass(tc):
    # about 50M vertex ids with 320k edges: hubs and planted triangles at ids around
    # 2^24 and 2^25 and at the last id; the oracle's CSR and counts
    n = 3 * (1 << 24) + 12345
    rng = np.random.default_rng(41)
    hubs = np.array([0, (1 << 24) - 1, 1 << 24, (2 << 24) + 7, n - 1], dtype=np.int64)
    tri = np.concatenate([rng.integers(0, n, (3000, 3)), np.array([[0, 1 << 24, n - 1], [(1 << 24) - 1, 1 << 24,
                                                                                      (2 << 24) + 7]])])
    a = np.concatenate([rng.integers(0, n, 300000), np.repeat(hubs, 2000), tri[:, 0], tri[:, 1], tri[:, 0],
                        np.repeat(hubs, 4)])
    b = np.concatenate([rng.integers(0, n, 300000), rng.integers(0, n, 10000), tri[:, 1], tri[:, 2], tri[:, 2],
                        np.tile(hubs, 4)])
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    keep = lo != hi
    e = np.unique(np.stack([lo[keep], hi[keep]], axis=1), axis=0).astype(np.int32)
    e = synth.shuffle_edges(e, 42)
    check_all(tc, n, e)


@pytest.mark.parametrize("make", [
    lambda: (1 << 20, synth.ba(1 << 20, 16, 45)),
    lambda: ((1 << 20) + 777, synth.er((1 << 20) + 777, 6_000_000, 46)),   # a ragged last bucket
    lambda: (1 << 20, synth.shuffle_edges(synth.rmat(20, 16, 47), 48)),    # any edge order and direction
])
def test_orientation_at_a_million_vertices(tc, make):
    # n >= 2^20 with mean degree >= 8, a ragged vertex count, and a shuffled edge order
    from oracle import par
    n, e = make()
    adj, g = check_orient(tc, n, e)
    off, cols, _ = adj.orient()
    assert tc.count(g) == par.count(n, off, cols, local=False)["T"]


def _top_and_bottom_ids(n, seed):
    # 60k random edges among the first and the last 40k ids, plus triangles across them
    rng = np.random.default_rng(seed)
    ids = np.concatenate([np.arange(40000), np.arange(n - 40000, n)])
    a, b = ids[rng.integers(0, len(ids), 60000)], ids[rng.integers(0, len(ids), 60000)]
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    keep = lo != hi
    return synth.shuffle_edges(np.unique(np.stack([lo[keep], hi[keep]], axis=1), axis=0).astype(np.int32), seed)


@pytest.mark.parametrize("make", [
    lambda: (1 << 27, _top_and_bottom_ids(1 << 27, 67)),
    lambda: ((1 << 27) + 1, _top_and_bottom_ids((1 << 27) + 1, 68)),
    lambda: ((1 << 23) + 5, synth.shuffle_edges(synth.er((1 << 23) + 5, 2_000_000, 70), 71)),
])
def test_orientation_over_large_id_ranges(tc, make):
    # sparse graphs whose ids span up to 2^27 + 1 vertices: the whole CSR, d_v and dhat_v, and T
    n, e = make()
    adj, g = check_orient(tc, n, e)
    assert tc.count(g) == adj.count()["T"]
    del g
    torch.cuda.empty_cache()


@pytest.mark.parametrize("make", [
    lambda: (1 << 21, synth.er(1 << 21, 20_000_000, 72)),                 # two copy chunks, the second ragged
    lambda: (1 << 14, synth.shuffle_edges(synth.rmat(14, 16, 73), 74)),   # one chunk
    lambda: (300, synth.complete(300)),
    lambda: (9, np.zeros((0, 2), np.int32)),
])
def test_orientation_from_host_memory(tc, make):
    # tc_orient_host gives the same CSR, d_v and dhat_v as tc_orient, and leaves the edges on the device
    n, e = make()
    host = torch.from_numpy(np.ascontiguousarray(e, dtype=np.int32)).pin_memory()
    g, ed = tc.orient_host(host, n)
    ref = tc.orient(to_dev(e), n)
    for a, b in ((g.offsets, ref.offsets), (g.cols, ref.cols), (g.deg, ref.deg), (g.dhat, ref.dhat)):
        assert torch.equal(a, b)
    assert torch.equal(ed.cpu(), host)
    if len(e) < 10 ** 6:
        check_orient(tc, n, e, g)
    # a second call reuses the device buffer
    g2, ed2 = tc.orient_host(host, n, edges_dev=ed)
    assert ed2.data_ptr() == ed.data_ptr() and torch.equal(g2.cols, ref.cols)


def test_orientation_from_host_memory_reports_errors(tc):
    e = synth.er(1 << 21, 20_000_000, 75)
    bad = e.copy()
    bad[-5] = (7, 1 << 21)  # an id outside [0, n) in the second chunk
    with pytest.raises(tc.TcError) as ex:
        tc.orient_host(torch.from_numpy(bad).pin_memory(), 1 << 21)
    assert ex.value.status == 2
    with pytest.raises(tc.TcError) as ex:  # pageable host memory is refused before anything is queued
        tc.orient_host(torch.from_numpy(e[:1000].copy()), 1 << 21)
    assert ex.value.status == 1
    g, _ = tc.orient_host(torch.from_numpy(e).pin_memory(), 1 << 21)  # the context is still usable
    assert int(g.dhat.sum()) == len(e)


def test_single_triangle_with_isolated_vertices(tc):
    check_all(tc, 10, np.array([[5, 2], [2, 9], [9, 5]], np.int32))


# ---- the paper's workload classes at oracle-friendly sizes ----------------------------

def test_erdos_renyi_config(tc):
    # G(n = 16384, M = 131072 draws): the small single-graph configuration
    n = 16384
    check_all(tc, n, synth.er(n, 131072, 1))


@pytest.mark.parametrize("n,k,seed", [(1 << 14, 16, 2), (100003, 16, 3), (5000, 40, 4)])
def test_preferential_attachment(tc, n, k, seed):
    check_all(tc, n, synth.shuffle_edges(synth.ba(n, k, seed), seed))


@pytest.mark.parametrize("scale,ef,seed", [(12, 16, 5), (14, 16, 6), (15, 8, 7)])
def test_rmat(tc, scale, ef, seed):
    check_all(tc, 1 << scale, synth.rmat(scale, ef, seed))


@pytest.mark.parametrize("n,dbar,seed", [(20000, 48.0, 8), (3000, 64.0, 9)])
def test_chung_lu(tc, n, dbar, seed):
    check_all(tc, n, synth.chung_lu(n, dbar, 2.1, seed, 0))


def test_dense_graph_uses_block_kernel(tc):
    # lists longer than one tile (512 ids) go to the block kernel
    rng = np.random.default_rng(10)
    n = 1400
    iu = np.triu_indices(n, 1)
    keep = rng.random(len(iu[0])) < 0.8
    e = np.stack([iu[0][keep], iu[1][keep]], axis=1).astype(np.int32)
    g, ref = check_all(tc, n, synth.shuffle_edges(e, 10), listing=False)
    assert int(g.dhat.max()) > 512


def test_chunked_block_kernel_on_large_clique(tc):
    # K_n with n > 8193: N_v longer than two shared-memory chunks (4096 ids) and
    # sorted by the block sorter; closed forms T = C(n,3), T_v = C(n-1,2), C_v = 1
    n = 8300
    e = synth.shuffle_edges(synth.complete(n), 11)
    g = tc.orient(to_dev(e), n)
    assert int(g.dhat.max()) == n - 1
    off = g.offsets.cpu().numpy()
    cols = g.cols.cpu().numpy()
    assert np.all(np.diff(cols[off[0]:off[1]]) > 0)
    assert tc.count(g) == math.comb(n, 3)
    T, tv, cc = tc.count_local(g)
    assert T == math.comb(n, 3)
    assert torch.all(tv == math.comb(n - 1, 2))
    assert torch.all(cc == 1.0)


# ---- invariants --------------------------------------------------------------------

def test_relabel_and_edge_order_invariance(tc):
    n = 1 << 13
    e = synth.rmat(13, 16, 12)
    perm = np.random.default_rng(12).permutation(n).astype(np.int32)
    g1 = tc.orient(to_dev(e), n)
    g2 = tc.orient(to_dev(synth.relabel(e, perm)), n)
    g3 = tc.orient(to_dev(synth.shuffle_edges(e, 13)), n)
    T1, tv1, _ = tc.count_local(g1)
    T2, tv2, _ = tc.count_local(g2)
    assert T1 == T2
    assert np.array_equal(tv2.cpu().numpy()[perm], tv1.cpu().numpy())
    assert torch.equal(g1.offsets, g3.offsets) and torch.equal(g1.cols, g3.cols)
    assert int(tv1.sum()) == 3 * T1


def test_repeated_runs_are_identical(tc):
    n = 1 << 14
    g = tc.orient(to_dev(synth.rmat(14, 16, 14)), n)
    a = tc.count_local(g)
    b = tc.count_local(g)
    assert a[0] == b[0] and torch.equal(a[1], b[1])
    t1 = tc.list_triangles(g)
    t2 = tc.list_triangles(g)
    # every triangle is written at a fixed position (its edge's offset plus its rank)
    assert torch.equal(t1, t2)
    T, _, _, t3 = tc.analyze(g)
    assert torch.equal(t1, t3)


# ---- sparsification (Section 9.1) -----------------------------------------------------

@pytest.mark.parametrize("q,seed", [(0.1, 1), (0.1, 2), (0.3, 3), (0.5, 4), (1.0, 5), (0.0, 6)])
def test_sparsify_matches_oracle(tc, q, seed):
    n = 1 << 14
    e = synth.rmat(14, 16, 15)
    g = tc.orient(to_dev(e), n)
    t, mk, est = tc.sparsify_count(g, q, seed)
    rt, rmk, rest = oracle.sparsify_count(n, e, seed, q)
    assert (t, mk) == (rt, rmk)
    if q > 0:
        assert est == rest


def test_sparsify_q_one_is_exact(tc):
    n = 1 << 12
    e = synth.ba(n, 16, 16)
    g = tc.orient(to_dev(e), n)
    t, mk, _ = tc.sparsify_count(g, 1.0, 123)
    assert mk == len(e) and t == tc.count(g)


@pytest.mark.parametrize("make,n", [
    (lambda: synth.er(1000, 6000, 31), 1000),              # n not a multiple of 32 or 64, isolated vertices
    (lambda: synth.chung_lu(3001, 24.0, 2.1, 32), 3001),   # skewed degrees: long lists beside empty ones
    (lambda: synth.complete(70), 70),                      # lists of 0 .. 69 ids, every edge in triangles
    (lambda: synth.wheel(130), 131),                       # hub of degree 130 last in the order
    (lambda: np.zeros((0, 2), np.int32), 65),              # no edges at all
])
@pytest.mark.parametrize("q", [0.05, 0.5])
def test_sparsify_ragged_sizes(tc, make, n, q):
    # the marking pass walks 32-vertex runs and the compaction 64-vertex runs:
    # sizes that end mid-run, empty lists and long lists must all match the oracle
    e = make()
    g = tc.orient(to_dev(e), n)
    for seed in (3, 4):
        t, mk, _ = tc.sparsify_count(g, q, seed)
        rt, rmk, _ = oracle.sparsify_count(n, e, seed, q)
        assert (t, mk) == (rt, rmk)


# ---- error handling -----------------------------------------------------------------

def test_invalid_graphs_are_reported(tc):
    bad = {
        "self-loop": (np.array([[0, 1], [2, 2]], np.int32), 3),
        "repeated": (np.array([[0, 1], [1, 0]], np.int32), 3),
        "out of range": (np.array([[0, 5]], np.int32), 3),
        "negative": (np.array([[0, -1]], np.int32), 3),
    }
    for what, (e, n) in bad.items():
        with pytest.raises(tc.TcError) as ex:
            tc.orient(to_dev(e), n)
        assert ex.value.status == 2, what


def test_repeated_edge_in_long_list_is_reported(tc):
    n = 600
    e = synth.complete(n)
    e = np.concatenate([e, e[-1:][:, ::-1]])  # the last edge again, reversed
    with pytest.raises(tc.TcError) as ex:
        tc.orient(to_dev(e), n)
    assert ex.value.status == 2


def test_workspace_and_capacity_errors(tc):
    import ctypes
    n = 1 << 10
    g = tc.orient(to_dev(synth.complete(40)), 40)
    ctx = tc.default_context()
    small = torch.empty(256, dtype=torch.uint8, device="cuda")
    total = torch.empty(1, dtype=torch.int64, device="cuda")
    st = ctx.lib.tc_count(ctx.handle, ctypes.byref(g.struct()), ctypes.c_void_p(total.data_ptr()),
                          ctypes.c_void_p(small.data_ptr()), 16, None)
    assert st == 3
    tri = torch.empty((10, 3), dtype=torch.int32, device="cuda")
    with pytest.raises(tc.TcError) as ex:
        tc.list_triangles_into(g, tri)
    assert ex.value.status == 4
    big = torch.empty((math.comb(40, 3), 3), dtype=torch.int32, device="cuda")
    assert tc.list_triangles_into(g, big) == math.comb(40, 3)
    with pytest.raises(tc.TcError) as ex:
        tc.sparsify_count(g, 1.5, 0)
    assert ex.value.status == 1
    del n


def test_broken_csr_is_reported_not_read(tc):
    # offsets pointing past m must give TC_ERR_INVALID_GRAPH, not an out-of-bounds read
    off = torch.tensor([0, 2, 50, 3], dtype=torch.int64, device="cuda")
    cols = torch.tensor([1, 2, 2], dtype=torch.int32, device="cuda")
    g = tc.graph_from_csr(off, cols)
    with pytest.raises(tc.TcError) as ex:
        tc.count(g)
    assert ex.value.status == 2
    cols_bad = torch.tensor([1, 7, 2], dtype=torch.int32, device="cuda")
    g2 = tc.graph_from_csr(torch.tensor([0, 2, 3, 3], dtype=torch.int64, device="cuda"), cols_bad)
    with pytest.raises(tc.TcError) as ex:
        tc.count(g2)
    assert ex.value.status == 2


# ---- tuning never changes results ---------------------------------------------------

@pytest.mark.parametrize("make", [
    lambda: (1 << 14, synth.rmat(14, 16, 40)),
    lambda: (700, synth.complete(700)),
    lambda: (20000, synth.chung_lu(20000, 48.0, 2.1, 41, 0)),
])
def test_results_independent_of_tuning(tc, make):
    n, e = make()
    ctx = tc.default_context()
    g = tc.orient(to_dev(e), n)
    ref = oracle.count(n, e, local=True)
    try:
        for tile_max, grid_div in [(32, 1), (128, 3), (512, 1), (1, 2)]:
            ctx.set_tuning(tile_max, grid_div)
            T, tv, cc, tri = tc.analyze(g)
            assert T == ref["T"] and np.array_equal(tv.cpu().numpy(), ref["tv"])
            assert len(tri) == T
            assert tc.count(g) == T
            assert tc.sparsify_count(g, 0.3, 5)[:2] == oracle.sparsify_count(n, e, 5, 0.3)[:2]
    finally:
        ctx.set_tuning(0, 1)


@pytest.mark.parametrize("make", [
    lambda: (1 << 14, synth.rmat(14, 16, 43)),
    lambda: (900, synth.complete(900)),          # every apex list in the block kernel, in chunks
    lambda: (1 << 15, synth.ba(1 << 15, 16, 44)),
])
def test_results_independent_of_kernel_shape(tc, make):
    # every instantiation of the tile kernel (ids x windows) and of the hash kernels (batch x windows),
    # with the hub side on and off: identical T, T_v and triangle list
    n, e = make()
    ctx = tc.default_context()
    g = tc.orient(to_dev(e), n)
    ref = oracle.count(n, e, local=True, listing=True)

    def row_keys(t: torch.Tensor) -> torch.Tensor:
        # each triple as one int64 (n < 2^21), sorted on the device: equal iff the row sets are
        t = t.to(torch.int64)
        return torch.sort((t[:, 0] * n + t[:, 1]) * n + t[:, 2]).values
    ref_keys = row_keys(torch.from_numpy(ref["tri"]).cuda())
    try:
        for (ids, windows) in ((256, 8), (256, 4), (128, 8)):
            for hb, hw in ((32, 4), (16, 4), (32, 8), (16, 8)):
                for hub in (0, -1):
                    ctx.set_kernel_shape(ids, windows, hb, hw)
                    ctx.set_hub_min(hub)
                    T, tv, cc, tri = tc.analyze(g)
                    assert T == ref["T"] and np.array_equal(tv.cpu().numpy(), ref["tv"]), (ids, windows, hb, hw, hub)
                    assert torch.equal(row_keys(tri), ref_keys)
                    assert tc.count(g) == T
    finally:
        ctx.set_kernel_shape(0, 0, 0, 0)
        ctx.set_hub_min(0)


def test_kernel_shape_refuses_unknown_shapes(tc):
    ctx = tc.default_context()
    for bad in ((512, 8, 32, 4), (256, 2, 32, 4), (256, 8, 8, 4), (128, 4, 0, 0), (256, 8, 32, 6)):
        with pytest.raises(tc.TcError):
            ctx.set_kernel_shape(*bad)
    ctx.set_kernel_shape(0, 0, 0, 0)


def test_autotuner_records_a_candidate(tc, tmp_path):
    from paper_1706_05151_gb300 import autotune
    n = 1 << 13
    g = tc.orient(to_dev(synth.rmat(13, 16, 42)), n)
    path = str(tmp_path / "tuning.json")
    try:
        best, times, hub, hub_times = autotune.tune(g, repeats=1, path=path)
        assert best in autotune.CANDIDATES and set(times) == set(autotune.CANDIDATES)
        assert hub in autotune.HUB_CANDIDATES and set(hub_times) == set(autotune.HUB_CANDIDATES)
        assert autotune.apply(g, path=path) == (best, hub)
        assert autotune.shape_class(g) in autotune.load_table(path)
        assert tc.count(g) == oracle.count(n, synth.rmat(13, 16, 42))["T"]
    finally:
        tc.default_context().set_tuning(0, 1)
        tc.default_context().set_hub_min(0)
        tc.default_context().set_kernel_shape(0, 0, 0, 0)


def test_listing_of_lists_longer_than_one_hash_chunk(tc):
    # K_2100: the write pass hashes N_v (up to 2099 ids) in two chunks of 2048;
    # every triangle must be listed once, in the same order every run.  All
    # degrees are equal, so the order is by id and each triple is v < u < w.
    n = 2100
    e = synth.shuffle_edges(synth.complete(n), 12)
    g = tc.orient(to_dev(e), n)
    T, tv, cc, tri = tc.analyze(g)
    assert T == math.comb(n, 3) and len(tri) == T
    t = tri.to(torch.int64)
    assert bool(torch.all((t[:, 0] < t[:, 1]) & (t[:, 1] < t[:, 2])))
    key = (t[:, 0] * n + t[:, 1]) * n + t[:, 2]
    del t
    key = torch.sort(key).values
    assert bool(torch.all(key[1:] > key[:-1]))  # all distinct, so all C(n, 3) present
    del key
    assert torch.equal(tc.list_triangles(g), tri)


def test_csr_in_host_memory(tc):
    """A CSR held in page-locked host memory is read over the CPU-GPU link: same results."""
    n, e = 1 << 14, synth.rmat(14, 16, 21)
    g = tc.orient(to_dev(e), n)
    T, tv, cc = tc.count_local(g)
    h = tc.Graph(n, g.m, g.offsets.cpu().pin_memory(), g.cols.cpu().pin_memory(), g.deg.cpu().pin_memory(),
                 g.dhat.cpu().pin_memory())
    T2, tv2, cc2 = tc.count_local(h)
    assert T2 == T
    assert torch.equal(tv2, tv) and torch.equal(cc2, cc)
    assert tc.count(h) == T
