"""The batched form (tc_batch) against the oracle and against one call per graph."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tc():
    from paper_1706_05151_gb300 import build
    build.build()
    import paper_1706_05151_gb300 as lib
    return lib


def mixed_graphs():
    gs = [
        (2000, synth.er(2000, 12000, 1)),
        (3000, synth.ba(3000, 12, 2)),
        (1 << 10, synth.rmat(10, 16, 3)),
        (5, np.zeros((0, 2), np.int32)),          # no edges
        (0, np.zeros((0, 2), np.int32)),          # no vertices
        (40, synth.complete(40)),
        (700, synth.complete(700)),               # lists longer than a tile
        (4, synth.wheel(3)),
        (1, np.zeros((0, 2), np.int32)),
    ]
    ns, ds = synth.batch_params(24, 77, nlo=100, nhi=5000)
    gs += [(int(n), synth.chung_lu(int(n), float(d), 2.1, 77, g)) for g, (n, d) in enumerate(zip(ns, ds))]
    return gs


def test_batch_matches_oracle_and_per_graph_calls(tc):
    graphs = mixed_graphs()
    b = tc.make_batch([(n, synth.shuffle_edges(e, i)) for i, (n, e) in enumerate(graphs)], "cuda")
    totals, tv, union = tc.batch(b)
    totals = totals.cpu().numpy()
    tv = tv.cpu().numpy()
    vbase = b.vbase.cpu().numpy()
    off = union.offsets.cpu().numpy()
    cols = union.cols.cpu().numpy()
    for g, (n, e) in enumerate(graphs):
        ref = oracle.count(n, e, local=True) if n > 0 else {"T": 0, "tv": np.zeros(0, np.int64)}
        assert totals[g] == ref["T"], g
        assert np.array_equal(tv[vbase[g]:vbase[g + 1]], ref["tv"]), g
        if n == 0:
            continue
        single = tc.orient(torch.from_numpy(np.ascontiguousarray(e)).cuda(), n)
        T1, tv1, _ = tc.count_local(single)
        assert T1 == ref["T"]
        # the union's lists of graph g are graph g's own lists, shifted by vbase[g]
        so = single.offsets.cpu().numpy()
        sc = single.cols.cpu().numpy()
        uo = off[vbase[g]:vbase[g + 1] + 1]
        assert np.array_equal(uo - uo[0], so)
        assert np.array_equal(cols[uo[0]:uo[-1]] - vbase[g], sc)


def test_batch_of_the_batched_configuration_shape(tc):
    # a slice of the 4096-graph Chung-Lu configuration (smaller n range)
    graphs = synth.batch_graphs(64, 2024, nhi=20000)
    b = tc.make_batch(graphs, "cuda")
    totals, tv, _ = tc.batch(b, local=False)
    assert tv is None
    totals = totals.cpu().numpy()
    for g in range(0, 64, 7):
        n, e = graphs[g]
        assert totals[g] == oracle.count(n, e)["T"]


def test_batch_rejects_bad_local_ids(tc):
    graphs = [(10, np.array([[0, 1], [1, 2]], np.int32)), (3, np.array([[0, 3]], np.int32))]
    b = tc.make_batch(graphs, "cuda")
    with pytest.raises(tc.TcError) as ex:
        tc.batch(b)
    assert ex.value.status == 2


def test_captured_batch_replays_match_plain_calls(tc):
    """tc_capture_begin/end around tc_batch: each replay equals a plain tc_batch on
    the buffers' current contents, including after the inputs are refilled in place."""
    graphs = mixed_graphs()
    b = tc.make_batch([(n, synth.shuffle_edges(e, i)) for i, (n, e) in enumerate(graphs)], "cuda")
    want_T, want_tv, _ = tc.batch(b)
    want_T, want_tv = want_T.clone(), want_tv.clone()
    cap = tc.CapturedBatch(b, local=True)
    assert cap.kernels > 0
    for _ in range(2):
        cap.totals.fill_(-1)
        cap.replay()
        torch.cuda.synchronize()
        T, tv, union = cap.result()
        assert torch.equal(T, want_T)
        assert torch.equal(tv, want_tv)
    tc.default_context().status()  # no device-side input error in the replays
    # refill in place: every graph relabelled by a random permutation of its own ids
    vbase = b.vbase.cpu().numpy()
    perm_edges = []
    perms = []
    for g, (n, e) in enumerate(graphs):
        p = np.random.default_rng(g).permutation(n).astype(np.int32) if n else np.zeros(0, np.int32)
        perms.append(p)
        perm_edges.append(synth.shuffle_edges(synth.relabel(e, p), 100 + g) if len(e) else e)
    b.edges.copy_(torch.from_numpy(np.concatenate([np.asarray(e, np.int32).reshape(-1, 2) for e in perm_edges])))
    cap.replay()
    torch.cuda.synchronize()
    T, tv, _ = cap.result()
    assert torch.equal(T, want_T)
    tv = tv.cpu().numpy()
    wtv = want_tv.cpu().numpy()
    for g, (n, _) in enumerate(graphs):
        if n:
            # vertex x of the original graph is vertex perms[g][x] of the relabelled one
            assert np.array_equal(tv[vbase[g] + perms[g]], wtv[vbase[g]:vbase[g + 1]]), g
    # a plain call on the refilled buffers agrees with the replay
    T2, tv2, _ = tc.batch(b)
    assert torch.equal(T2, cap.totals)
    assert np.array_equal(tv2.cpu().numpy(), tv)
    cap.close()


def test_capture_refuses_synchronizing_calls(tc):
    INVALID_ARG = 1
    ctx = tc.Context(0)
    g = tc.orient(torch.from_numpy(synth.complete(10)).cuda(), 10, ctx)
    s = torch.cuda.Stream()
    lib = ctx.lib
    sp = tc.ctypes.c_void_p(s.cuda_stream)
    assert lib.tc_capture_begin(ctx.handle, sp) == 0
    cnt = tc.ctypes.c_int64()
    ws = ctx.workspace(tc.TC_OP_LIST, g.n, g.m)
    st = lib.tc_list(ctx.handle, tc.ctypes.byref(g.struct()), None, 0, tc.ctypes.byref(cnt), tc._ptr(ws),
                     ws.numel(), sp)
    assert st == INVALID_ARG
    x = tc.ctypes.c_void_p()
    # the refused call spoils the capture: end reports it and returns no sequence
    assert lib.tc_capture_end(ctx.handle, sp, tc.ctypes.byref(x)) == INVALID_ARG
    # the context works normally afterwards
    assert tc.count(g, ctx) == 120
    ctx.close()


def test_host_memory_orientation_can_be_captured(tc):
    """tc_orient_host inside tc_capture_begin/end on a fresh context: the chunked copies
    (two chunks here) join the recorded sequence, and each replay reads the page-locked
    buffer as it is then -- refilled between replays with a relabelled graph of the same size."""
    ctx = tc.Context(0)
    n = 1 << 21
    e1 = synth.er(n, 20_000_000, 83)
    m = len(e1)
    perm = np.random.default_rng(84).permutation(n).astype(np.int32)
    e2 = np.ascontiguousarray(perm[e1])
    host = torch.from_numpy(e1.copy()).pin_memory()
    dev = torch.device("cuda")
    ed = torch.empty((m, 2), dtype=torch.int32, device=dev)
    offsets = torch.empty(n + 1, dtype=torch.int64, device=dev)
    cols = torch.empty(m, dtype=torch.int32, device=dev)
    deg = torch.empty(n, dtype=torch.int32, device=dev)
    dhat = torch.empty(n, dtype=torch.int32, device=dev)
    ws = ctx.workspace(tc.TC_OP_ORIENT, n, m)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    lib, P = ctx.lib, tc._ptr
    sp = tc.ctypes.c_void_p(s.cuda_stream)
    assert lib.tc_capture_begin(ctx.handle, sp) == 0
    st = lib.tc_orient_host(ctx.handle, n, m, host.data_ptr(), P(ed), P(offsets), P(cols), P(deg), P(dhat),
                            P(ws), ws.numel(), sp)
    x = tc.ctypes.c_void_p()
    assert lib.tc_capture_end(ctx.handle, sp, tc.ctypes.byref(x)) == 0 and st == 0
    try:
        for e in (e1, e2):
            host.copy_(torch.from_numpy(e))
            assert lib.tc_exec_launch(x, sp) == 0
            s.synchronize()
            ref = tc.orient(torch.from_numpy(e).cuda(), n, ctx)
            assert torch.equal(offsets, ref.offsets) and torch.equal(cols, ref.cols)
            assert torch.equal(deg, ref.deg) and torch.equal(dhat, ref.dhat)
    finally:
        lib.tc_exec_destroy(x)
        ctx.close()
