"""tc_count_static, the counting entry point for callers that cannot allocate.

Some callers cannot call cudaMalloc: their device memory belongs to another
allocator, or they run on a path where an allocation would synchronize the
device.  tc_count_static keeps its scratch in a fixed file-scope device array
instead of a caller workspace.  This file checks it through the C ABI against
tc_count and the CPU oracle on the same graphs, on two calls in a row (the
second call reuses the array the first one left behind), that a warm call
takes no device memory, that the kernels' input checks still reach check_dev,
and that misaligned pointers are refused before anything is enqueued.  It is
collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

STATIC_MAX_N = 1 << 20


@pytest.fixture(scope="module")
def tc():
    from paper_1706_05151_gb300 import build
    build.build()
    import paper_1706_05151_gb300 as lib
    raw = ctypes.CDLL(lib.LIB_PATH)
    raw.tc_count_static.restype = ctypes.c_int32
    raw.tc_count_static.argtypes = [ctypes.POINTER(lib.TcGraph), ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p]
    lib._static_fn = raw.tc_count_static
    return lib


def call_static(tc, g, total, check):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    gs = g.struct()
    return tc._static_fn(ctypes.byref(gs), ctypes.c_void_p(total.data_ptr()), ctypes.c_void_p(check.data_ptr()),
                         stream)


@pytest.mark.parametrize("make", [
    lambda: (1 << 14, synth.rmat(14, 16, 31)),
    lambda: (1 << 16, synth.ba(1 << 16, 16, 32)),
    lambda: (700, synth.complete(700)),          # lists longer than a tile: the block kernel's queue
    lambda: (STATIC_MAX_N, synth.er(STATIC_MAX_N, 4 * STATIC_MAX_N, 33)),
])
def test_static_count_matches_tc_count_twice(tc, make):
    n, e = make()
    g = tc.orient(torch.from_numpy(np.ascontiguousarray(e)).cuda(), n)
    expected = tc.count(g)
    assert expected == oracle.count(n, e)["T"]
    total = torch.empty(1, dtype=torch.int64, device="cuda")
    check = torch.empty(1, dtype=torch.int32, device="cuda")
    for _ in range(2):
        total.fill_(-1)
        check.fill_(-1)
        assert call_static(tc, g, total, check) == 0
        torch.cuda.synchronize()
        assert int(check.item()) == 0
        assert int(total.item()) == expected


def test_static_count_rejects_graphs_above_the_limit(tc):
    n = STATIC_MAX_N + 1
    off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    cols = torch.zeros(1, dtype=torch.int32, device="cuda")
    g = tc.graph_from_csr(off, cols[:0])
    total = torch.zeros(1, dtype=torch.int64, device="cuda")
    check = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert call_static(tc, g, total, check) == 6  # TC_ERR_UNSUPPORTED, nothing launched


def test_static_count_takes_no_device_memory(tc):
    n, e = 1 << 14, synth.rmat(14, 16, 34)
    g = tc.orient(torch.from_numpy(e).cuda(), n)
    total = torch.empty(1, dtype=torch.int64, device="cuda")
    check = torch.empty(1, dtype=torch.int32, device="cuda")
    assert call_static(tc, g, total, check) == 0  # loads the kernels and looks up the array once
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert call_static(tc, g, total, check) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert int(total.item()) == oracle.count(n, e)["T"]


def test_static_count_reports_bad_ids_in_check(tc):
    # N_0 = {1, 2}, N_1 = {2, 9}: id 9 is outside [0, 4)
    off = torch.tensor([0, 2, 4, 4, 4], dtype=torch.int64, device="cuda")
    cols = torch.tensor([1, 2, 2, 9], dtype=torch.int32, device="cuda")
    g = tc.graph_from_csr(off, cols)
    total = torch.zeros(1, dtype=torch.int64, device="cuda")
    check = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert call_static(tc, g, total, check) == 0
    torch.cuda.synchronize()
    assert int(check.item()) & 1  # the bad-id bit


def test_static_count_refuses_misaligned_pointers(tc):
    n, e = 1 << 10, synth.rmat(10, 8, 35)
    g = tc.orient(torch.from_numpy(e).cuda(), n)
    buf = torch.full((4,), -1, dtype=torch.int64, device="cuda")
    check = torch.full((2,), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    gs = g.struct()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def raw(gs, total_ptr, check_ptr):
        return tc._static_fn(ctypes.byref(gs), ctypes.c_void_p(total_ptr), ctypes.c_void_p(check_ptr), stream)
    bad_off = tc.TcGraph(gs.n, gs.m, gs.offsets + 4, gs.cols, gs.deg, gs.dhat)
    assert raw(bad_off, buf.data_ptr(), check.data_ptr()) == 1
    assert raw(gs, buf.data_ptr() + 4, check.data_ptr()) == 1
    assert raw(gs, buf.data_ptr(), check.data_ptr() + 2) == 1
    torch.cuda.synchronize()
    assert bool((buf == -1).all()) and bool((check == -1).all())  # nothing was enqueued
