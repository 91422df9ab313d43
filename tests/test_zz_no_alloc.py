"""tc_count_static, the counting entry point for callers that cannot allocate.

Some callers cannot call cudaMalloc: their device memory belongs to another
allocator, or they run on a path where an allocation would synchronize the
device.  tc_count_static keeps its scratch in a fixed file-scope device array
instead of a caller workspace.  This file checks it through the C ABI against
tc_count on the same graphs, on two calls in a row (the second call reuses the
array the first one left behind).  It is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

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
