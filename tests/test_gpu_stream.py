"""Counting an oriented CSR held in host memory (tc_count_streamed), against the oracle.

The list buffer is made deliberately small, so that the lists are cut into
several resident target ranges and many streamed apex chunks (and the two
copy slots are reused many times); T and every T_v must still equal the
oracle's, for any buffer size, and a buffer too small for the longest list is
refused before anything is copied.
"""
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


def host_csr(tc, n, e):
    g = tc.orient(torch.from_numpy(np.ascontiguousarray(e)).cuda(), n)
    return g, g.offsets.cpu().pin_memory(), g.cols.cpu().pin_memory()


@pytest.mark.parametrize("make,fractions", [
    (lambda: (1 << 16, synth.ba(1 << 16, 16, 51)), (0.02, 0.1, 0.37, 4.0)),
    (lambda: (1 << 14, synth.rmat(14, 16, 52)), (0.08, 0.3, 1.0)),        # hub lists: the block kernel's queue
    (lambda: (20000, synth.chung_lu(20000, 48.0, 2.1, 53, 0)), (0.05, 0.5)),
    (lambda: (900, synth.complete(900)), (0.9, 3.0)),                    # 899-id lists, apex lists of the block kernel
])
def test_streamed_count_equals_oracle(tc, make, fractions):
    n, e = make()
    ref = oracle.count(n, e, local=True)
    g, off_h, cols_h = host_csr(tc, n, e)
    longest = int((g.offsets[1:] - g.offsets[:-1]).max().item())
    for f in fractions:
        # list buffer: f times the CSR's ids, but at least 4 quarters of the longest list
        list_bytes = max(int(f * 4 * g.m), 4 * 4 * (longest + 64))
        T, tv = tc.count_streamed(off_h, cols_h, list_bytes, local=True)
        assert T == ref["T"], f
        assert np.array_equal(tv.cpu().numpy(), ref["tv"]), f
        assert tc.count_streamed(off_h, cols_h, list_bytes)[0] == ref["T"]


def test_streamed_count_of_empty_and_edgeless_graphs(tc):
    off = torch.zeros(11, dtype=torch.int64).pin_memory()
    cols = torch.zeros(0, dtype=torch.int32).pin_memory()
    T, tv = tc.count_streamed(off, cols, 1 << 16, local=True)
    assert T == 0 and int(tv.abs().sum().item()) == 0


def test_streamed_count_refuses_a_buffer_smaller_than_a_list(tc):
    n, e = 300, synth.complete(300)
    g, off_h, cols_h = host_csr(tc, n, e)
    with pytest.raises(tc.TcError) as ex:
        tc.count_streamed(off_h, cols_h, 4 * 4 * 200)  # a quarter holds 200 ids; the longest list has 299
    assert ex.value.status == 3  # TC_ERR_WORKSPACE


def test_streamed_count_refuses_inconsistent_offsets(tc):
    n, e = 1 << 10, synth.rmat(10, 8, 54)
    g, off_h, cols_h = host_csr(tc, n, e)
    bad = off_h.clone()
    bad[-1] = g.m + 5  # does not end at m: the copies would read past cols
    with pytest.raises(tc.TcError) as ex:
        tc.count_streamed(bad.pin_memory(), cols_h, 1 << 20)
    assert ex.value.status == 2  # TC_ERR_INVALID_GRAPH


def test_streamed_count_at_two_million_edges_several_ranges(tc):
    n, e = 1 << 18, synth.ba(1 << 18, 8, 55)
    g, off_h, cols_h = host_csr(tc, n, e)
    expected = tc.count(g)
    T, tv = tc.count_streamed(off_h, cols_h, g.m, local=True)  # a buffer of a quarter of the CSR
    T2, tv2, _ = tc.count_local(g)
    assert T == expected == T2
    assert torch.equal(tv, tv2)
