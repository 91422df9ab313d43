"""Sanity checks of the seeded input generators (shared by oracle and CUDA tests)."""
import math

import numpy as np
import pytest

import synth


def assert_simple(n, e):
    assert e.dtype == np.int32 and e.ndim == 2 and e.shape[1] == 2
    if len(e) == 0:
        return
    assert e.min() >= 0 and e.max() < n
    assert np.all(e[:, 0] != e[:, 1])
    lo, hi = e.min(axis=1).astype(np.int64), e.max(axis=1).astype(np.int64)
    keys = lo * n + hi
    assert len(np.unique(keys)) == len(keys)


@pytest.mark.parametrize("make,n", [
    (lambda: synth.er(1000, 5000, 1), 1000),
    (lambda: synth.ba(5000, 16, 2), 5000),
    (lambda: synth.rmat(12, 16, 3), 4096),
    (lambda: synth.chung_lu(3000, 30.0, 2.1, 4, 9), 3000),
])
def test_generators_give_simple_graphs(make, n):
    e = make()
    assert_simple(n, e)
    assert np.array_equal(e, make())          # same seed, same graph


def test_ba_edge_count_and_shape():
    n, k = 20000, 16
    e = synth.ba(n, k, 5)
    full = k * (k - 1) // 2 + (n - k) * k
    assert full - len(e) < 0.01 * full        # few repeated targets merged
    deg = np.bincount(e.ravel(), minlength=n)
    assert deg[k:].min() >= 1 and deg.max() > 20 * k   # heavy tail
    assert np.all(e[:, 0] < e[:, 1])


def test_ba_rejects_k_one():
    with pytest.raises(RuntimeError):
        synth.ba(100, 1, 0)


def test_er_triangle_free_cases_and_counts():
    e = synth.er(16384, 131072, 1)
    assert 130000 < len(e) <= 131072


def test_batch_params_ranges():
    ns, ds = synth.batch_params(4096, 7)
    assert ns.min() >= 100 and ns.max() <= 100000
    assert ds.min() >= 8 and ds.max() <= 64
    # log-uniform: the median sits near the geometric mean sqrt(100 * 1e5)
    assert 2000 < np.median(ns) < 6000


def test_closed_form_fixtures():
    assert len(synth.complete(6)) == 15
    assert len(synth.wheel(5)) == 10
    assert len(synth.cycle(7)) == 7
    assert len(synth.complete_bipartite(3, 4)) == 12
    assert len(synth.random_tree(50, 1)) == 49
    e = synth.shuffle_edges(synth.complete(10), 3)
    assert_simple(10, e)
