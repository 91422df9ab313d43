"""Pins of the parallel oracle: every function equals its serial counterpart.

The serial oracle is pinned by brute force, trace(A^3), closed forms and the
paper's printed values (test_oracle_pins.py); the parallel one is pinned to
it here, result by result, on the same kinds of graphs plus preferential
attachment and R-MAT graphs of 2^16 vertices, and on the rejection of
non-simple inputs.  Its listing fingerprint is pinned to a plain Python sum
over the serial oracle's triangle list and to the tensor restatement the
full-size GPU tests use.
"""
from __future__ import annotations

import itertools

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import par
from tests.fingerprint import listing_fingerprint


def _graphs():
    rng = np.random.default_rng(3)
    out = [("K9", 9, synth.complete(9)), ("wheel12", 13, synth.wheel(12)), ("cycle7", 7, synth.cycle(7)),
           ("star", 9, synth.star(8)), ("K4,5", 9, synth.complete_bipartite(4, 5)),
           ("empty", 5, np.zeros((0, 2), np.int32)),
           ("er", 600, synth.er(600, 6000, 11)), ("ba", 700, synth.ba(700, 6, 12)),
           ("rmat9", 1 << 9, synth.rmat(9, 16, 13)), ("cl", 800, synth.chung_lu(800, 24.0, 2.1, 14, 0)),
           ("ba16", 1 << 16, synth.ba(1 << 16, 16, 5)), ("rmat16", 1 << 16, synth.rmat(16, 16, 6))]
    for s in range(3):
        n = int(rng.integers(20, 60))
        p = float(rng.uniform(0.05, 0.5))
        e = np.array([(i, j) for i, j in itertools.combinations(range(n), 2) if rng.random() < p],
                     dtype=np.int32).reshape(-1, 2)
        out.append((f"gnp{s}", n, synth.shuffle_edges(e, s)))
    return out


GRAPHS = _graphs()


@pytest.mark.parametrize("name,n,e", GRAPHS, ids=[g[0] for g in GRAPHS])
def test_parallel_oracle_equals_serial(name, n, e):
    a = oracle.Adjacency(n, e)
    b = par.adjacency(n, e)
    assert np.array_equal(a.off, b.off) and np.array_equal(a.adj[:2 * a.m], b.adj[:2 * b.m])
    off, cols, dhat = a.orient()
    poff, pcols, pdhat = par.orient(b)
    assert np.array_equal(off, poff) and np.array_equal(cols, pcols) and np.array_equal(dhat, pdhat)
    s = a.count(local=True, listing=True)
    p = par.count(n, poff, pcols, local=True, fingerprint=True)
    assert p["T"] == s["T"]
    assert np.array_equal(p["tv"], s["tv"])
    # the serial oracle writes (v, u, w) with v first in the order: its first column is the apex
    assert np.array_equal(p["apex"], np.bincount(s["tri"][:, 0], minlength=n) if s["T"] else np.zeros(n))
    tri = par.listing(n, poff, pcols, p["apex"])
    # both write each triple as (v, u, w) in the order: equal as sets iff equal once rows are sorted
    rows = lambda t: t[np.lexsort((t[:, 2], t[:, 1], t[:, 0]))]
    assert np.array_equal(rows(tri), rows(s["tri"]))
    # fingerprint: the C sum, a plain Python sum over the serial listing, and the tensor form agree
    assert p["fp"] == listing_fingerprint(torch.from_numpy(s["tri"]))
    if s["T"] <= 5000:
        py = [0, 0]
        for v, u, w in s["tri"]:
            h = par.fingerprint_of(v, u, w)
            py = [(py[0] + h[0]) % par.FP_P, (py[1] + h[1]) % par.FP_P]
        assert p["fp"] == tuple(py)


@pytest.mark.parametrize("name,n,e", [g for g in GRAPHS if g[0] in ("ba", "rmat9", "cl", "ba16", "rmat16")],
                         ids=["ba", "rmat9", "cl", "ba16", "rmat16"])
def test_parallel_sparsify_equals_serial(name, n, e):
    deg = oracle.Adjacency(n, e).deg
    for seed, q in ((1, 0.1), (7, 0.5), (3, 1.0)):
        assert par.sparsify_count(n, e, deg, seed, q) == oracle.sparsify_count(n, e, seed, q)


def test_parallel_orientation_by_other_orders():
    n, e = 1 << 12, synth.rmat(12, 16, 9)
    a = oracle.Adjacency(n, e)
    for key in (np.zeros(n, np.int64), np.random.default_rng(2).integers(0, 1 << 40, n)):
        s = a.orient(key)
        p = par.orient(par.adjacency(n, e), key)
        assert all(np.array_equal(x, y) for x, y in zip(s, p))
        assert par.count(n, p[0], p[1])["T"] == a.count()["T"]  # Theorem 1


def test_fingerprint_hash_matches_its_definition():
    rng = np.random.default_rng(4)
    P = par.FP_P
    for v, u, w in rng.integers(0, 1 << 31, (200, 3)):
        for k in range(2):
            x = ((int(v) * par.FP_A[k]) % P + int(u)) % P
            x = ((x * par.FP_A[k]) % P + int(w)) % P
            y = (x * x + par.FP_B[k]) % P
            assert par.fingerprint_of(v, u, w)[k] == (y * y + par.FP_C[k]) % P


def test_fingerprint_separates_near_misses():
    # a listing that swaps the last vertices of two triples, or shifts one id, changes both sums
    n, e = 1 << 9, synth.rmat(9, 16, 13)
    tri = oracle.count(n, e, listing=True)["tri"].copy()
    base = listing_fingerprint(torch.from_numpy(tri))
    for i, j in ((0, 1), (5, 50), (10, len(tri) - 1)):
        t = tri.copy()
        t[i, 2], t[j, 2] = t[j, 2], t[i, 2]
        if not np.array_equal(t, tri):
            f = listing_fingerprint(torch.from_numpy(t))
            assert f[0] != base[0] and f[1] != base[1]
    t = tri.copy()
    t[3, 1] += 1
    f = listing_fingerprint(torch.from_numpy(t))
    assert f[0] != base[0] and f[1] != base[1]


@pytest.mark.parametrize("bad,code", [([[0, 1], [1, 1]], "self-loop"), ([[0, 1], [0, 9]], "vertex id"),
                                      ([[0, 1], [2, 3], [1, 0]], "repeated"), ([[0, -1]], "vertex id")])
def test_parallel_adjacency_rejects_non_simple_input(bad, code):
    e = np.array(bad, np.int32)
    with pytest.raises(oracle.OracleError, match=code):
        oracle.Adjacency(4, e)
    with pytest.raises(oracle.OracleError, match=code):
        par.adjacency(4, e)
