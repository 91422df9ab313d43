"""Orientation by other total orders (tc_orient_by): the CSR equals the
oracle's for the same order, T and T_v do not depend on the order (Theorem 1),
and the degree order has the smallest counting cost sum_v d_v * dhat_v
(Theorem 3)."""
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


def orders(n, deg, seed):
    rng = np.random.default_rng(seed)
    return {
        "id": np.zeros(n, np.int64),
        "degree": deg.astype(np.int64),
        "random": rng.permutation(n).astype(np.int64),
        "reverse_degree": -deg.astype(np.int64),
        "coarse": (deg.astype(np.int64) // 4),  # many ties, broken by id
    }


@pytest.mark.parametrize("name,n,e", [
    ("er", 3000, synth.er(3000, 40000, 1)),
    ("ba", 5000, synth.ba(5000, 8, 2)),
    ("rmat", 1 << 12, synth.rmat(12, 16, 3)),
    ("chung_lu", 6000, synth.chung_lu(6000, 20.0, 2.1, 4, 0)),
])
def test_orders_match_oracle_and_theorems(tc, name, n, e):
    adj = oracle.Adjacency(n, e)
    deg = adj.deg
    ref = oracle.count(n, e, local=True)
    ed = torch.from_numpy(np.ascontiguousarray(synth.shuffle_edges(e, 5))).cuda()
    W = {}
    for oname, key in orders(n, deg, 7).items():
        g = tc.orient(ed, n, keys=torch.from_numpy(key).cuda())
        off, cols, dhat = adj.orient(order_key=key)
        assert np.array_equal(g.offsets.cpu().numpy(), off), oname
        assert np.array_equal(g.cols.cpu().numpy(), cols), oname
        assert np.array_equal(g.dhat.cpu().numpy(), dhat), oname
        T, tv, _ = tc.count_local(g, clustering=False)
        assert T == ref["T"], oname                        # Theorem 1: any order counts each triangle once
        assert np.array_equal(tv.cpu().numpy(), ref["tv"]), oname
        W[oname] = int((g.deg.to(torch.int64) * g.dhat.to(torch.int64)).sum().item())
        assert W[oname] == adj.cost(order_key=key), oname
    assert all(W["degree"] <= w for w in W.values()), W  # Theorem 3


def test_degree_keys_reproduce_tc_orient(tc):
    n, e = 1 << 11, synth.rmat(11, 16, 9)
    ed = torch.from_numpy(e).cuda()
    g0 = tc.orient(ed, n)
    g1 = tc.orient(ed, n, keys=g0.deg.to(torch.int64))
    assert torch.equal(g0.offsets, g1.offsets) and torch.equal(g0.cols, g1.cols)


def test_lists_longer_than_a_block_sort(tc):
    # under the id order the hub (vertex 0) keeps all 70000 neighbours: its list is
    # sorted in place in global memory (longer than the shared-memory sort holds)
    n = 70001
    rng = np.random.default_rng(3)
    leaves = synth.shuffle_edges(synth.star(n - 1), 4)
    extra = synth.er(n, 200000, 5)
    e = np.unique(np.concatenate([np.sort(leaves, axis=1), extra]), axis=0).astype(np.int32)
    e = e[e[:, 0] != e[:, 1]]
    adj = oracle.Adjacency(n, e)
    ed = torch.from_numpy(np.ascontiguousarray(synth.shuffle_edges(e, 6))).cuda()
    for key in (np.zeros(n, np.int64), rng.permutation(n).astype(np.int64)):
        g = tc.orient(ed, n, keys=torch.from_numpy(key).cuda())
        off, cols, dhat = adj.orient(order_key=key)
        assert np.array_equal(g.offsets.cpu().numpy(), off)
        assert np.array_equal(g.cols.cpu().numpy(), cols)
        assert tc.count(g) == oracle.count(n, e)["T"]
    g = tc.orient(ed, n, keys=torch.zeros(n, dtype=torch.int64, device="cuda"))
    assert int(g.dhat.max().item()) > 32768
