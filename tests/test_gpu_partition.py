"""The cost-balanced partition of the apex vertices (the paper's load-balancing
step, Table "lbscheme") and counting by apex range: boundary nodes and part
costs equal the oracle's, each part's triangles and per-vertex counts equal the
oracle's triangles with their first vertex in the part, and the parts of any
partition sum to T and T_v exactly."""
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


def graphs():
    return [
        ("er", 3000, synth.er(3000, 30000, 1)),
        ("ba", 4000, synth.ba(4000, 8, 2)),
        ("rmat", 1 << 12, synth.rmat(12, 16, 3)),
        ("chung_lu", 5000, synth.chung_lu(5000, 16.0, 2.1, 4, 0)),
        ("clique", 300, synth.complete(300)),
        ("star", 51, synth.star(50)),
        ("empty", 9, np.zeros((0, 2), np.int32)),
    ]


def to_dev(e):
    return torch.from_numpy(np.ascontiguousarray(e, dtype=np.int32)).cuda()


@pytest.mark.parametrize("cost", range(6))
def test_partition_matches_oracle(tc, cost):
    for name, n, e in graphs():
        g = tc.orient(to_dev(e), n)
        for parts in (1, 3, 8, 64):
            b, c = tc.partition(g, parts, cost)
            rb, rc = oracle.partition(n, e, parts, cost)
            assert np.array_equal(b.cpu().numpy(), rb), (name, parts)
            assert np.array_equal(c.cpu().numpy(), rc), (name, parts)


@pytest.mark.parametrize("hub_min,tile_max", [(-1, 0), (0, 0), (16, 32)])
def test_part_counts_match_oracle(tc, hub_min, tile_max):
    ctx = tc.Context(0)
    ctx.set_hub_min(hub_min)
    ctx.set_tuning(tile_max, 1)
    for name, n, e in graphs()[1:4]:
        g = tc.orient(to_dev(synth.shuffle_edges(e, 9)), n, ctx)
        b, _ = tc.partition(g, 8, tc.COST_WORK, ctx)
        b = b.cpu().numpy()
        T_all = torch.zeros(1, dtype=torch.int64, device="cuda")
        tv_all = torch.zeros(n, dtype=torch.int64, device="cuda")
        for j in range(8):
            T = torch.zeros(1, dtype=torch.int64, device="cuda")
            tv = torch.zeros(n, dtype=torch.int64, device="cuda")
            tc.count_range(g, int(b[j]), int(b[j + 1]), T, tv, ctx)
            rT, rtv = oracle.count_apex_range(n, e, int(b[j]), int(b[j + 1]))
            assert int(T.item()) == rT, (name, j)
            assert np.array_equal(tv.cpu().numpy(), rtv), (name, j)
            tc.count_range(g, int(b[j]), int(b[j + 1]), T_all, tv_all, ctx)
        Tl, tvl, _ = tc.count_local(g, clustering=False, ctx=ctx)
        assert int(T_all.item()) == Tl
        assert torch.equal(tv_all, tvl)
    ctx.close()


def test_arbitrary_ranges_sum_to_the_count(tc):
    n, e = 1 << 13, synth.rmat(13, 16, 7)
    g = tc.orient(to_dev(e), n)
    T_ref = tc.count(g)
    rng = np.random.default_rng(3)
    for _ in range(3):
        cuts = np.sort(rng.choice(np.arange(1, n), 11, replace=False))
        cuts = np.concatenate([[0, 0], cuts, [cuts[-1], n]])  # includes empty ranges
        T = torch.zeros(1, dtype=torch.int64, device="cuda")
        for lo, hi in zip(cuts[:-1], cuts[1:]):
            tc.count_range(g, int(lo), int(hi), T)
        assert int(T.item()) == T_ref


def test_range_and_partition_errors(tc):
    n, e = 100, synth.er(100, 500, 2)
    g = tc.orient(to_dev(e), n)
    T = torch.zeros(1, dtype=torch.int64, device="cuda")
    for lo, hi in ((5, 4), (-1, 3), (0, 101)):
        with pytest.raises(tc.TcError):
            tc.count_range(g, lo, hi, T)
    for parts, cost in ((0, 5), (70000, 5), (4, 6)):
        with pytest.raises(tc.TcError):
            tc.partition(g, parts, cost)
    assert int(T.item()) == 0


def test_partition_local_sparsification_matches_oracle(tc):
    for name, n, e in graphs()[:4]:
        g = tc.orient(to_dev(synth.shuffle_edges(e, 2)), n)
        b, _ = tc.partition(g, 4, tc.COST_WORK)
        b = b.cpu().numpy()
        for seed, q in ((1, 0.3), (7, 0.1)):
            kept = torch.zeros(1, dtype=torch.int64, device="cuda")
            for j in range(4):
                before = int(kept.item())
                tc.sparsify_count_part(g, q, seed, j, int(b[j]), int(b[j + 1]), kept)
                ref = oracle.sparsify_count_part(n, e, seed, q, j, int(b[j]), int(b[j + 1]))
                assert int(kept.item()) - before == ref, (name, seed, j)
        # part 0 over every apex is tc_sparsify_count
        kept = torch.zeros(1, dtype=torch.int64, device="cuda")
        mk = tc.sparsify_count_part(g, 0.2, 5, 0, 0, n, kept)
        t, mk2, _ = tc.sparsify_count(g, 0.2, 5)
        assert (int(kept.item()), mk) == (t, mk2)
