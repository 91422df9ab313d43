"""Pins of the CPU oracle against things other than itself.

Each test checks the oracle against a fact the paper or mathematics fixes:
brute force on tiny graphs, trace(A^3)/6, closed forms, the paper's printed
values, Theorems 1 and 3, the unbiasedness and variance of the sparsified
estimate (Section 9.1, Eq. var1), and the published known answers of
Philox4x32-10.
"""
from __future__ import annotations

import itertools
import math
import os

import numpy as np
import pytest

import oracle
import synth
from tests import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v) if "." in v else int(v)
    return vals


# ---- Philox4x32-10 against its published known answers ---------------------

def _kat_rows():
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                w = [int(x, 16) for x in line.split()]
                yield w[:4], w[4:6], w[6:10]


@pytest.mark.parametrize("ctr,key,expected", list(_kat_rows()))
def test_philox_known_answers(ctr, key, expected):
    assert [int(x) for x in oracle.philox(ctr, key)] == expected


def test_philox_words_are_uniform():
    # every output bit of a counter-based generator is a fair coin: over 4096
    # consecutive counters each of the 128 bits is set about half the time
    counts = np.zeros(128)
    for i in range(4096):
        w = oracle.philox([i, 7, 0, 0], [0x1234, 0x5678])
        counts += [(int(w[j]) >> b) & 1 for j in range(4) for b in range(32)]
    assert np.all(np.abs(counts - 2048) < 5 * 32)  # 5 sigma of Binomial(4096, 1/2)


# ---- brute force ------------------------------------------------------------

def _all_graphs(n):
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        yield np.array([p for i, p in enumerate(pairs) if mask >> i & 1], dtype=np.int32).reshape(-1, 2)


@pytest.mark.parametrize("n", [3, 4, 5])
def test_exhaustive_small_graphs(n):
    for e in _all_graphs(n):
        tris = brute.triangles_by_triples(n, e)
        r = oracle.count(n, e, local=True, listing=True)
        assert r["T"] == len(tris)
        assert np.array_equal(r["tv"], brute.per_vertex_from_list(n, tris))
        assert np.array_equal(brute.canon(r["tri"]), brute.canon(tris))


def test_random_six_vertex_graphs():
    rng = np.random.default_rng(6)
    pairs = list(itertools.combinations(range(6), 2))
    for _ in range(1500):
        mask = rng.integers(0, 2, len(pairs)).astype(bool)
        e = np.array([p for p, k in zip(pairs, mask) if k], dtype=np.int32).reshape(-1, 2)
        tris = brute.triangles_by_triples(6, e)
        r = oracle.count(6, e, local=True, listing=True)
        assert r["T"] == len(tris)
        assert np.array_equal(brute.canon(r["tri"]), brute.canon(tris))


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_random_graphs(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(20, 60))
    p = float(rng.uniform(0.05, 0.5))
    e = np.array([(i, j) for i, j in itertools.combinations(range(n), 2) if rng.random() < p],
                 dtype=np.int32).reshape(-1, 2)
    e = synth.shuffle_edges(e, seed)
    tris = brute.triangles_by_triples(n, e)
    r = oracle.count(n, e, local=True, listing=True)
    assert r["T"] == len(tris)
    assert np.array_equal(r["tv"], brute.per_vertex_from_list(n, tris))
    assert np.array_equal(brute.canon(r["tri"]), brute.canon(tris))


@pytest.mark.parametrize("kind", ["er", "ba", "rmat", "chung_lu"])
def test_trace_a_cubed(kind):
    if kind == "er":
        n, e = 600, synth.er(600, 6000, 11)
    elif kind == "ba":
        n, e = 700, synth.ba(700, 6, 12)
    elif kind == "rmat":
        n, e = 1 << 9, synth.rmat(9, 16, 13)
    else:
        n, e = 800, synth.chung_lu(800, 24.0, 2.1, 14, 0)
    T, tv = brute.trace_cubed(n, e)
    r = oracle.count(n, e, local=True)
    assert r["T"] == T
    assert np.array_equal(r["tv"], tv)
    assert int(r["tv"].sum()) == 3 * r["T"]


# ---- closed forms -------------------------------------------------------------

@pytest.mark.parametrize("n", [3, 4, 5, 9, 17, 40])
def test_complete_graph(n):
    r = oracle.count(n, synth.complete(n), local=True)
    assert r["T"] == math.comb(n, 3)
    assert np.all(r["tv"] == math.comb(n - 1, 2))
    adj = oracle.Adjacency(n, synth.complete(n))
    cc = oracle.clustering(adj.deg, r["tv"])
    assert np.all(cc == 1.0)


@pytest.mark.parametrize("n", [4, 5, 6, 50, 1000])
def test_cycle_has_no_triangle(n):
    assert oracle.count(n, synth.cycle(n))["T"] == 0


def test_triangle_cycle():
    assert oracle.count(3, synth.cycle(3))["T"] == 1


@pytest.mark.parametrize("k", [3, 4, 5, 8, 31, 200])
def test_wheel(k):
    r = oracle.count(k + 1, synth.wheel(k), local=True)
    if k == 3:  # the wheel with three rim vertices is K4
        assert r["T"] == 4
        assert np.all(r["tv"] == 3)
    else:
        assert r["T"] == k
        assert r["tv"][0] == k
        assert np.all(r["tv"][1:] == 2)


@pytest.mark.parametrize("k", [5, 12, 100])
def test_wheel_orientation_matches_paper(k):
    g = read_golden("wheel.txt")
    adj = oracle.Adjacency(k + 1, synth.wheel(k))
    _, _, dhat = adj.orient()
    assert dhat[0] == g["hub_dhat"]
    assert dhat[1:].max() <= g["rim_dhat_max"]


@pytest.mark.parametrize("edges,n", [
    (synth.star(10), 11), (synth.complete_bipartite(4, 7), 11),
    (synth.complete_bipartite(1, 1), 2), (synth.random_tree(300, 3), 300),
])
def test_triangle_free(edges, n):
    r = oracle.count(n, edges, local=True)
    assert r["T"] == 0
    assert np.all(r["tv"] == 0)
    assert np.all(oracle.clustering(oracle.Adjacency(n, edges).deg, r["tv"]) == 0.0)


def test_empty_and_isolated():
    assert oracle.count(0, np.zeros((0, 2), np.int32))["T"] == 0
    assert oracle.count(10, np.zeros((0, 2), np.int32))["T"] == 0
    r = oracle.count(10, np.array([[0, 1], [1, 2], [0, 2]], np.int32), local=True)
    assert r["T"] == 1 and r["tv"].tolist() == [1, 1, 1, 0, 0, 0, 0, 0, 0, 0]


def test_rejects_non_simple_input():
    with pytest.raises(oracle.OracleError, match="self-loop"):
        oracle.count(3, np.array([[0, 1], [1, 1]], np.int32))
    with pytest.raises(oracle.OracleError, match="repeated"):
        oracle.count(3, np.array([[0, 1], [1, 0]], np.int32))
    with pytest.raises(oracle.OracleError, match="out of range"):
        oracle.count(3, np.array([[0, 3]], np.int32))


# ---- theorems and invariants ----------------------------------------------------

@pytest.mark.parametrize("seed", range(4))
def test_total_order_does_not_change_count(seed):
    # Theorem 1 and Section 4: any total order counts each triangle exactly once.
    n = 500
    e = synth.ba(n, 5, seed)
    adj = oracle.Adjacency(n, e)
    base = adj.count(local=True)
    rng = np.random.default_rng(seed)
    for key in (np.zeros(n, np.int64), rng.integers(0, 50, n), rng.permutation(n)):
        r = adj.count(order_key=key, local=True)
        assert r["T"] == base["T"]
        assert np.array_equal(r["tv"], base["tv"])


@pytest.mark.parametrize("seed", range(4))
def test_relabelling_invariance(seed):
    n = 400
    e = synth.rmat(9, 8, seed)
    n = 1 << 9
    perm = np.random.default_rng(seed).permutation(n).astype(np.int32)
    a = oracle.count(n, e, local=True, listing=True)
    b = oracle.count(n, synth.relabel(e, perm), local=True, listing=True)
    assert a["T"] == b["T"]
    assert np.array_equal(b["tv"][perm], a["tv"])
    assert np.array_equal(brute.canon(perm[a["tri"]]), brute.canon(b["tri"]))


def test_orientation_worked_by_hand():
    # Eq. (1): u precedes v iff d_u < d_v, or d_u = d_v and u < v.  Lists and
    # listed triples below are worked out by hand from that definition; each
    # graph has degree ties, so a tie broken the other way changes the answer.
    k4 = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    cases = [
        # path 0-1-2: d = (1, 2, 1), order 0, 2, 1
        (3, [(0, 1), (1, 2)], [[1], [], [1]], []),
        # K4: all d = 3, order 0, 1, 2, 3
        (4, k4, [[1, 2, 3], [2, 3], [3], []], [(0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)]),
        # triangle 0-1-2 with a pendant on 2: d = (2, 2, 3, 1), order 3, 0, 1, 2
        (4, [(0, 1), (1, 2), (0, 2), (2, 3)], [[1, 2], [2], [], [2]], [(0, 1, 2)]),
        # triangle 0-1-2 with a pendant on 0: d = (3, 2, 2, 1), order 3, 1, 2, 0
        (4, [(0, 1), (1, 2), (0, 2), (0, 3)], [[], [0, 2], [0], [0]], [(1, 2, 0)]),
    ]
    for n, e, lists, tris in cases:
        adj = oracle.Adjacency(n, np.array(e, np.int32))
        off, cols, dhat = adj.orient()
        assert [cols[off[v]:off[v + 1]].tolist() for v in range(n)] == lists
        assert dhat.tolist() == [len(x) for x in lists]
        # NodeIterator++ lists each triangle as (v, u, w) with v < u < w in the order
        assert sorted(map(tuple, adj.count(listing=True)["tri"].tolist())) == sorted(tris)


@pytest.mark.parametrize("seed", range(3))
def test_degree_order_minimises_cost(seed):
    # Theorem 3: sum_v d_v * dhat_v is smallest under the degree order.
    n = 600
    e = synth.chung_lu(n, 16.0, 2.1, seed, 0)
    adj = oracle.Adjacency(n, e)
    best = adj.cost()
    rng = np.random.default_rng(seed)
    for key in (np.zeros(n, np.int64), rng.permutation(n), -adj.deg.astype(np.int64)):
        assert adj.cost(order_key=key) >= best


@pytest.mark.parametrize("seed", range(3))
def test_orientation_properties(seed):
    n = 1 << 10
    e = synth.rmat(10, 16, seed)
    adj = oracle.Adjacency(n, e)
    off, cols, dhat = adj.orient()
    deg = adj.deg
    assert off[-1] == len(e) == dhat.sum()          # sum_v dhat_v = m (Section 3)
    for v in range(n):
        lst = cols[off[v]:off[v + 1]]
        assert np.all(np.diff(lst) > 0)               # sorted, no repeats
        for u in lst:                                 # v precedes u (Eq. 1)
            assert deg[v] < deg[u] or (deg[v] == deg[u] and v < u)
    assert adj.cost() == int((deg.astype(np.int64) * dhat).sum())


def test_vertex_triangles_definition():
    n = 1 << 9
    e = synth.rmat(9, 16, 5)
    adj = oracle.Adjacency(n, e)
    tv = adj.count(local=True)["tv"]
    for v in range(0, n, 7):
        assert adj.vertex_triangles(v) == tv[v]


def test_clustering_formula_bits():
    deg = np.array([0, 1, 2, 3, 7, 100000, 46341], np.int32)
    tv = np.array([0, 0, 1, 2, 5, 123456789, 1000], np.int64)
    cc = oracle.clustering(deg, tv)
    assert cc[0] == 0.0 and cc[1] == 0.0
    for i in range(2, len(deg)):
        d = int(deg[i])
        # exactly one correctly rounded division: compare with the exact rational
        from fractions import Fraction
        exact = Fraction(2 * int(tv[i]), d * (d - 1))
        assert cc[i] == float(exact)


# ---- the paper's printed values ---------------------------------------------------

def test_gnp_500k_20_matches_paper_table():
    g = read_golden("gnp_500k_20.txt")
    n, d = g["n"], g["avg_degree"]
    p = d / (n - 1)
    mean = math.comb(n, 3) * p ** 3
    sd = math.sqrt(mean)
    # the paper's realisation is consistent with E[T] = C(n,3) p^3 ...
    assert abs(g["triangles"] - mean) < 2 * sd
    # ... and so is the oracle's count on our own Gnp(500K, 20) instance
    e = synth.er(n, n * d // 2, 2024)
    m = len(e)
    p_m = m / math.comb(n, 2)
    mean_m = math.comb(n, 3) * p_m ** 3
    T = oracle.count(n, e)["T"]
    assert abs(T - mean_m) < 5 * math.sqrt(mean_m)


# ---- sparsification (Section 9.1) ----------------------------------------------------

def test_sparsify_q_one_and_zero():
    n = 1 << 9
    e = synth.rmat(9, 16, 3)
    T = oracle.count(n, e)["T"]
    t1, m1, est1 = oracle.sparsify_count(n, e, 7, 1.0)
    assert (t1, m1, est1) == (T, len(e), float(T))
    t0, m0, _ = oracle.sparsify_count(n, e, 7, 0.0)
    assert (t0, m0) == (0, 0)


def test_sparsify_coin_depends_only_on_edge():
    n = 1 << 9
    e = synth.rmat(9, 16, 4)
    a = oracle.sparsify_count(n, e, 99, 0.3)
    b = oracle.sparsify_count(n, synth.shuffle_edges(e, 1), 99, 0.3)
    assert a == b


def test_sparsify_kept_fraction_binomial():
    n = 1 << 12
    e = synth.er(n, 40000, 8)
    q = 0.1
    _, mk, _ = oracle.sparsify_count(n, e, 1234, q)
    m = len(e)
    assert abs(mk - q * m) < 5 * math.sqrt(m * q * (1 - q))


def test_sparsify_unbiased_with_paper_variance():
    # E[T'/q^3] = T and Var = (1/q^3 - 1) T + 2k (1/q - 1) (Eq. var1).
    n = 300
    e = synth.ba(n, 8, 21)
    tris = brute.triangles_by_neighbours(n, e)
    T = len(tris)
    k = brute.edge_triangle_pairs(tris)
    q = 0.5
    var = (1 / q ** 3 - 1) * T + 2 * k * (1 / q - 1)
    S = 400
    ests = np.array([oracle.sparsify_count(n, e, s, q)[2] for s in range(S)])
    assert abs(ests.mean() - T) < 4.5 * math.sqrt(var / S)
    assert 0.7 * var < ests.var(ddof=1) < 1.4 * var


def test_clique_with_pendants_closed_form():
    """The closed form the GPU hub tests use, checked against the oracle and the definition."""
    from tests.brute import clique_with_pendants, triangles_by_triples, per_vertex_from_list
    for k, a, width in ((12, 4, 4), (9, 3, 3), (40, 12, 4)):
        n, e, T, tv = clique_with_pendants(k, a, width)
        r = oracle.count(n, e, local=True)
        assert r["T"] == T
        assert np.array_equal(r["tv"], tv)
        if n <= 40:
            tris = triangles_by_triples(n, e)
            assert len(tris) == T
            assert np.array_equal(per_vertex_from_list(n, tris), tv)


# ---- load-balancing partition (Table "lbscheme", the boundary-node definition) ----

def _fraction_bounds(F, parts):
    """Boundary nodes straight from the definition, with rational arithmetic:
    x_j = min{v : F(v) >= j * alpha}, alpha = F(n-1) / parts."""
    from fractions import Fraction
    n = len(F)
    alpha = Fraction(int(F[-1]), parts) if n else Fraction(0)
    out = [0]
    for j in range(1, parts):
        out.append(next((v for v in range(n) if F[v] >= j * alpha), n))
    return out + [n]


@pytest.mark.parametrize("cost", range(6))
def test_partition_follows_the_boundary_definition(cost):
    for n, e in ((50, synth.er(50, 300, 1)), (120, synth.ba(120, 3, 2)), (256, synth.rmat(8, 6, 3)),
                 (7, synth.star(6)), (12, np.zeros((0, 2), np.int32))):
        f = oracle.partition_costs(n, e, cost)
        F = np.cumsum(f)
        for parts in (1, 2, 5, 16, n + 3):
            b, c = oracle.partition(n, e, parts, cost)
            assert list(b) == _fraction_bounds(F, parts)
            assert b[0] == 0 and b[-1] == n and all(b[i] <= b[i + 1] for i in range(parts))
            assert int(c.sum()) == (int(F[-1]) if n else 0)


def test_partition_costs_match_their_closed_sums():
    n, e = 256, synth.rmat(8, 10, 4)
    adj = oracle.Adjacency(n, e)
    m = len(e)
    assert oracle.partition_costs(n, e, oracle.COST_VERTICES).sum() == n
    assert oracle.partition_costs(n, e, oracle.COST_DEGREE).sum() == 2 * m
    assert oracle.partition_costs(n, e, oracle.COST_DHAT).sum() == m           # sum dhat = m
    # sum over v, u in N_v of (dhat_v + dhat_u) = sum_v d_v dhat_v (Theorem 2's cost)
    assert oracle.partition_costs(n, e, oracle.COST_WORK).sum() == adj.cost()
    assert oracle.partition_costs(n, e, oracle.COST_DEG_DHAT).sum() == adj.cost()


def test_apex_ranges_sum_to_the_whole():
    n, e = 128, synth.rmat(7, 12, 5)
    ref = oracle.count(n, e, local=True)
    total, tv = 0, np.zeros(n, np.int64)
    for lo, hi in ((0, 17), (17, 17), (17, 90), (90, 128)):
        c, t = oracle.count_apex_range(n, e, lo, hi)
        total += c
        tv += t
    assert total == ref["T"]
    assert np.array_equal(tv, ref["tv"])


# ---- sparsification with partition-local coins (Section 9.2, Eq. var2) ----

def test_part_coin_reduces_to_the_plain_coin_and_to_philox():
    rng = np.random.default_rng(1)
    for _ in range(300):
        a, b = (int(x) for x in rng.integers(0, 1 << 20, 2))
        seed, q = int(rng.integers(0, 1 << 40)), float(rng.random())
        assert oracle.sparsify_keep_part(a, b, seed, q, 0) == oracle.sparsify_keep(a, b, seed, q)
        part = int(rng.integers(0, 64))
        x = oracle.philox([min(a, b), max(a, b), part, 0], [seed & 0xFFFFFFFF, seed >> 32])
        r = (int(x[0]) << 21) | (int(x[1]) >> 11)  # top 53 bits of x0:x1
        assert oracle.sparsify_keep_part(a, b, seed, q, part) == (r * 2.0 ** -53 < q)


def test_coin_switches_exactly_at_its_53_bit_value():
    # the coin keeps an edge iff r * 2^-53 < q, r the top 53 bits of Philox's
    # words x0:x1: at q = r * 2^-53 (exact in a double) it drops the edge and at
    # q = (r + 1) * 2^-53 it keeps it, for every part
    rng = np.random.default_rng(7)
    for _ in range(200):
        a, b = (int(x) for x in rng.integers(0, 1 << 30, 2))
        if a == b:
            continue
        seed, part = int(rng.integers(0, 1 << 62)), int(rng.integers(0, 1 << 20))
        x = oracle.philox([min(a, b), max(a, b), part, 0], [seed & 0xFFFFFFFF, seed >> 32])
        r = (int(x[0]) << 21) | (int(x[1]) >> 11)
        assert not oracle.sparsify_keep_part(a, b, seed, r * 2.0 ** -53, part)
        assert oracle.sparsify_keep_part(a, b, seed, (r + 1) * 2.0 ** -53, part)


def test_parts_with_q_one_sum_to_t():
    n, e = 256, synth.rmat(8, 8, 2)
    b, _ = oracle.partition(n, e, 4, oracle.COST_WORK)
    total = sum(oracle.sparsify_count_part(n, e, 3, 1.0, j, int(b[j]), int(b[j + 1])) for j in range(4))
    assert total == oracle.count(n, e)["T"]


def test_partitioned_estimator_unbiased_with_var2():
    # parts sparsify independently: E[sum T'_j / q^3] = T and
    # Var' = (1/q^3 - 1) T + 2 k' (1/q - 1), k' = pairs of triangles sharing an edge
    # with both apexes (first vertices in the order of Eq. (1)) in the same part (Eq. var2)
    n = 200
    e = synth.ba(n, 6, 21)
    deg = oracle.Adjacency(n, e).deg
    parts = 4
    bounds, _ = oracle.partition(n, e, parts, oracle.COST_WORK)
    tris = brute.triangles_by_neighbours(n, e)
    T = len(tris)
    part_of = np.searchsorted(bounds, np.arange(n), side="right") - 1
    apex = [min(t, key=lambda x: (deg[x], x)) for t in tris]
    k_same = 0
    for j in range(parts):
        k_same += brute.edge_triangle_pairs([t for t, a in zip(tris, apex) if part_of[a] == j])
    k_all = brute.edge_triangle_pairs(tris)
    assert k_same < k_all  # the partition separates some pairs: var2 < var1 here
    q = 0.5
    var2 = (1 / q ** 3 - 1) * T + 2 * k_same * (1 / q - 1)
    S = 240
    ests = np.array([sum(oracle.sparsify_count_part(n, e, s, q, j, int(bounds[j]), int(bounds[j + 1]))
                         for j in range(parts)) / q ** 3 for s in range(S)])
    assert abs(ests.mean() - T) < 4.5 * math.sqrt(var2 / S)
    assert 0.65 * var2 < ests.var(ddof=1) < 1.45 * var2
