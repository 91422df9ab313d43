"""Planted mistakes: every plausible slip in the oracle must fail one of its pins.

Each case compiles a copy of ``oracle/tc_oracle.c`` with one mistake planted
(a dropped term, a reversed comparison, a wrong bound, a swapped word, a wrong
constant), points the oracle at that copy, and runs the pins of
``test_oracle_pins`` that should notice; at least one of them has to fail.
The mistakes live only in the temporary copy, on the CPU; the real oracle is
restored when each case ends.
"""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

import oracle
from tests import test_oracle_pins as pins

# (what the slip is, the line as written, the line with the slip, pins that must catch it)
MUTANTS = [
    ("per-vertex count misses the third vertex (Figure \"localcount\")",
     "          tv[w] += 1;\n", "\n",
     [lambda: pins.test_complete_graph(5), lambda: pins.test_exhaustive_small_graphs(4)]),
    ("inner loop without u < w (Figure 1): triangles counted more than once",
     "        if (!precedes(order_key, u, w)) continue;\n", "        if (w == u) continue;\n",
     [lambda: pins.test_complete_graph(4), lambda: pins.test_exhaustive_small_graphs(4)]),
    ("outer loop without v < u (Figure 1)",
     "      if (!precedes(order_key, v, u)) continue;\n", "\n",
     [lambda: pins.test_complete_graph(4), lambda: pins.test_exhaustive_small_graphs(4)]),
    ("binary search drops an element (adjacency test)",
     "    else if (adj[mid] > w) hi = mid;\n", "    else if (adj[mid] > w) hi = mid - 1;\n",
     [lambda: pins.test_exhaustive_small_graphs(5), lambda: pins.test_brute_force_random_graphs(0)]),
    ("order's tie broken by the larger id (Eq. 1)",
     "  return key[u] < key[v] || (key[u] == key[v] && u < v);\n",
     "  return key[u] < key[v] || (key[u] == key[v] && u > v);\n",
     [pins.test_orientation_worked_by_hand]),
    ("orientation's tie broken by the larger id (Eq. 1, Definition 1)",
     "      else keep = dv < du || (dv == du && v < u);\n",
     "      else keep = dv < du || (dv == du && v > u);\n",
     [pins.test_orientation_worked_by_hand]),
    ("orientation keeps the earlier endpoint instead of the later one (Definition 1)",
     "      else keep = dv < du || (dv == du && v < u);\n",
     "      else keep = du < dv || (du == dv && u < v);\n",
     [pins.test_orientation_worked_by_hand, lambda: pins.test_wheel_orientation_matches_paper(12)]),
    ("Theorem 2's cost with dhat_v in place of d_v",
     "    W += (uint64_t)(dv * dhat);\n", "    W += (uint64_t)(dhat * dhat);\n",
     [lambda: pins.test_orientation_properties(0), lambda: pins.test_degree_order_minimises_cost(0)]),
    ("clustering coefficient without the factor 2 (Section 11)",
     "    else cc[v] = (2.0 * (double)tv[v]) / (double)(d * (d - 1));\n",
     "    else cc[v] = ((double)tv[v]) / (double)(d * (d - 1));\n",
     [lambda: pins.test_complete_graph(5), pins.test_clustering_formula_bits]),
    ("Philox multiplier with one wrong digit",
     "  const uint32_t mul0 = 0xD2511F53u, mul1 = 0xCD9E8D57u;\n",
     "  const uint32_t mul0 = 0xD2511F57u, mul1 = 0xCD9E8D57u;\n",
     [lambda row=row: pins.test_philox_known_answers(*row) for row in pins._kat_rows()]),
    ("Philox round takes the low half of the wrong product",
     "    uint32_t y1 = (uint32_t)r;\n", "    uint32_t y1 = (uint32_t)p;\n",
     [lambda row=row: pins.test_philox_known_answers(*row) for row in pins._kat_rows()]),
    ("Philox key schedule not advanced",
     "    k0 += weyl0;\n", "\n",
     [lambda row=row: pins.test_philox_known_answers(*row) for row in pins._kat_rows()]),
    ("sparsification coin compared the wrong way (Section 9.1)",
     "  return u < q;\n", "  return u > q;\n",
     [pins.test_sparsify_q_one_and_zero, pins.test_sparsify_kept_fraction_binomial]),
    ("sparsified estimate scaled by 1/q^2 instead of 1/q^3 (Section 9.1)",
     "  *estimate = (double)(*T_kept) / (q * q * q);\n", "  *estimate = (double)(*T_kept) / (q * q);\n",
     [pins.test_sparsify_unbiased_with_paper_variance]),
    ("coin built from one output word only",
     "  uint64_t r = ((uint64_t)out[0] << 21) | (out[1] >> 11); /* top 53 bits of x0:x1 */\n",
     "  uint64_t r = (uint64_t)out[0] << 21;\n",
     [pins.test_coin_switches_exactly_at_its_53_bit_value]),
]


def _caught(check) -> bool:
    try:
        check()
    except (AssertionError, pytest.fail.Exception):  # a failed assert, or pytest.raises that saw nothing
        return True
    return False


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc to build the planted copies")
@pytest.mark.parametrize("what,line,slip,checks", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(what, line, slip, checks, tmp_path, monkeypatch):
    with open(oracle._SRC) as f:
        src = f.read()
    assert src.count(line) == 1, f"the line to plant in is not unique or missing: {line!r}"
    planted = tmp_path / "tc_oracle.c"
    planted.write_text(src.replace(line, slip))
    lib = tmp_path / "liboracle_planted.so"
    subprocess.run(["gcc", "-O2", "-shared", "-fPIC", "-std=c11", str(planted), "-o", str(lib)], check=True)
    os.utime(lib)  # newer than the planted source, so the oracle loads it as built
    monkeypatch.setattr(oracle, "_SRC", str(planted))
    monkeypatch.setattr(oracle, "_LIB_PATH", str(lib))
    monkeypatch.setattr(oracle, "_lib", None)
    caught = [_caught(c) for c in checks]
    assert any(caught), f"no pin noticed: {what}"


# ---- the parallel oracle: each slip must break its equality with the serial oracle ----

from tests import test_oracle_par as par_pins  # noqa: E402

_PAR_GRAPHS = {g[0]: g for g in par_pins.GRAPHS}


def _par_equal(*names):
    return [lambda nm=nm: par_pins.test_parallel_oracle_equals_serial(*_PAR_GRAPHS[nm]) for nm in names]


PAR_MUTANTS = [
    ("T_w share of a triangle dropped (Section 11)",
     "            per_w[a - lo] += 1;\n", "\n", _par_equal("K9", "rmat9")),
    ("T_u share of a triangle dropped (Section 11)",
     "        if (tv && t_e) __atomic_fetch_add(&tv[u], t_e, __ATOMIC_RELAXED);\n", "\n", _par_equal("K9", "rmat9")),
    ("merge skips the first id of N_v (Figure 2)",
     "        int64_t a = lo, b = off[u], be = off[u + 1], t_e = 0;\n",
     "        int64_t a = lo + 1, b = off[u], be = off[u + 1], t_e = 0;\n", _par_equal("K9", "wheel12")),
    ("order's tie broken by the larger id (Eq. 1)",
     "  return ku < kv || (ku == kv && u < v);\n", "  return ku < kv || (ku == kv && u > v);\n",
     _par_equal("K9", "cycle7")),
    ("repeated edges accepted",
     "      if (adj[i] == adj[i - 1]) dup = 1;\n", "      ;\n",
     [lambda: par_pins.test_parallel_adjacency_rejects_non_simple_input([[0, 1], [2, 3], [1, 0]], "repeated")]),
    ("a fingerprint constant differs from its tensor restatement",
     "static const uint64_t FP_B[2] = {12345ULL, 1013904223ULL};\n",
     "static const uint64_t FP_B[2] = {12346ULL, 1013904223ULL};\n", _par_equal("K9")),
]


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc to build the planted copies")
@pytest.mark.parametrize("what,line,slip,checks", PAR_MUTANTS, ids=[m[0] for m in PAR_MUTANTS])
def test_planted_mistake_in_parallel_oracle_fails_a_pin(what, line, slip, checks, tmp_path, monkeypatch):
    from oracle import par
    src_par, src_serial = par._SRCS
    with open(src_par) as f:
        src = f.read()
    assert src.count(line) == 1, f"the line to plant in is not unique or missing: {line!r}"
    planted = tmp_path / "tc_oracle_par.c"
    planted.write_text(src.replace(line, slip))
    lib = tmp_path / "liboracle_par_planted.so"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", str(planted), src_serial, "-o",
                    str(lib)], check=True)
    os.utime(lib)
    monkeypatch.setattr(par, "_SRCS", [str(planted), src_serial])
    monkeypatch.setattr(par, "_LIB_PATH", str(lib))
    monkeypatch.setattr(par, "_lib", None)
    caught = [_caught(c) for c in checks]
    assert any(caught), f"no pin noticed: {what}"
