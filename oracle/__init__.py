"""CPU oracle -- TEST INFRASTRUCTURE ONLY.

Python access to ``tc_oracle.c``, a plain serial restatement of the paper's
NodeIterator++ (Figure 1) with the degree order of Eq. (1), per-vertex counts
(Section 11), listing (Section 10), clustering coefficients (Preliminaries)
and edge sparsification (Section 9.1).  Only the tests, the smoke check and the
benchmark's CPU-baseline leg use it; the library under ``paper_1706_05151_gb300``
never imports it, and it imports nothing from there.

All functions take host numpy arrays: ``edges`` is ``int32[m, 2]`` with each
undirected edge once, in any direction.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tc_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

i32p = ctypes.POINTER(ctypes.c_int32)
i64p = ctypes.POINTER(ctypes.c_int64)
u64p = ctypes.POINTER(ctypes.c_uint64)
u32p = ctypes.POINTER(ctypes.c_uint32)
f64p = ctypes.POINTER(ctypes.c_double)

ERRORS = {1: "vertex id out of range", 2: "self-loop", 3: "repeated edge", 4: "out of memory",
          5: "listing capacity"}


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile ``tc_oracle.c`` to ``liboracle.so`` beside it (plain gcc -O2, one thread)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-shared", "-fPIC", "-std=c11", _SRC, "-o", tmp], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.orc_build_adjacency.restype = ctypes.c_int
        lib.orc_build_adjacency.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i64p, i32p]
        lib.orc_degrees.restype = None
        lib.orc_degrees.argtypes = [ctypes.c_int32, i64p, i32p]
        lib.orc_node_iterator_pp.restype = ctypes.c_int
        lib.orc_node_iterator_pp.argtypes = [ctypes.c_int32, i64p, i32p, i64p, u64p, i64p, i32p,
                                             ctypes.c_int64, i64p]
        lib.orc_orient.restype = None
        lib.orc_orient.argtypes = [ctypes.c_int32, i64p, i32p, i64p, i64p, i32p, i32p]
        lib.orc_cost.restype = ctypes.c_uint64
        lib.orc_cost.argtypes = [ctypes.c_int32, i64p, i32p, i64p]
        lib.orc_clustering.restype = None
        lib.orc_clustering.argtypes = [ctypes.c_int32, i32p, i64p, f64p]
        lib.orc_vertex_triangles.restype = ctypes.c_int64
        lib.orc_vertex_triangles.argtypes = [i64p, i32p, ctypes.c_int32]
        lib.orc_philox.restype = None
        lib.orc_philox.argtypes = [u32p, u32p, u32p]
        lib.orc_sparsify_keep.restype = ctypes.c_int
        lib.orc_sparsify_keep.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double]
        lib.orc_sparsify_keep_part.restype = ctypes.c_int
        lib.orc_sparsify_keep_part.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double,
                                               ctypes.c_uint32]
        lib.orc_sparsify_count.restype = ctypes.c_int
        lib.orc_sparsify_count.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, ctypes.c_uint64,
                                           ctypes.c_double, u64p, i64p, f64p]
        _lib = lib
        return lib


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _check(rc: int):
    if rc != 0:
        raise OracleError(ERRORS.get(rc, f"oracle error {rc}"))


def _edges(edges) -> np.ndarray:
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    return e


class Adjacency:
    """Full sorted adjacency N(v): ``off[n+1]`` (int64) and ``adj[2m]`` (int32)."""

    def __init__(self, n: int, edges):
        lib = _load()
        e = _edges(edges)
        self.n, self.m = int(n), len(e)
        self.off = np.zeros(self.n + 1, dtype=np.int64)
        self.adj = np.zeros(max(2 * self.m, 1), dtype=np.int32)
        _check(lib.orc_build_adjacency(self.n, self.m, _p(e, i32p), _p(self.off, i64p), _p(self.adj, i32p)))

    @property
    def deg(self) -> np.ndarray:
        d = np.zeros(self.n, dtype=np.int32)
        _load().orc_degrees(self.n, _p(self.off, i64p), _p(d, i32p))
        return d

    def _key(self, order_key):
        if order_key is None:
            return None
        k = np.ascontiguousarray(np.asarray(order_key, dtype=np.int64))
        assert k.shape == (self.n,)
        return k

    def count(self, order_key=None, local: bool = False, listing: bool = False, tri_cap: int | None = None):
        """NodeIterator++ (Figure 1).  Returns dict with T and, if asked, tv and tri."""
        lib = _load()
        key = self._key(order_key)
        T = ctypes.c_uint64(0)
        tv = np.zeros(self.n, dtype=np.int64) if local else None
        tri = None
        cnt = ctypes.c_int64(0)
        cap = 0
        if listing:
            cap = tri_cap if tri_cap is not None else self._listing_bound()
            tri = np.zeros((max(cap, 1), 3), dtype=np.int32)
        rc = lib.orc_node_iterator_pp(
            self.n, _p(self.off, i64p), _p(self.adj, i32p),
            _p(key, i64p) if key is not None else None, ctypes.byref(T),
            _p(tv, i64p) if tv is not None else None,
            _p(tri, i32p) if tri is not None else None, cap, ctypes.byref(cnt))
        if rc == 5 and listing and tri_cap is None:
            return self.count(order_key, local, True, tri_cap=int(cnt.value))
        _check(rc)
        out = {"T": int(T.value)}
        if local:
            out["tv"] = tv
        if listing:
            out["tri"] = tri[: int(cnt.value)]
        return out

    def _listing_bound(self) -> int:
        # every triangle contains an edge; a safe first guess, enlarged on demand
        return max(16, 2 * self.m)

    def orient(self, order_key=None):
        """Oriented CSR (Definition 1 / Figure 2 preprocessing): (off, cols, dhat)."""
        lib = _load()
        key = self._key(order_key)
        off = np.zeros(self.n + 1, dtype=np.int64)
        cols = np.zeros(max(self.m, 1), dtype=np.int32)
        dhat = np.zeros(self.n, dtype=np.int32)
        lib.orc_orient(self.n, _p(self.off, i64p), _p(self.adj, i32p),
                       _p(key, i64p) if key is not None else None,
                       _p(off, i64p), _p(cols, i32p), _p(dhat, i32p))
        return off, cols[: self.m], dhat

    def cost(self, order_key=None) -> int:
        """Theorem 2's cost sum_v d_v * dhat_v."""
        key = self._key(order_key)
        return int(_load().orc_cost(self.n, _p(self.off, i64p), _p(self.adj, i32p),
                                    _p(key, i64p) if key is not None else None))

    def vertex_triangles(self, v: int) -> int:
        """T_v by definition: edges among the neighbours of v."""
        return int(_load().orc_vertex_triangles(_p(self.off, i64p), _p(self.adj, i32p), int(v)))


def count(n: int, edges, order_key=None, local: bool = False, listing: bool = False):
    return Adjacency(n, edges).count(order_key, local, listing)


def clustering(deg: np.ndarray, tv: np.ndarray) -> np.ndarray:
    """C_v = 2 T_v / (d_v (d_v - 1)), 0 for d_v < 2."""
    d = np.ascontiguousarray(deg, dtype=np.int32)
    t = np.ascontiguousarray(tv, dtype=np.int64)
    cc = np.zeros(len(d), dtype=np.float64)
    _load().orc_clustering(len(d), _p(d, i32p), _p(t, i64p), _p(cc, f64p))
    return cc


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 (Salmon et al., SC'11): four 32-bit counter words and two
    32-bit key words in, four 32-bit words out."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox(_p(c, u32p), _p(k, u32p), _p(out, u32p))
    return out


def sparsify_keep(a: int, b: int, seed: int, q: float) -> bool:
    return bool(_load().orc_sparsify_keep(int(a), int(b), int(seed), float(q)))


def sparsify_count(n: int, edges, seed: int, q: float):
    """Section 9.1: returns (T' of the kept graph, kept edge count, T'/q^3)."""
    e = _edges(edges)
    T = ctypes.c_uint64(0)
    mk = ctypes.c_int64(0)
    est = ctypes.c_double(0.0)
    _check(_load().orc_sparsify_count(int(n), len(e), _p(e, i32p), int(seed), float(q),
                                      ctypes.byref(T), ctypes.byref(mk), ctypes.byref(est)))
    return int(T.value), int(mk.value), float(est.value)


# ---- load-balancing partition (Section "load balancing", Table "lbscheme") ----

COST_VERTICES, COST_DEGREE, COST_DHAT, COST_DEG_DHAT, COST_DHAT_SQ, COST_WORK = 0, 1, 2, 3, 4, 5


def partition_costs(n: int, edges, cost: int) -> np.ndarray:
    """f(v) of the paper's load-balancing schemes (Table "lbscheme"), with d_v the
    degree and dhat_v = |N_v| of the degree-ordered orientation:
    1, d_v, dhat_v, d_v * dhat_v, dhat_v^2, and sum over u in N_v of (dhat_v + dhat_u)."""
    adj = Adjacency(n, edges)
    off, cols, dhat = adj.orient()
    deg = adj.deg.astype(np.int64)
    dh = dhat.astype(np.int64)
    if cost == COST_VERTICES:
        return np.ones(n, dtype=np.int64)
    if cost == COST_DEGREE:
        return deg
    if cost == COST_DHAT:
        return dh
    if cost == COST_DEG_DHAT:
        return deg * dh
    if cost == COST_DHAT_SQ:
        return dh * dh
    if cost == COST_WORK:
        f = np.zeros(n, dtype=np.int64)
        for v in range(n):
            for u in cols[off[v]:off[v + 1]]:
                f[v] += dh[v] + dh[u]
        return f
    raise ValueError("unknown cost function")


def partition(n: int, edges, parts: int, cost: int):
    """The paper's partition of V into `parts` contiguous ranges: F(t) = f(0) + ... + f(t),
    alpha = F(n-1) / parts, and the boundary node of part j (0 < j < parts) is the
    smallest v with F(v) >= j * alpha (n if there is none); bounds[0] = 0,
    bounds[parts] = n.  Returns (bounds int64[parts+1], part costs int64[parts])."""
    f = partition_costs(n, edges, cost)
    F = np.cumsum(f) if n else np.zeros(0, dtype=np.int64)
    total = int(F[-1]) if n else 0
    bounds = [0]
    for j in range(1, parts):
        x = n
        for v in range(n):          # smallest v with parts * F(v) >= j * total, in exact integers
            if parts * int(F[v]) >= j * total:
                x = v
                break
        bounds.append(x)
    bounds.append(n)
    Fx = np.concatenate([[0], F]).astype(np.int64)
    costs = np.array([Fx[bounds[j + 1]] - Fx[bounds[j]] for j in range(parts)], dtype=np.int64)
    return np.array(bounds, dtype=np.int64), costs


def count_apex_range(n: int, edges, lo: int, hi: int):
    """Triangles whose first vertex in the order of Eq. (1) lies in [lo, hi), and each
    vertex's share of them: (count, tv int64[n]), from NodeIterator++'s listing, whose
    triples are written in that order (first vertex first)."""
    r = count(n, edges, listing=True)
    tri = r["tri"]
    sel = tri[(tri[:, 0] >= lo) & (tri[:, 0] < hi)]
    tv = np.bincount(sel.ravel(), minlength=n).astype(np.int64) if len(sel) else np.zeros(n, np.int64)
    return int(len(sel)), tv


# ---- sparsification with partition-local coins (Section 9.2) ----

def sparsify_keep_part(a: int, b: int, seed: int, q: float, part: int) -> bool:
    """The coin of edge {a, b} drawn by part `part`: Philox4x32-10 with counter
    (min, max, part, 0) and key (lo32(seed), hi32(seed)); with r the top 53 bits
    of the output words x0:x1, kept iff r * 2^-53 < q."""
    return bool(_load().orc_sparsify_keep_part(int(a), int(b), int(seed), float(q), int(part)))


def sparsify_count_part(n: int, edges, seed: int, q: float, part: int, lo: int, hi: int) -> int:
    """Figure "sparsification" run by one processor on its partition: the part keeps
    each edge by its own coin, and counts the triangles of the kept graph whose first
    vertex -- in the order of the ORIGINAL degrees -- lies in [lo, hi)."""
    e = _edges(edges)
    deg = Adjacency(n, e).deg.astype(np.int64)
    kept = np.array([p for p in e if sparsify_keep_part(int(p[0]), int(p[1]), seed, q, part)],
                    dtype=np.int32).reshape(-1, 2)
    tri = count(n, kept, order_key=deg, listing=True)["tri"]
    return int(((tri[:, 0] >= lo) & (tri[:, 0] < hi)).sum())
