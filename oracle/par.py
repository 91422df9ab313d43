"""Parallel CPU oracle -- TEST INFRASTRUCTURE ONLY.

Python access to ``tc_oracle_par.c``: the same definitions as the serial
oracle (full sorted adjacency, the oriented lists of Definition 1, the
triangle count with per-vertex and per-apex counts, the listing, the
sparsified count of Section 9.1), restated for all host cores so that the
full-size configurations are compared with a complete oracle result.  The
counting loop is NodeIteratorN (Figure 2) with a two-pointer merge of the two
sorted oriented lists.  Each function is pinned by equality with the serial
oracle on graphs the serial oracle is itself pinned on
(``tests/test_oracle_par.py``).

Only the tests, the smoke check and the benchmark's CPU legs use it; the
library under ``paper_1706_05151_gb300`` never imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import Adjacency, OracleError, ERRORS, _edges, _p, i32p, i64p, u64p

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "tc_oracle_par.c"), os.path.join(_HERE, "tc_oracle.c")]
_LIB_PATH = os.path.join(_HERE, "liboracle_par.so")
_lock = threading.Lock()
_lib = None

# the listing fingerprint's modulus (tc_oracle_par.c, orp_fingerprint)
FP_P = 2147483647
FP_A = (1103515245, 1664525)
FP_B = (12345, 1013904223)
FP_C = (2147480009, 305419896)


def build(force: bool = False) -> str:
    """Compile the parallel oracle (gcc -O2 -fopenmp) into ``liboracle_par.so``; the
    serial oracle's source is linked in for the sparsification coin."""
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(s) for s in _SRCS)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11"] + _SRCS + ["-o", tmp],
                   check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.orp_num_threads.restype = ctypes.c_int
        lib.orp_build_adjacency.restype = ctypes.c_int
        lib.orp_build_adjacency.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i64p, i32p]
        lib.orp_orient.restype = None
        lib.orp_orient.argtypes = [ctypes.c_int32, i64p, i32p, i64p, i64p, i32p, i32p]
        lib.orp_count.restype = ctypes.c_int
        lib.orp_count.argtypes = [ctypes.c_int32, i64p, i32p, u64p, i64p, i64p, u64p]
        lib.orp_list.restype = None
        lib.orp_list.argtypes = [ctypes.c_int32, i64p, i32p, i64p, i32p]
        lib.orp_fingerprint.restype = None
        lib.orp_fingerprint.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, u64p]
        lib.orp_sparsify_count.restype = ctypes.c_int
        lib.orp_sparsify_count.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, ctypes.c_uint64,
                                           ctypes.c_double, u64p, i64p]
        _lib = lib
        return lib


def _check(rc: int):
    if rc != 0:
        raise OracleError(ERRORS.get(rc, f"oracle error {rc}"))


def num_threads() -> int:
    return int(_load().orp_num_threads())


def adjacency(n: int, edges) -> Adjacency:
    """The full sorted adjacency N(v), built on all cores; the same object (and the
    same arrays) as ``oracle.Adjacency(n, edges)``."""
    lib = _load()
    e = _edges(edges)
    adj = Adjacency.__new__(Adjacency)
    adj.n, adj.m = int(n), len(e)
    adj.off = np.empty(adj.n + 1, dtype=np.int64)
    adj.adj = np.empty(max(2 * adj.m, 1), dtype=np.int32)
    _check(lib.orp_build_adjacency(adj.n, adj.m, _p(e, i32p), _p(adj.off, i64p), _p(adj.adj, i32p)))
    return adj


def orient(adj: Adjacency, order_key=None):
    """Oriented CSR (Definition 1) on all cores: (off int64[n+1], cols int32[m], dhat int32[n])."""
    lib = _load()
    key = None
    if order_key is not None:
        key = np.ascontiguousarray(np.asarray(order_key, dtype=np.int64))
        assert key.shape == (adj.n,)
    off = np.empty(adj.n + 1, dtype=np.int64)
    cols = np.empty(max(adj.m, 1), dtype=np.int32)
    dhat = np.empty(adj.n, dtype=np.int32)
    lib.orp_orient(adj.n, _p(adj.off, i64p), _p(adj.adj, i32p),
                   _p(key, i64p) if key is not None else None, _p(off, i64p), _p(cols, i32p), _p(dhat, i32p))
    return off, cols[: adj.m], dhat


def count(n: int, off: np.ndarray, cols: np.ndarray, local: bool = True, fingerprint: bool = False):
    """NodeIteratorN (Figure 2) on an oriented CSR.  Returns a dict with T and, if asked,
    ``tv`` (T_v), ``apex`` (triangles per first vertex) and ``fp`` (the listing fingerprint
    pair)."""
    lib = _load()
    off = np.ascontiguousarray(off, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    if len(cols) == 0:
        cols = np.zeros(1, dtype=np.int32)
    T = ctypes.c_uint64(0)
    tv = np.empty(n, dtype=np.int64) if local else None
    apex = np.empty(n, dtype=np.int64) if local else None
    fp = np.zeros(2, dtype=np.uint64) if fingerprint else None
    _check(lib.orp_count(int(n), _p(off, i64p), _p(cols, i32p), ctypes.byref(T),
                         _p(tv, i64p) if local else None, _p(apex, i64p) if local else None,
                         _p(fp, u64p) if fingerprint else None))
    out = {"T": int(T.value)}
    if local:
        out["tv"], out["apex"] = tv, apex
    if fingerprint:
        out["fp"] = (int(fp[0]), int(fp[1]))
    return out


def listing(n: int, off: np.ndarray, cols: np.ndarray, apex: np.ndarray) -> np.ndarray:
    """All triangles as int32[T, 3] rows (v, u, w), v before u before w in the order,
    grouped by apex v in id order (Figure "tlisting")."""
    lib = _load()
    off = np.ascontiguousarray(off, dtype=np.int64)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    if len(cols) == 0:
        cols = np.zeros(1, dtype=np.int32)
    apex_off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(apex, out=apex_off[1:])
    T = int(apex_off[-1])
    tri = np.empty((max(T, 1), 3), dtype=np.int32)
    lib.orp_list(int(n), _p(off, i64p), _p(cols, i32p), _p(apex_off, i64p), _p(tri, i32p))
    return tri[:T]


def fingerprint_of(v: int, u: int, w: int):
    """The two listing hashes of one triple (v, u, w), as the C side computes them."""
    out = np.zeros(2, dtype=np.uint64)
    _load().orp_fingerprint(int(v), int(u), int(w), _p(out, u64p))
    return int(out[0]), int(out[1])


def sparsify_count(n: int, edges, deg: np.ndarray, seed: int, q: float):
    """Section 9.1 on all cores: (T' of the kept graph, kept edge count, T'/q^3).  ``deg``
    are the original degrees, which fix the order of the kept graph."""
    e = _edges(edges)
    d = np.ascontiguousarray(deg, dtype=np.int32)
    T = ctypes.c_uint64(0)
    mk = ctypes.c_int64(0)
    _check(_load().orp_sparsify_count(int(n), len(e), _p(e, i32p), _p(d, i32p), int(seed), float(q),
                                      ctypes.byref(T), ctypes.byref(mk)))
    t = int(T.value)
    return t, int(mk.value), float(t) / (q * q * q)
