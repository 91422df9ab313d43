"""Seeded synthetic graph inputs, shared by the CPU oracle and the CUDA path.

This module holds no triangle-counting arithmetic.  It only makes undirected
simple edge lists -- ``int32[m, 2]`` numpy arrays, each edge once, written
``(lo, hi)`` with ``lo < hi`` unless a helper says otherwise -- for the paper's
workload classes (Section "Preliminaries", Datasets: Gnp and PA(n, d)) plus
R-MAT and Chung-Lu stand-ins for skewed real graphs, and small closed-form
graphs (complete, cycle, wheel, star, bipartite, trees) used as fixtures.

The random generators live in ``graphgen.c`` (Philox4x64-10, OpenMP), built
on first use with the host C compiler.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB_PATH = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

i32p = ctypes.POINTER(ctypes.c_int32)
f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile ``graphgen.c`` into ``libsynth.so`` beside it (gcc, OpenMP)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.gen_er.restype = ctypes.c_int64
        lib.gen_er.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, i32p, ctypes.c_int64]
        lib.gen_ba.restype = ctypes.c_int64
        lib.gen_ba.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, i32p, ctypes.c_int64]
        lib.gen_rmat.restype = ctypes.c_int64
        lib.gen_rmat.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_uint64, i32p, ctypes.c_int64]
        lib.gen_chung_lu.restype = ctypes.c_int64
        lib.gen_chung_lu.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                     ctypes.c_uint64, i32p, ctypes.c_int64, ctypes.c_int]
        lib.gen_batch_params.restype = None
        lib.gen_batch_params.argtypes = [ctypes.c_int32, ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, i32p, f64p]
        lib.gen_ba_max_edges.restype = ctypes.c_int64
        lib.gen_ba_max_edges.argtypes = [ctypes.c_int32, ctypes.c_int32]
        lib.gen_num_threads.restype = ctypes.c_int
        _lib = lib
        return lib


def _finish(buf: np.ndarray, m: int, what: str) -> np.ndarray:
    if m < 0:
        raise RuntimeError(f"{what}: generator failed with code {m}")
    return np.ascontiguousarray(buf[:m])


def er(n: int, draws: int, seed: int) -> np.ndarray:
    """G(n, M) Erdos-Renyi: `draws` uniform endpoint pairs, loops dropped, duplicates merged."""
    lib = _load()
    buf = np.empty((max(draws, 1), 2), dtype=np.int32)
    m = lib.gen_er(n, draws, seed, buf.ctypes.data_as(i32p), draws)
    return _finish(buf, m, "er")


def ba(n: int, k: int, seed: int) -> np.ndarray:
    """Preferential attachment PA(n, d = 2k): K_k seed, k endpoint-copy edges per new vertex."""
    lib = _load()
    cap = lib.gen_ba_max_edges(n, k)
    buf = np.empty((max(cap, 1), 2), dtype=np.int32)
    m = lib.gen_ba(n, k, seed, buf.ctypes.data_as(i32p), cap)
    return _finish(buf, m, "ba")


def rmat(scale: int, edge_factor: int, seed: int, a: float = 0.57, b: float = 0.19,
         c: float = 0.19) -> np.ndarray:
    """R-MAT graph on 2**scale vertices from edge_factor * 2**scale samples (symmetrised, merged)."""
    lib = _load()
    samples = edge_factor << scale
    buf = np.empty((max(samples, 1), 2), dtype=np.int32)
    m = lib.gen_rmat(scale, edge_factor, a, b, c, seed, buf.ctypes.data_as(i32p), samples)
    return _finish(buf, m, "rmat")


def chung_lu(n: int, dbar: float, gamma: float, seed: int, stream: int = 0, threads: int = 0) -> np.ndarray:
    """Chung-Lu graph with weights (i+1)^(-1/(gamma-1)) and floor(n*dbar/2) endpoint pairs."""
    lib = _load()
    pairs = int(math.floor(n * dbar / 2.0))
    buf = np.empty((max(pairs, 1), 2), dtype=np.int32)
    m = lib.gen_chung_lu(n, dbar, gamma, seed, stream, buf.ctypes.data_as(i32p), pairs, threads)
    return _finish(buf, m, "chung_lu")


def batch_params(num_graphs: int, seed: int, nlo: float = 100.0, nhi: float = 100000.0,
                 dlo: float = 8.0, dhi: float = 64.0):
    """Per-graph (n_g, dbar_g) of the batched workload: n log-uniform, dbar uniform."""
    lib = _load()
    ns = np.empty(num_graphs, dtype=np.int32)
    ds = np.empty(num_graphs, dtype=np.float64)
    lib.gen_batch_params(num_graphs, seed, nlo, nhi, dlo, dhi, ns.ctypes.data_as(i32p),
                         ds.ctypes.data_as(f64p))
    return ns, ds


def batch_graphs(num_graphs: int, seed: int, gamma: float = 2.1, **kw):
    """The batched workload: a list of (n_g, edges_g) Chung-Lu graphs with per-graph streams."""
    import concurrent.futures as cf
    ns, ds = batch_params(num_graphs, seed, **kw)
    # one graph per worker thread (ctypes releases the GIL), each generated single-threaded
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        edges = list(ex.map(lambda g: chung_lu(int(ns[g]), float(ds[g]), gamma, seed, stream=g, threads=1),
                            range(num_graphs)))
    return list(zip((int(n) for n in ns), edges))


def num_threads() -> int:
    return int(_load().gen_num_threads())


# ---- closed-form fixtures -------------------------------------------------

def _pairs(pairs) -> np.ndarray:
    arr = np.array(sorted((min(a, b), max(a, b)) for a, b in pairs), dtype=np.int32)
    return arr.reshape(-1, 2)


def complete(n: int) -> np.ndarray:
    return _pairs((i, j) for i in range(n) for j in range(i + 1, n))


def cycle(n: int) -> np.ndarray:
    return _pairs((i, (i + 1) % n) for i in range(n)) if n >= 3 else np.zeros((0, 2), np.int32)


def wheel(k: int) -> np.ndarray:
    """Hub 0 joined to every vertex of the rim cycle 1..k."""
    rim = [(1 + i, 1 + (i + 1) % k) for i in range(k)]
    return _pairs([(0, 1 + i) for i in range(k)] + rim)


def star(k: int) -> np.ndarray:
    return _pairs((0, 1 + i) for i in range(k))


def complete_bipartite(a: int, b: int) -> np.ndarray:
    return _pairs((i, a + j) for i in range(a) for j in range(b))


def random_tree(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return _pairs((v, int(rng.integers(0, v))) for v in range(1, n))


def relabel(edges: np.ndarray, perm: np.ndarray) -> np.ndarray:
    """Apply the vertex permutation v -> perm[v] and re-canonicalise each pair."""
    e = perm[edges]
    return np.ascontiguousarray(np.stack([e.min(axis=1), e.max(axis=1)], axis=1).astype(np.int32))


def shuffle_edges(edges: np.ndarray, seed: int, flip: bool = True) -> np.ndarray:
    """Random edge order and, optionally, random direction of each pair (the input
    contract takes each undirected edge once, in any order and direction)."""
    rng = np.random.default_rng(seed)
    e = edges[rng.permutation(len(edges))].copy()
    if flip and len(e):
        f = rng.integers(0, 2, len(e)).astype(bool)
        e[f] = e[f][:, ::-1]
    return np.ascontiguousarray(e)
