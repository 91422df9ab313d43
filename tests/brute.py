"""Independent brute-force references for tiny graphs (pure Python / numpy).

These restate the plain definitions of the Preliminaries without any order,
orientation or intersection, so they pin the oracle from outside.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def edge_set(edges) -> set:
    return {(min(int(a), int(b)), max(int(a), int(b))) for a, b in np.asarray(edges).reshape(-1, 2)}


def triangles_by_triples(n: int, edges) -> list:
    """Every {x, y, z} with all three pairs in E, as sorted tuples (definition)."""
    es = edge_set(edges)
    out = []
    for x, y, z in itertools.combinations(range(n), 3):
        if (x, y) in es and (y, z) in es and (x, z) in es:
            out.append((x, y, z))
    return out


def triangles_by_neighbours(n: int, edges) -> list:
    """Same set, enumerated from each edge's common neighbours (faster, still plain)."""
    es = edge_set(edges)
    nb = [set() for _ in range(n)]
    for a, b in es:
        nb[a].add(b)
        nb[b].add(a)
    out = set()
    for a, b in es:
        for c in nb[a] & nb[b]:
            out.add(tuple(sorted((a, b, c))))
    return sorted(out)


def adjacency_matrix(n: int, edges) -> np.ndarray:
    A = np.zeros((n, n), dtype=np.int64)
    e = np.asarray(edges).reshape(-1, 2)
    A[e[:, 0], e[:, 1]] = 1
    A[e[:, 1], e[:, 0]] = 1
    return A


def trace_cubed(n: int, edges):
    """T = trace(A^3)/6 and T_v = (A^3)_vv / 2, in exact int64 arithmetic."""
    A = adjacency_matrix(n, edges)
    A3 = A @ A @ A
    return int(np.trace(A3)) // 6, np.diagonal(A3).astype(np.int64) // 2


def per_vertex_from_list(n: int, tris) -> np.ndarray:
    tv = np.zeros(n, dtype=np.int64)
    for t in tris:
        for v in t:
            tv[v] += 1
    return tv


def edge_triangle_pairs(tris) -> int:
    """k of Eq. (var1): pairs of triangles that share an edge = sum_e C(t_e, 2)."""
    cnt = {}
    for x, y, z in tris:
        for e in ((x, y), (y, z), (x, z)):
            e = (min(e), max(e))
            cnt[e] = cnt.get(e, 0) + 1
    return sum(c * (c - 1) // 2 for c in cnt.values())


def canon(tri) -> np.ndarray:
    """Canonical form of a triangle list: each triple sorted, rows sorted."""
    t = np.sort(np.asarray(tri, dtype=np.int64).reshape(-1, 3), axis=1)
    if len(t) == 0:
        return t
    order = np.lexsort((t[:, 2], t[:, 1], t[:, 0]))
    return t[order]


def clique_with_pendants(k: int, a: int, width: int = 4):
    """K_k plus k*a/width pendant vertices, pendant j joined to clique vertices
    width*j .. width*j + width - 1 (mod k): every clique vertex gets exactly `a`
    pendants, so clique degrees stay equal and the order of Eq. (1) among them
    is by id -- clique vertex 0 has the longest list (k - 1 ids) and every
    pendant (degree width) precedes it.  Closed forms: T = C(k,3) + P*C(width,2);
    T_v = C(k-1,2) + (width-1)*a on the clique, C(width,2) on a pendant."""
    assert (k * a) % width == 0
    P = k * a // width
    clique = np.array([(i, j) for i in range(k) for j in range(i + 1, k)], dtype=np.int32)
    pend = np.empty((P * width, 2), dtype=np.int32)
    j = np.repeat(np.arange(P), width)
    pend[:, 0] = (width * j + np.tile(np.arange(width), P)) % k
    pend[:, 1] = k + j
    e = np.concatenate([clique, pend])
    T = math.comb(k, 3) + P * math.comb(width, 2)
    tv = np.concatenate([np.full(k, math.comb(k - 1, 2) + (width - 1) * a, np.int64),
                         np.full(P, math.comb(width, 2), np.int64)])
    return k + P, e, T, tv
