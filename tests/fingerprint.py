"""The listing fingerprint computed over a triangle list held in a tensor.

A listing of ~10^10 triples does not fit in host memory, so the full-size
tests compare it with the oracle as a set: each row (v, u, w) is hashed by two
degree-4 polynomials modulo P = 2^31 - 1 (the parallel oracle's
``orp_fingerprint``, written out again here in tensor operations) and the
hashes are summed mod P.  Every intermediate stays below 2^62, so signed
64-bit tensor arithmetic never wraps.  With the row count equal and no row
repeated (checked separately), two different lists agree only by a collision
of both sums.
"""
from __future__ import annotations

import torch

from oracle.par import FP_A, FP_B, FP_C, FP_P


def _hash(k: int, v: torch.Tensor, u: torch.Tensor, w: torch.Tensor) -> torch.Tensor:
    x = (v * FP_A[k]) % FP_P
    x = (x + u) % FP_P
    x = (x * FP_A[k]) % FP_P
    x = (x + w) % FP_P
    y = (x * x + FP_B[k]) % FP_P
    return (y * y + FP_C[k]) % FP_P


def listing_fingerprint(tri: torch.Tensor, chunk: int = 1 << 26):
    """(sum of hash 0, sum of hash 1) mod P over the rows of an int32[T, 3] tensor (any device)."""
    s0 = s1 = 0
    for s in range(0, tri.shape[0], chunk):
        t = tri[s:s + chunk].to(torch.int64)
        v, u, w = t[:, 0], t[:, 1], t[:, 2]
        # a chunk's sum of values below 2^31 stays below 2^57
        s0 = (s0 + int(_hash(0, v, u, w).sum().item())) % FP_P
        s1 = (s1 + int(_hash(1, v, u, w).sum().item())) % FP_P
    return s0, s1
