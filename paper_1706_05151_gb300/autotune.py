"""Autotuner for the counting kernels' cost bin.

The one threshold that changes how work is split is `tile_max`: apex vertices
whose oriented list N_v has more than tile_max ids are counted one thread
block per vertex, the others 32 to a warp.  Skewed graphs (R-MAT, Chung-Lu)
want a low threshold, so that the few heavy vertices do not leave one warp
working while the rest of the GPU idles; graphs with short lists (PA, ER) do
not care.  The tuner times tc_count on the graph itself for each candidate and
records the winner per graph-shape class in a JSON table, so that later runs
on graphs of the same shape start from it.  Results never depend on the
threshold; only the time does.
"""
from __future__ import annotations

import json
import math
import os

import torch

CANDIDATES = (32, 64, 128, 256, 512)
TABLE_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")


def shape_class(g) -> str:
    """Graph-shape key: log2 buckets of the largest and of the mean |N_v|."""
    if g.n == 0:
        return "empty"
    dmax = int(g.dhat.max().item()) if g.dhat is not None else int((g.offsets[1:] - g.offsets[:-1]).max().item())
    mean = g.m / max(g.n, 1)
    return f"dmax{int(math.log2(max(dmax, 1)))}_mean{int(math.log2(max(mean, 1)))}"


def load_table(path: str = TABLE_PATH) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_table(table: dict, path: str = TABLE_PATH):
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_count(tc, g, ctx, tile_max: int, repeats: int) -> float:
    ctx.set_tuning(tile_max, 1)
    out = torch.empty(1, dtype=torch.int64, device=ctx.device)
    tc.count(g, ctx, out=out)  # warm-up
    stream = torch.cuda.current_stream(ctx.device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(repeats):
        tc.count(g, ctx, out=out)
    e1.record(stream)
    torch.cuda.synchronize(ctx.device)
    return e0.elapsed_time(e1) / repeats


def tune(g, ctx=None, candidates=CANDIDATES, repeats: int = 3, record: bool = True, path: str = TABLE_PATH):
    """Time every candidate threshold on g; apply and (optionally) record the best.

    Returns (best tile_max, {candidate: ms}).
    """
    import paper_1706_05151_gb300 as tc
    ctx = ctx or tc.default_context()
    times = {t: time_count(tc, g, ctx, t, repeats) for t in candidates}
    best = min(times, key=times.get)
    ctx.set_tuning(best, 1)
    if record:
        table = load_table(path)
        table[shape_class(g)] = {"tile_max": best, "ms": {str(k): round(v, 4) for k, v in times.items()},
                                 "n": g.n, "m": g.m}
        save_table(table, path)
    return best, times


def apply(g, ctx=None, path: str = TABLE_PATH) -> int:
    """Use the recorded threshold for g's shape class (the default if none)."""
    import paper_1706_05151_gb300 as tc
    ctx = ctx or tc.default_context()
    rec = load_table(path).get(shape_class(g))
    best = int(rec["tile_max"]) if rec else 0
    ctx.set_tuning(best, 1)
    return best
