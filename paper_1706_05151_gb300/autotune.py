"""Autotuner for the counting kernels' cost bins.

Two thresholds change how work is split.  `tile_max`: apex vertices whose
oriented list N_v has more than tile_max ids are counted one thread block per
vertex, the others 32 to a warp.  Skewed graphs (R-MAT, Chung-Lu) want a low
threshold, so that the few heavy vertices do not leave one warp working while
the rest of the GPU idles; graphs with short lists (PA, ER) do not care.
`hub_min`: an edge (v, u) whose N_u has at least hub_min ids and more than N_v
is counted from u's side (N_u hashed once, the shorter N_v streamed).  Then
the kernels' own shapes: the warp-tile kernel's ids per warp and candidate
windows in flight (256 x 8, 256 x 4, 128 x 8), and the block and hub kernels'
lists per warp batch and windows in flight ((32, 4), (16, 4), (32, 8)).  The tuner times tc_count on the graph
itself for each candidate of tile_max, then of hub_min, then of the tile shape
and the hash-kernel shape, and records the winners per graph-shape class in a JSON
table, so that later runs on graphs of the same shape start from them.
Results never depend on any of these; only the time does.
"""
from __future__ import annotations

import json
import math
import os

import torch

CANDIDATES = (32, 64, 128, 256)
HUB_CANDIDATES = (-1, 32, 64, 128, 256)   # -1: hub side off
TILE_SHAPES = ((256, 8), (256, 4), (128, 8))  # the first is the default
HASH_SHAPES = ((32, 4), (16, 4), (32, 8))      # (lists per warp batch, windows in flight); the first is the default
TABLE_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")


def shape_class(g) -> str:
    """Graph-shape key: log2 buckets of the largest and of the mean |N_v|."""
    if g.n == 0:
        return "empty"
    dmax = int(g.dhat.max().item()) if g.dhat is not None else int((g.offsets[1:] - g.offsets[:-1]).max().item())
    mean = g.m / max(g.n, 1)
    return f"dmax{int(math.log2(max(dmax, 1)))}_mean{int(math.log2(max(mean, 1)))}"


def load_table(path: str = TABLE_PATH) -> dict:
    """The recorded thresholds by shape class; empty when the file is missing or not a JSON object."""
    try:
        with open(path) as f:
            table = json.load(f)
    except (OSError, ValueError):
        return {}
    return table if isinstance(table, dict) else {}


def save_table(table: dict, path: str = TABLE_PATH):
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_count(tc, g, ctx, tile_max: int, repeats: int, hub_min: int = 0, local: bool = False,
               shape=None) -> float:
    """ms of one tc_count (or, with local, one per-vertex tc_count_local) at these thresholds
    (and kernel shape: ((tile ids, windows), (hash batch, hash windows)), None = the defaults)."""
    ctx.set_tuning(tile_max, 1)
    ctx.set_hub_min(hub_min)
    (tile_ids, windows), (hb, hw) = shape or (TILE_SHAPES[0], HASH_SHAPES[0])
    ctx.set_kernel_shape(tile_ids, windows, hb, hw)
    if local:
        def run():
            tc.count_local(g, clustering=False, ctx=ctx)
    else:
        out = torch.empty(1, dtype=torch.int64, device=ctx.device)

        def run():
            tc.count(g, ctx, out=out)
    run()  # warm-up
    stream = torch.cuda.current_stream(ctx.device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(repeats):
        run()
    e1.record(stream)
    torch.cuda.synchronize(ctx.device)
    return e0.elapsed_time(e1) / repeats


def tune(g, ctx=None, candidates=CANDIDATES, repeats: int = 3, record: bool = True, path: str = TABLE_PATH,
         hub_candidates=HUB_CANDIDATES, local: bool = False, shapes: bool = True, info: dict | None = None):
    """Time every candidate tile_max on g, then every hub_min at the best
    tile_max, then (shapes) every tile shape and hash-kernel shape at those; apply
    and (optionally) record the winners.  local: time the per-vertex pass
    (tc_count_local) instead of the plain count.  info, if given, receives the
    shape search: {"tile_shape": [ids, windows], "hash_shape": [batch, windows],
    "shape_ms": {...}}.

    Returns (best tile_max, {candidate: ms}, best hub_min, {candidate: ms}).
    """
    import paper_1706_05151_gb300 as tc
    ctx = ctx or tc.default_context()
    times = {t: time_count(tc, g, ctx, t, repeats, local=local) for t in candidates}
    best = min(times, key=times.get)
    hub_times = {h: time_count(tc, g, ctx, best, repeats, h, local=local) for h in hub_candidates}
    best_hub = min(hub_times, key=hub_times.get)
    best_shape = (TILE_SHAPES[0], HASH_SHAPES[0])
    shape_ms = {}
    if shapes:
        tile_ms = {TILE_SHAPES[0]: hub_times[best_hub]}
        for ts in TILE_SHAPES[1:]:
            tile_ms[ts] = time_count(tc, g, ctx, best, repeats, best_hub, local=local, shape=(ts, HASH_SHAPES[0]))
        best_tile = min(tile_ms, key=tile_ms.get)
        hs_ms = {HASH_SHAPES[0]: tile_ms[best_tile]}
        for hs in HASH_SHAPES[1:]:
            hs_ms[hs] = time_count(tc, g, ctx, best, repeats, best_hub, local=local, shape=(best_tile, hs))
        best_shape = (best_tile, min(hs_ms, key=hs_ms.get))
        shape_ms = {f"tile{ts[0]}x{ts[1]}": round(v, 4) for ts, v in tile_ms.items()}
        shape_ms.update({f"hash{hs[0]}x{hs[1]}": round(v, 4) for hs, v in hs_ms.items()})
    ctx.set_tuning(best, 1)
    ctx.set_hub_min(best_hub)
    ctx.set_kernel_shape(best_shape[0][0], best_shape[0][1], best_shape[1][0], best_shape[1][1])
    if info is not None:
        info.update({"tile_shape": list(best_shape[0]), "hash_shape": list(best_shape[1]), "shape_ms": shape_ms})
    if record:
        table = load_table(path)
        table[shape_class(g)] = {"tile_max": best, "ms": {str(k): round(v, 4) for k, v in times.items()},
                                 "hub_min": best_hub,
                                 "hub_ms": {str(k): round(v, 4) for k, v in hub_times.items()},
                                 "tile_shape": list(best_shape[0]), "hash_shape": list(best_shape[1]),
                                 "shape_ms": shape_ms, "n": g.n, "m": g.m}
        save_table(table, path)
    return best, times, best_hub, hub_times


def apply(g, ctx=None, path: str = TABLE_PATH):
    """Use the recorded thresholds and kernel shapes for g's shape class (the defaults if
    none); returns (tile_max, hub_min)."""
    import paper_1706_05151_gb300 as tc
    ctx = ctx or tc.default_context()
    rec = load_table(path).get(shape_class(g))
    best = int(rec["tile_max"]) if rec else 0
    hub = int(rec.get("hub_min", 0)) if rec else 0
    tile = rec.get("tile_shape", [0, 0]) if rec else [0, 0]
    hs = rec.get("hash_shape", [0, 0]) if rec else [0, 0]
    ctx.set_tuning(best, 1)
    ctx.set_hub_min(hub)
    ctx.set_kernel_shape(int(tile[0]), int(tile[1]), int(hs[0]), int(hs[1]))
    return best, hub
