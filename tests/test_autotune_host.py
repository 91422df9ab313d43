"""The threshold autotuner's host logic, on the CPU with a fake timer and context.

Timing needs a GPU; choosing the winners, tuning hub_min at the best tile_max,
recording them per graph-shape class and applying them later do not.
"""
from __future__ import annotations

import json
from types import SimpleNamespace

import pytest
import torch

from paper_1706_05151_gb300 import autotune


class FakeCtx:
    def __init__(self):
        self.calls = []

    def set_tuning(self, tile_max, grid_div):
        self.calls.append(("tile_max", tile_max, grid_div))

    def set_hub_min(self, hub_min):
        self.calls.append(("hub_min", hub_min))

    def set_kernel_shape(self, tile_ids, windows, hash_batch, hash_windows):
        self.calls.append(("shape", tile_ids, windows, hash_batch, hash_windows))


def fake_graph(n, m, dmax):
    dhat = torch.zeros(max(n, 1), dtype=torch.int32)
    if n:
        dhat[0] = dmax
    return SimpleNamespace(n=n, m=m, dhat=dhat, offsets=None)


def test_shape_class_buckets_by_log2():
    assert autotune.shape_class(fake_graph(0, 0, 0)) == "empty"
    assert autotune.shape_class(fake_graph(1024, 16 * 1024, 300)) == "dmax8_mean4"
    assert autotune.shape_class(fake_graph(1024, 16 * 1024, 511)) == "dmax8_mean4"
    assert autotune.shape_class(fake_graph(1024, 16 * 1024, 512)) == "dmax9_mean4"
    assert autotune.shape_class(fake_graph(10, 5, 1)) == "dmax0_mean0"


def test_tune_picks_fastest_then_tunes_hub_at_it_and_records(tmp_path, monkeypatch):
    tile_ms = {32: 5.0, 64: 4.0, 128: 3.0, 256: 3.5}
    hub_ms = {-1: 2.9, 32: 3.1, 64: 2.5, 128: 2.7, 256: 2.8}
    seen = []

    def fake_time(tc, g, ctx, tile_max, repeats, hub_min=0, local=False, shape=None):
        seen.append((tile_max, hub_min, local, shape))
        if shape is not None:
            return {((256, 4), (32, 4)): 2.4, ((128, 8), (32, 4)): 2.6, ((256, 4), (16, 4)): 2.45,
                    ((256, 4), (32, 8)): 2.3}[shape]
        return tile_ms[tile_max] if hub_min == 0 else hub_ms[hub_min]

    monkeypatch.setattr(autotune, "time_count", fake_time)
    path = str(tmp_path / "tuning.json")
    g, ctx = fake_graph(4096, 65536, 700), FakeCtx()
    info = {}
    best, times, hub, hub_times = autotune.tune(g, ctx=ctx, repeats=1, path=path, local=True, info=info)
    assert (best, hub) == (128, 64)
    assert times == tile_ms and hub_times == hub_ms
    # hub_min candidates are all timed at the winning tile_max, on the per-vertex pass
    assert [s[:3] for s in seen if s[1] != 0 and s[3] is None] == \
        [(128, h, True) for h in autotune.HUB_CANDIDATES if h != 0]
    # then the other tile shapes at both winners, then the other hash-kernel shapes at the best tile shape
    assert [s for s in seen if s[3] is not None] == [
        (128, 64, True, ((256, 4), (32, 4))), (128, 64, True, ((128, 8), (32, 4))),
        (128, 64, True, ((256, 4), (16, 4))), (128, 64, True, ((256, 4), (32, 8)))]
    assert info["tile_shape"] == [256, 4] and info["hash_shape"] == [32, 8]
    assert info["shape_ms"] == {"tile256x8": 2.5, "tile256x4": 2.4, "tile128x8": 2.6, "hash32x4": 2.4,
                                "hash16x4": 2.45, "hash32x8": 2.3}
    assert ctx.calls[-3:] == [("tile_max", 128, 1), ("hub_min", 64), ("shape", 256, 4, 32, 8)]
    rec = json.load(open(path))[autotune.shape_class(g)]
    assert rec["tile_max"] == 128 and rec["hub_min"] == 64 and rec["n"] == 4096 and rec["m"] == 65536
    assert rec["tile_shape"] == [256, 4] and rec["hash_shape"] == [32, 8]
    # a later run on a graph of the same shape class starts from the recorded choices
    ctx2 = FakeCtx()
    assert autotune.apply(fake_graph(4000, 64000, 600), ctx=ctx2, path=path) == (128, 64)
    assert ctx2.calls == [("tile_max", 128, 1), ("hub_min", 64), ("shape", 256, 4, 32, 8)]
    # another shape class falls back to the defaults (0 = the library's own)
    assert autotune.apply(fake_graph(4096, 65536, 5000), ctx=FakeCtx(), path=path) == (0, 0)


def test_tune_without_record_leaves_the_table_alone(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "time_count",
                        lambda tc, g, ctx, t, r, h=0, local=False, shape=None: float(t + (h or 0)))
    path = tmp_path / "tuning.json"
    autotune.tune(fake_graph(100, 800, 20), ctx=FakeCtx(), repeats=1, path=str(path), record=False)
    assert not path.exists()


@pytest.mark.parametrize("content", ["", "{not json", "[]"])
def test_unreadable_table_reads_as_empty(tmp_path, content):
    path = tmp_path / "tuning.json"
    path.write_text(content)
    assert autotune.load_table(str(path)) == {}
    assert autotune.load_table(str(tmp_path / "missing.json")) == {}


def test_save_table_replaces_atomically(tmp_path):
    path = str(tmp_path / "tuning.json")
    autotune.save_table({"a": {"tile_max": 64}}, path)
    autotune.save_table({"b": {"tile_max": 32}}, path)
    assert json.load(open(path)) == {"b": {"tile_max": 32}}
    assert [p.name for p in tmp_path.iterdir()] == ["tuning.json"]
