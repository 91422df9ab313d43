"""The several-GPU form of bench.py (independent replicas, one process per GPU)
on CPU: its rank aggregation run by two gloo processes."""
from __future__ import annotations

import importlib.util
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        b = _bench()
        cpu = torch.device("cpu")
        ms = b.max_over_ranks(10.0 + 5.0 * rank, cpu, world)       # rank 1 is the slow one
        units = b.sum_over_ranks(1000 * (rank + 1), cpu, world)      # 1000 + 2000
        seeds = [None] * world
        dist.all_gather_object(seeds, b.replica_seed(7, rank))
        out.put((rank, ms, units, b.job_throughput(units, ms), seeds))
    finally:
        dist.destroy_process_group()


def test_replicas_aggregate_over_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, units, value, seeds in res:
        assert ms == 15.0                      # the slowest rank's time
        assert units == 3000                   # every rank's edges
        assert value == pytest.approx(3000 / 0.015)
        assert len(set(seeds)) == world        # each replica counts its own graph


def test_single_process_needs_no_collective():
    b = _bench()
    assert b.max_over_ranks(3.5, torch.device("cpu"), 1) == 3.5
    assert b.sum_over_ranks(42, torch.device("cpu"), 1) == 42
