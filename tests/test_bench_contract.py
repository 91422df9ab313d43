"""bench.py on the CPU: the reference arm's JSON line, and no CPU fallback for the GPU arm.

The reference arm times the oracle on host cores, so its whole contract can be
checked here on a tiny sample.  The GPU arm must refuse to run without a GPU
rather than fall back to any CPU path.
"""
from __future__ import annotations

import json
import os
import subprocess
import sys

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*args, timeout=300):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                          capture_output=True, text=True, timeout=timeout)


def test_reference_arm_prints_one_contract_line():
    r = _bench("--impl", "reference", "--steps", "2", "--warmup", "1", "--ref-log-n", "9")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["higher_is_better"] is True
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    assert "2^9" in cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the behaviour without a GPU")
def test_gpu_arm_fails_loudly_without_a_gpu():
    r = _bench("--steps", "1", "--warmup", "1", "--e2e-steps", "0", "--no-cpu-baseline", timeout=120)
    assert r.returncode != 0
    # no measurement line: there is no CPU fallback for the CUDA path
    assert not any(ln.strip().startswith("{") for ln in r.stdout.splitlines())


def _bench_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_clock_summary_of_nvidia_smi_rows():
    bench = _bench_module()
    quiet = "2070, 2070, 910.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
    capped = "1965, 2070, 1399.8, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
    hot = "1500, 2070, 1200.0, 0x0000000000000040, Not Active, Active, Not Active, Not Active"
    samples = [(0.0, hot), (1.0, quiet), (1.1, capped), (1.2, quiet), (1.3, "garbage"), (1.35, "[N/A], 2070"),
               (5.0, hot)]
    # only the rows inside the timed window (1.0 .. 1.3, with 0.15 s of slack) count
    s = bench.ClockSampler.summarize(samples, (1.0, 1.3))
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    # a window with no rows falls back to the last three samples
    s = bench.ClockSampler.summarize(samples, (10.0, 11.0))
    assert s["reasons"] == ["hw_thermal_slowdown"] and s["samples"] == 1
    assert bench.ClockSampler.summarize([], None) is None


def test_serving_size_classes_and_request_weights():
    bench = _bench_module()
    assert bench.size_class(1 << 21) == "small" and bench.size_class((1 << 21) + 1) == "medium"
    assert bench.size_class(1 << 25) == "medium" and bench.size_class(260_000_000) == "large"
    ms = [32_768, 1_000_000, 62_000_000, 260_000_000]
    p = bench.request_weights(ms)
    assert abs(p.sum() - 1.0) < 1e-12 and all(a > b for a, b in zip(p, p[1:]))
    # proportional to m^(-1/2): the ratio of two graphs' shares is the root of their sizes' ratio
    assert abs(p[0] / p[3] - (ms[3] / ms[0]) ** 0.5) < 1e-9


def test_cpu_baselines_agree_on_the_sample_they_time():
    # the single-core and all-cores CPU baselines run the same step: the same T on the same graph
    import bench
    import synth
    n = 1 << 12
    e = synth.ba(n, 8, 3)
    dt, m, T = bench.cpu_oracle_pipeline(n, e, 0.1, 3)
    pdt, pm, pT, threads = bench.cpu_parallel_pipeline(n, e, 0.1, 3)
    assert (m, T) == (pm, pT) and T > 0
    assert threads >= 1 and dt > 0 and pdt > 0
