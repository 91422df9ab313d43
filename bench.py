#!/usr/bin/env python3
"""Benchmark of the triangle-counting hot path on GB300.

One step = the whole hot path over one synthetic graph already resident in
HBM: orientation by the degree order (tc_orient), exact count with per-vertex
counts, clustering coefficients and the two-pass triangle list (tc_analyze),
and edge sparsification at q = 0.1 (tc_sparsify_count).  The metric is oriented edges per second (m per step),
with the intersection kernel's achieved fraction of the measured HBM roofline.

Default workload (the headline): preferential attachment PA(n = 2^27, 16
edges per new vertex), ~2.15G undirected edges (edge list 17.2 GB, larger
than L2, so no L2 flush is needed between steps).  The same line carries the
same measurement for PA(n = 2^24) and R-MAT scale 24 under "workloads".

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload ba27|ba24|rmat24|er] [--also ba24,rmat24]
    python bench.py --impl reference   # the CPU oracle on a bounded sample
Multi-GPU (torchrun, one rank per GPU): each rank counts its own independent
graph (different seed); no collective on the data path (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "oriented edges/sec & HBM roofline %"
UNIT = "oriented edges/s"

WORKLOADS = {
    "ba24": dict(kind="ba", n=1 << 24, k=16, label="preferential attachment PA(n=2^24, k=16)"),
    "ba27": dict(kind="ba", n=1 << 27, k=16, label="preferential attachment PA(n=2^27, k=16)"),
    "rmat24": dict(kind="rmat", scale=24, ef=16, label="R-MAT scale 24, edge factor 16 (0.57/0.19/0.19/0.05)"),
    "er": dict(kind="er", n=16384, draws=131072, label="Erdos-Renyi G(n=16384, M=131072 draws)"),
    "ba22": dict(kind="ba", n=1 << 22, k=16, label="preferential attachment PA(n=2^22, k=16)"),
    "rmat22": dict(kind="rmat", scale=22, ef=16, label="R-MAT scale 22, edge factor 16 (0.57/0.19/0.19/0.05)"),
    "rmat20": dict(kind="rmat", scale=20, ef=16, label="R-MAT scale 20, edge factor 16 (0.57/0.19/0.19/0.05)"),
}


def make_graph(w: dict, seed: int):
    import synth
    if w["kind"] == "ba":
        return w["n"], synth.ba(w["n"], w["k"], seed)
    if w["kind"] == "rmat":
        return 1 << w["scale"], synth.rmat(w["scale"], w["ef"], seed)
    return w["n"], synth.er(w["n"], w["draws"], seed)


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def source_sha(*names) -> str:
    h = hashlib.sha256()
    for nm in names:
        with open(os.path.join(ROOT, "paper_1706_05151_gb300", "csrc", nm), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary, if it matches the current source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except Exception:
        return None
    for r in rec.get("records", []):
        if r.get("kernel") == kernel and r.get("workload") == workload and r.get("covers_pass") and \
                r.get("source_sha") == source_sha(*r.get("sources", [])):
            return float(r["dram_bytes_per_launch"])
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.samples = []
        self.proc = None
        self.window = None
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
        if gpu_id:
            cmd += ["-i", gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), line.strip()))

    def mark(self, start: float, end: float):
        self.window = (start, end)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        return self.summarize(self.samples, self.window)

    @staticmethod
    def summarize(samples, window):
        """Median SM clock, max clock and active throttle reasons of the (time, csv line)
        samples taken inside the window (with 0.15 s of slack), else of the last three."""
        lo, hi = window if window else (0, 1e18)
        rows = [s for t, s in samples if lo - 0.15 <= t <= hi + 0.15] or [s for _, s in samples[-3:]]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            parts = [p.strip() for p in r.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_pipeline(n, e, q, seed):
    """The oracle's version of one step: adjacency, NodeIterator++ with T_v and
    listing, clustering, and the sparsified count.  Returns (seconds, m, T)."""
    import oracle
    t0 = time.perf_counter()
    adj = oracle.Adjacency(n, e)
    r = adj.count(local=True, listing=True)
    oracle.clustering(adj.deg, r["tv"])
    oracle.sparsify_count(n, e, seed, q)
    return time.perf_counter() - t0, len(e), r["T"]


def cpu_parallel_pipeline(n, e, q, seed):
    """The same step on all host cores: the parallel oracle's adjacency, orientation,
    NodeIteratorN (Figure 2) with T_v, the listing, clustering and the sparsified
    count.  Returns (seconds, m, T, threads)."""
    import oracle
    from oracle import par
    t0 = time.perf_counter()
    adj = par.adjacency(n, e)
    off, cols, _ = par.orient(adj)
    r = par.count(n, off, cols, local=True)
    par.listing(n, off, cols, r["apex"])
    oracle.clustering(adj.deg, r["tv"])
    par.sparsify_count(n, e, adj.deg, seed, q)
    return time.perf_counter() - t0, len(e), r["T"], par.num_threads()


def run_reference(args, rank):
    if rank != 0:
        return 0
    import synth
    sample_n = 1 << args.ref_log_n
    n, e = sample_n, synth.ba(sample_n, 16, args.seed)
    times = []
    for i in range(args.warmup + args.steps):
        dt, m, T = cpu_oracle_pipeline(n, e, args.q, args.seed)
        if i >= args.warmup:
            times.append(dt)
    t = statistics.mean(times)
    value = len(e) / t
    sample = (f"CPU oracle (NodeIterator++, 1 thread) on PA(n=2^{args.ref_log_n}, k=16), m={len(e)}, "
              f"full step: adjacency, T, T_v, listing, C_v, sparsified count q={args.q}")
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload]["label"], "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)
    return 0


def bench_batched(tc, ctx, dev, args, rank):
    """The batched form (one launch sequence over G graphs) against the plain
    per-graph-launch form (tc_orient + tc_count_local per graph) on the same GPU."""
    import ctypes
    import torch
    import synth
    graphs = synth.batch_graphs(args.batch_graphs, 4096 + replica_seed(args.seed, rank))
    b = tc.make_batch(graphs, dev)
    G, N, E = b.G, b.N, b.E
    stream = torch.cuda.current_stream(dev)
    # batched: time K calls at the default thresholds and shapes, then tuned on the union
    # (outside the timing); the per-graph arm below is timed both ways as well
    totals, tv, union = tc.batch(b, True, ctx)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.batch_steps):
        tc.batch(b, True, ctx)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    batched_default_ms = e0.elapsed_time(e1) / args.batch_steps
    tuned = None
    if not args.no_tune:
        from paper_1706_05151_gb300 import autotune
        shape = {}
        best, times, hub, hub_times = autotune.tune(union, ctx, record=False, local=True, info=shape)
        tuned = {"tile_max": best, "count_ms_by_tile_max": {str(k): round(v, 3) for k, v in times.items()},
                 "hub_min": hub, "count_ms_by_hub_min": {str(k): round(v, 3) for k, v in hub_times.items()},
                 "tile_shape": shape.get("tile_shape"), "hash_shape": shape.get("hash_shape"),
                 "count_ms_by_shape": shape.get("shape_ms")}
    del union
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.batch_steps):
        totals, tv, _ = tc.batch(b, True, ctx)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    batched_ms = e0.elapsed_time(e1) / args.batch_steps
    # the same sequence recorded once as a CUDA graph and replayed (tc_capture_begin / tc_capture_end)
    cap = tc.CapturedBatch(b, True, ctx)
    cap.replay(stream)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(args.batch_steps):
        cap.replay(stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    captured_ms = e0.elapsed_time(e1) / args.batch_steps
    captured_same = bool(torch.equal(cap.totals, totals)) and bool(torch.equal(cap.tv[:N], tv))
    captured_kernels = cap.kernels
    cap.close()
    del cap
    # per graph: one tc_orient + tc_count_local launch sequence per graph, no host wait in between
    lib = ctx.lib
    offsets = torch.empty(N + G, dtype=torch.int64, device=dev)
    cols = torch.empty(max(E, 1), dtype=torch.int32, device=dev)
    deg = torch.empty(max(N, 1), dtype=torch.int32, device=dev)
    dhat = torch.empty(max(N, 1), dtype=torch.int32, device=dev)
    tv1 = torch.empty(max(N, 1), dtype=torch.int64, device=dev)
    tot1 = torch.zeros(G, dtype=torch.int64, device=dev)
    nmax = max(n for n, _ in graphs)
    mmax = max(len(e) for _, e in graphs)
    ws = torch.empty(max(ctx.workspace_size(tc.TC_OP_ORIENT, nmax, mmax),
                         ctx.workspace_size(tc.TC_OP_COUNT, nmax, mmax)), dtype=torch.uint8, device=dev)
    vb = b.vbase.cpu().numpy()
    eb = b.ebase.cpu().numpy()
    hs = ctypes.c_void_p(stream.cuda_stream)
    ep, op, cp, dp, hp = b.edges.data_ptr(), offsets.data_ptr(), cols.data_ptr(), deg.data_ptr(), dhat.data_ptr()
    tvp, tp, wsp, wsn = tv1.data_ptr(), tot1.data_ptr(), ws.data_ptr(), ws.numel()

    def per_graph():
        for g in range(G):
            n, m = int(vb[g + 1] - vb[g]), int(eb[g + 1] - eb[g])
            o = op + 8 * (int(vb[g]) + g)
            c = cp + 4 * int(eb[g])
            ctx.check(lib.tc_orient(ctx.handle, n, m, ctypes.c_void_p(ep + 8 * int(eb[g])), ctypes.c_void_p(o),
                                    ctypes.c_void_p(c), ctypes.c_void_p(dp + 4 * int(vb[g])),
                                    ctypes.c_void_p(hp + 4 * int(vb[g])), ctypes.c_void_p(wsp), wsn, hs))
            gs = tc.TcGraph(n, m, o, c, dp + 4 * int(vb[g]), hp + 4 * int(vb[g]))
            ctx.check(lib.tc_count_local(ctx.handle, ctypes.byref(gs), ctypes.c_void_p(tp + 8 * g),
                                         ctypes.c_void_p(tvp + 8 * int(vb[g])), None, ctypes.c_void_p(wsp), wsn, hs))

    def time_per_graph():
        ctx.set_async(True)
        try:
            per_graph()  # warm-up
            torch.cuda.synchronize(dev)
            e0.record(stream)
            per_graph()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ctx.status()
        finally:
            ctx.set_async(False)
        return e0.elapsed_time(e1)

    # the per-graph form with the thresholds and shapes tuned on the union (the same as the
    # batched arm's), then with the defaults
    per_graph_tuned_ms = time_per_graph()
    same = bool(torch.equal(tot1, totals)) and bool(torch.equal(tv1[:N], tv))
    ctx.set_tuning(0, 1)
    ctx.set_hub_min(0)
    ctx.set_kernel_shape(0, 0, 0, 0)
    per_graph_ms = time_per_graph()
    same = same and bool(torch.equal(tot1, totals)) and bool(torch.equal(tv1[:N], tv))
    return {"workload": f"{G} Chung-Lu graphs (gamma 2.1), n log-uniform in [100, 1e5], mean degree U[8, 64]",
            "graphs": G, "vertices": N, "edges": E, "triangles": int(totals.sum().item()),
            "tuning": "speedup: both arms with the thresholds and shapes tuned on the union; "
                      "speedup_default: both arms with the library defaults",
            "batched_ms": batched_ms, "per_graph_ms": per_graph_tuned_ms,
            "speedup": per_graph_tuned_ms / batched_ms,
            "batched_default_ms": batched_default_ms, "per_graph_default_ms": per_graph_ms,
            "speedup_default": per_graph_ms / batched_default_ms,
            "captured_ms": captured_ms, "captured_speedup": per_graph_tuned_ms / captured_ms,
            "captured_kernels_per_replay": captured_kernels, "captured_results_equal": captured_same,
            "batched_edges_per_s": E / (batched_ms * 1e-3), "results_equal": same, "autotune": tuned}


def bench_partition(tc, ctx, g, T, dev, parts: int = 8):
    """The paper's load-balancing step on this graph: parts by the vertex-count
    scheme (f = 1) and by the work scheme (f = sum over N_v of dhat_v + dhat_u),
    each part counted by apex range; reports cost and measured-time imbalance
    (max / mean) and checks that the parts sum to T."""
    import torch
    stream = torch.cuda.current_stream(dev)
    out = {"parts": parts}
    for label, cost in (("vertices", tc.COST_VERTICES), ("work", tc.COST_WORK)):
        b, c = tc.partition(g, parts, cost, ctx)
        b = b.cpu().numpy()
        c = c.cpu().numpy().astype(np.float64)
        total = torch.zeros(1, dtype=torch.int64, device=dev)
        ms = []
        for j in range(parts):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            tc.count_range(g, int(b[j]), int(b[j + 1]), total, None, ctx)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms.append(e0.elapsed_time(e1))
        ms = np.array(ms)
        out[label] = {"bounds": [int(x) for x in b], "cost_imbalance": float(c.max() / max(c.mean(), 1e-30)),
                      "part_ms": [round(float(x), 3) for x in ms],
                      "time_imbalance": float(ms.max() / max(ms.mean(), 1e-30)),
                      "parts_sum_to_T": int(total.item()) == T}
    return out


def bench_orders(tc, ctx, edges_dev, n, T, dev, seed):
    """Section "An Optimal Node Ordering" on this graph: the counting cost
    W = sum_v d_v * dhat_v and the measured orientation and count times under
    the id, degree and random orders (Theorem 3: the degree order minimises W)."""
    import torch
    stream = torch.cuda.current_stream(dev)
    g0 = tc.orient(edges_dev, n, ctx)
    gen = torch.Generator(device="cpu").manual_seed(seed)
    keys = {"id": torch.zeros(n, dtype=torch.int64, device=dev),
            "degree": g0.deg.to(torch.int64),
            "random": torch.randperm(n, generator=gen).to(dev)}
    del g0
    out = {}
    for name, k in keys.items():
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        g = tc.orient(edges_dev, n, ctx, keys=k)
        e1.record(stream)
        t = tc.count(g, ctx)
        e2.record(stream)
        torch.cuda.synchronize(dev)
        W = int((g.deg.to(torch.int64) * g.dhat.to(torch.int64)).sum().item())
        out[name] = {"W": W, "orient_ms": round(e0.elapsed_time(e1), 3), "count_ms": round(e1.elapsed_time(e2), 3),
                     "triangles_equal": t == T}
        del g
        torch.cuda.empty_cache()
    return out


def bench_sparsify_accuracy(tc, ctx, g, T, dev, q, seeds: int = 25, parts: int = 8):
    """Section 9.2's accuracy comparison on this graph: the estimate T'/q^3 over
    `seeds` independent runs, with one coin per edge (DOULION) and with
    partition-local coins (each of `parts` work-balanced parts draws its own)."""
    import torch
    b, _ = tc.partition(g, parts, tc.COST_WORK, ctx)
    b = b.cpu().numpy()
    plain, parted = [], []
    for s in range(seeds):
        t, _, _ = tc.sparsify_count(g, q, 1000 + s, ctx)
        plain.append(t / q ** 3)
        kept = torch.zeros(1, dtype=torch.int64, device=dev)
        for j in range(parts):
            tc.sparsify_count_part(g, q, 1000 + s, j, int(b[j]), int(b[j + 1]), kept, ctx)
        parted.append(int(kept.item()) / q ** 3)

    def stats(x):
        x = np.array(x)
        err = np.abs(x - T) / T if T else np.zeros_like(x)
        return {"mean_estimate": float(x.mean()), "variance": float(x.var(ddof=1)),
                "mean_rel_error": float(err.mean()), "max_rel_error": float(err.max())}
    return {"q": q, "seeds": seeds, "parts": parts, "T": T, "one_coin_per_edge": stats(plain),
            "partition_local_coins": stats(parted)}


def bench_host_resident(tc, ctx, g, T, dev):
    """The count with the oriented CSR in page-locked host memory (graphs that do not fit
    in the device memory left free): read by the kernels over the CPU-GPU link (zero
    copy), and streamed through a device list buffer (tc_count_streamed)."""
    import torch
    h = tc.Graph(g.n, g.m, g.offsets.cpu().pin_memory(), g.cols.cpu().pin_memory(), g.deg.cpu().pin_memory(),
                 g.dhat.cpu().pin_memory())
    stream = torch.cuda.current_stream(dev)
    out = torch.empty(1, dtype=torch.int64, device=dev)
    tc.count(h, ctx, out=out)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(3):
        tc.count(h, ctx, out=out)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / 3
    zero_copy = {"count_ms": round(ms, 3), "edges_per_s": g.m / (ms * 1e-3), "triangles_equal": int(out.item()) == T,
                 "csr_bytes": 8 * (g.n + 1) + 4 * g.m + 8 * g.n}
    # the same CSR streamed through a device list buffer of half its lists' bytes
    # (tc_count_streamed: resident target ranges of a quarter, apex chunks streamed past them)
    list_bytes = 2 * g.m
    off_h, cols_h = h.offsets, h.cols
    ranges = int(np.ceil(g.m / (list_bytes // 8)))
    tc.count_streamed(off_h, cols_h, list_bytes, ctx=ctx)
    t0 = time.perf_counter()
    Ts = tc.count_streamed(off_h, cols_h, list_bytes, ctx=ctx)[0]
    sms = (time.perf_counter() - t0) * 1e3
    host_bytes = (ranges + 1) * 4 * g.m + 8 * (g.n + 1)
    streamed = {"count_ms": round(sms, 3), "edges_per_s": g.m / (sms * 1e-3), "triangles_equal": Ts == T,
                "list_buffer_bytes": list_bytes, "target_ranges_about": ranges, "host_bytes_read": host_bytes,
                "host_link_gb_s": host_bytes / (sms * 1e-3) / 1e9,
                "timing": "wall clock around the synchronous call (host planning, copies and kernels)"}
    return {"zero_copy": zero_copy, "streamed": streamed}


SIZE_CLASSES = (("small", 1 << 21), ("medium", 1 << 25), ("large", 1 << 62))


def size_class(m: int) -> str:
    """Requests are grouped by their graph's edge count: small (m <= 2^21, the server's
    high-priority class by default), medium (m <= 2^25), large."""
    for name, top in SIZE_CLASSES:
        if m <= top:
            return name
    return "large"


def serving_pool():
    """The serving configuration's graph pool (seeded): ER n = 2^12..2^18 with mean
    degree 16, R-MAT scale 16..24 with edge factor 16, Chung-Lu (gamma 2.1) with
    n = 1e4..1e6 and mean degree 16."""
    import synth
    pool = []
    for lg in (12, 14, 16, 18):
        pool.append((f"ER n=2^{lg}", 1 << lg, synth.er(1 << lg, 8 << lg, 100 + lg)))
    for sc in (16, 18, 20, 22, 24):
        pool.append((f"R-MAT scale {sc}", 1 << sc, synth.rmat(sc, 16, 200 + sc)))
    for n in (10 ** 4, 10 ** 5, 10 ** 6):
        pool.append((f"Chung-Lu n={n}", n, synth.chung_lu(n, 16.0, 2.1, 300, n)))
    return pool


def request_weights(ms) -> np.ndarray:
    """Probability that a request targets each graph: proportional to m^(-1/2), so that
    most requests hit small graphs while each of the largest still gets dozens per
    10,000 (R-MAT scale 24 about 0.4%)."""
    w = np.array([1.0 / np.sqrt(max(m, 1)) for m in ms])
    return w / w.sum()


def bench_serving(tc, dev, args):
    """Poisson arrivals of count / local / list requests (60/30/10) on resident graphs."""
    import threading
    import torch
    free, _ = torch.cuda.mem_get_info(dev)
    pool_bytes = int(min(args.serve_pool_gb * 1e9, free - 8e9))
    srv = tc.Server(pool_bytes, slots=8)
    graphs = serving_pool()
    gids = [srv.add_graph(n, e) for _, n, e in graphs]
    m_of = {gid: len(e) for gid, (_, _, e) in zip(gids, graphs)}
    class_of = {gid: size_class(len(e)) for gid, (_, _, e) in zip(gids, graphs)}
    pg = request_weights([len(e) for _, _, e in graphs])
    kinds_p = [0.6, 0.3, 0.1]
    # capacity: mean service time of the mix, one request at a time
    service = {}
    for gid in gids:
        for kind in range(3):
            srv.wait(srv.submit(gid, kind), timeout_ms=600000, copy=False)
            t0 = time.perf_counter()
            for _ in range(2):
                srv.wait(srv.submit(gid, kind), timeout_ms=600000, copy=False)
            service[(gid, kind)] = (time.perf_counter() - t0) / 2
    mean_service = sum(pg[i] * kinds_p[k] * service[(g, k)] for i, g in enumerate(gids) for k in range(3))
    capacity = 1.0 / mean_service
    out = {"workload": "; ".join(name for name, _, _ in graphs), "pool_gb": pool_bytes / 1e9, "slots": 8,
           "mix": "60% count, 30% local (T_v, C_v), 10% list",
           "graph_choice": "probability proportional to m^(-1/2)",
           "request_share": {name: round(float(p), 5) for (name, _, _), p in zip(graphs, pg)},
           "size_classes": "small m <= 2^21, medium m <= 2^25, large above",
           "service_ms": {f"{name}/{('count', 'local', 'list')[k]}": round(service[(gid, k)] * 1e3, 3)
                          for (name, _, _), gid in zip(graphs, gids) for k in range(3)},
           "sequential_capacity_rps": capacity, "rates": []}
    for li, load in enumerate(float(x) for x in args.serve_loads.split(",")):
        rate = load * capacity
        warm = 500
        total = warm + args.serve_requests
        rng = np.random.default_rng(1000 + li)
        arrivals = np.cumsum(rng.exponential(1.0 / rate, total))
        kinds = rng.choice(3, total, p=kinds_p)
        which = rng.choice(len(gids), total, p=pg)
        tickets = [None] * total
        ready = threading.Semaphore(0)
        t_start = time.perf_counter()

        def submitter():
            for i in range(total):
                target = t_start + arrivals[i]
                while True:
                    now = time.perf_counter()
                    if now >= target:
                        break
                    if target - now > 0.0004:
                        time.sleep(target - now - 0.0002)
                tickets[i] = (srv.submit(gids[which[i]], int(kinds[i])), time.perf_counter())
                ready.release()

        th = threading.Thread(target=submitter)
        th.start()
        lat, lat_kind, edges, statuses = [], {0: [], 1: [], 2: []}, 0, {}
        lat_class = {name: [] for name, _ in SIZE_CLASSES}
        t_first = None
        for i in range(total):
            ready.acquire()
            tk, t_sub = tickets[i]
            r = srv.wait(tk, timeout_ms=600000, copy=False)
            statuses[r.status] = statuses.get(r.status, 0) + 1
            if i >= warm:
                if t_first is None:
                    t_first = t_sub
                lat.append(r.latency_ms)
                lat_kind[r.kind].append(r.latency_ms)
                lat_class[class_of[r.graph_id]].append(r.latency_ms)
                edges += m_of[r.graph_id]
        th.join()
        t_last = time.perf_counter()
        span = t_last - t_first
        la = np.array(lat)

        def pct(v, p):
            return float(np.percentile(v, p)) if v else None
        out["rates"].append({
            "offered_rps": rate, "load": load, "requests": len(lat), "achieved_rps": len(lat) / span,
            "p50_ms": float(np.percentile(la, 50)), "p99_ms": float(np.percentile(la, 99)),
            "p50_ms_by_kind": {k: pct(v, 50) for k, v in zip(("count", "local", "list"), lat_kind.values()) if v},
            "p99_ms_by_kind": {k: pct(v, 99) for k, v in zip(("count", "local", "list"), lat_kind.values()) if v},
            "by_size_class": {c: {"requests": len(v), "p50_ms": pct(v, 50), "p99_ms": pct(v, 99)}
                              for c, v in lat_class.items() if v},
            "edges_per_s": edges / span, "statuses": {str(k): v for k, v in statuses.items()}})
    out["stats"] = srv.stats()
    srv.close()
    return out


# ---- replicas on several GPUs (one process per GPU; no collective on the data path) ----

def replica_seed(seed: int, rank: int) -> int:
    """Each rank counts its own independent graph of the same workload."""
    return seed + rank


def max_over_ranks(x: float, device, world: int) -> float:
    """The slowest rank's time (the job's time): an all-reduce MAX, or x alone."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: int, device, world: int) -> int:
    """Units processed by the whole job: an all-reduce SUM, or x alone."""
    if world <= 1:
        return int(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([int(x)], dtype=torch.int64, device=device)
    dist.all_reduce(t)
    return int(t.item())


def job_throughput(units_all_ranks: int, ms_slowest: float) -> float:
    """value: every rank's units over the slowest rank's time."""
    return units_all_ranks / (ms_slowest * 1e-3)


def run_e2e(args, tc, ctx, dev, edges_host, n, T, q, seed, tri_buf, barrier, world, steps):
    """The step end to end through the public API: H2D of the edge list and D2H of
    T_v, C_v, the sparsified count and the listing inside the timed region.  The
    edge list goes up through tc_orient_host (chunked copies overlapped with the
    degree pass); T_v, C_v and the listing come back on a second stream while the
    sparsified count runs, the listing through a page-locked staging buffer of at
    most 2 GiB, chunk by chunk (a 10^10-triple listing is larger than the host's
    memory).  Returns (ms per step, max over ranks; H2D bytes; D2H bytes)."""
    import torch
    stream = torch.cuda.current_stream(dev)
    side = torch.cuda.Stream(dev)
    tv_host = torch.empty(n, dtype=torch.int64).pin_memory()
    cc_host = torch.empty(n, dtype=torch.float64).pin_memory()
    stage_rows = max(1, min(T, (2 << 30) // 12))
    tri_host = torch.empty((stage_rows, 3), dtype=torch.int32).pin_memory()
    ed_buf = torch.empty((max(len(edges_host), 1), 2), dtype=torch.int32, device=dev)  # the caller's device copy

    def one():
        g2, _ = tc.orient_host(edges_host, n, ctx, edges_dev=ed_buf)
        T2, tv2, cc2, tri2 = tc.analyze(g2, True, tri_buf[0], ctx)
        ready = torch.cuda.Event()
        ready.record(stream)
        side.wait_event(ready)
        with torch.cuda.stream(side):
            tv_host.copy_(tv2, non_blocking=True)
            cc_host.copy_(cc2, non_blocking=True)
            for s0 in range(0, len(tri2), stage_rows):
                r = min(stage_rows, len(tri2) - s0)
                tri_host[:r].copy_(tri2[s0:s0 + r], non_blocking=True)
                if s0 + r < len(tri2):
                    side.synchronize()  # the staging buffer is read out before the next chunk
        tc.sparsify_count(g2, q, seed, ctx)  # its two counts come back to the host inside the call
        side.synchronize()
        stream.synchronize()

    one()  # untimed: the caching allocator takes this path's device buffers once
    barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        one()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = e0.elapsed_time(e1) / steps
    h2d = int(edges_host.numel()) * 4
    d2h = 16 * n + 12 * T + 8 + 16  # T_v, C_v, the listing, T, and the two sparsified counts
    return max_over_ranks(e2e_ms, dev, world), h2d, d2h


def gpu_identity(torch, dev, local_rank):
    try:
        gpu_id = str(torch.cuda.get_device_properties(dev).uuid)
        return gpu_id if gpu_id.startswith("GPU-") else "GPU-" + gpu_id
    except Exception:
        return str(local_rank)


ORIENT_STAGES = ("orient.degree", "orient.orient_count", "orient.scan", "orient.scatter", "orient.sort_small",
                 "orient.sort_mid", "orient.sort_big")
LOCAL_STAGES = ("local.prep", "local.tile", "local.block", "local.hub")


def measure_workload(args, tc, ctx, dev, name, steps, warmup, e2e_steps, world, rank, local_rank, barrier,
                     keep=False):
    """One workload: W untimed steps, the thresholds autotuned on the per-vertex pass,
    then K timed steps on the device (CUDA events, clocks sampled), then the e2e steps.
    Returns (record, state); state holds the graph for the side studies when keep."""
    import torch
    w = WORKLOADS[name]
    n, e_np = make_graph(w, replica_seed(args.seed, rank))
    m = len(e_np)
    edges_host = torch.from_numpy(e_np).pin_memory()
    del e_np
    edges_dev = edges_host.to(dev)
    q, seed = args.q, args.seed
    tri_buf = [None]

    def step():
        g = tc.orient(edges_dev, n, ctx)
        T, tv, cc, tri = tc.analyze(g, True, tri_buf[0], ctx)
        tri_buf[0] = tri if tri_buf[0] is None or len(tri) > tri_buf[0].shape[0] else tri_buf[0]
        sp = tc.sparsify_count(g, q, seed, ctx)
        return g, T, tv, cc, tri, sp

    ctx.set_tuning(0, 1)
    ctx.set_hub_min(0)
    ctx.set_kernel_shape(0, 0, 0, 0)
    for _ in range(max(warmup, 1)):
        g, T, tv, cc, tri, sp = step()
    tuned = None
    if not args.no_tune:  # pick the cost-bin thresholds on this graph (outside the timed region)
        from paper_1706_05151_gb300 import autotune
        # tuned on the per-vertex pass: with the listing write pass it is most of the step
        shape = {}
        best, times, hub, hub_times = autotune.tune(g, ctx, record=False, local=True, info=shape)
        tuned = {"tile_max": best, "local_ms_by_tile_max": {str(k): round(v, 3) for k, v in times.items()},
                 "hub_min": hub, "local_ms_by_hub_min": {str(k): round(v, 3) for k, v in hub_times.items()},
                 "tile_shape": shape.get("tile_shape"), "hash_shape": shape.get("hash_shape"),
                 "local_ms_by_shape": shape.get("shape_ms")}
        g, T, tv, cc, tri, sp = step()
    W = int((g.deg.to(torch.int64) * g.dhat.to(torch.int64)).sum().item())
    assert int(tv.sum().item()) == 3 * T and len(tri) == T
    del g, tv, cc, tri

    sampler = ClockSampler(gpu_identity(torch, dev, local_rank))
    time.sleep(0.3)
    ctx.reset_stats()
    ctx.set_profiling(True)
    stream = torch.cuda.current_stream(dev)
    barrier()
    torch.cuda.synchronize(dev)
    t_wall0 = time.time()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        out = step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    t_wall1 = time.time()
    ctx.set_profiling(False)
    launches = ctx.launches
    stages = ctx.stages()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / steps, dev, world)
    sampler.mark(t_wall0, t_wall1)
    clocks = sampler.stop()
    g, T, tv, cc, tri, sp = out
    del out

    e2e = None
    if e2e_steps > 0:
        if not keep:
            del g, tv, cc, tri
            torch.cuda.empty_cache()
        e2e_ms, h2d, d2h = run_e2e(args, tc, ctx, dev, edges_host, n, T, q, seed, tri_buf, barrier, world,
                                   e2e_steps)
        m_all = sum_over_ranks(m, dev, world)
        e2e = {"value": job_throughput(m_all, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms, "steps": e2e_steps,
               "listing_d2h": "through a page-locked staging buffer of at most 2 GiB, chunk by chunk"}
    m_total = sum_over_ranks(m, dev, world)

    peak, peak_src = load_peaks()
    # every kernel of the per-vertex counting pass: preparation (int32 offsets, hub
    # schedule), tile, block and hub kernels
    inter_ms = sum(stages.get(k, (0.0, 0))[0] for k in LOCAL_STAGES)
    inter_calls = max(stages.get("local.tile", (0.0, 0))[1], 1)
    inter_avg_ms = inter_ms / inter_calls
    b_alg = 4 * W + 4 * m + 8 * (n + 1)
    achieved = b_alg / (inter_avg_ms * 1e-3) / 1e9
    orient_ms = sum(stages.get(k, (0.0, 0))[0] for k in ORIENT_STAGES) / steps
    b_orient = 8 * m + 4 * m + 8 * (n + 1) + 4 * n
    rec = {
        "workload": w["label"], "n": n, "m": m, "triangles": T, "W_sum_d_dhat": W,
        "value": job_throughput(m_total, ms), "unit": UNIT, "steps": steps, "warmup": warmup,
        "ms_per_step": ms,
        "l2": "inputs larger than L2 (edge list %.2f GB, CSR %.2f GB): no flush between steps" % (
            8 * m / 1e9, (4 * m + 8 * n) / 1e9),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": recorded_traffic("local.tile", name),
                     "kernel": "k_count_tile+k_count_block+hub side, per-vertex pass of tc_analyze",
                     "algorithmic_bytes": b_alg, "avg_launch_ms": inter_avg_ms, "peak_source": peak_src},
        "orient_roofline": {"bound": "hbm", "algorithmic_bytes": b_orient, "avg_launch_ms": orient_ms,
                            "achieved": b_orient / (orient_ms * 1e-3) / 1e9 if orient_ms else None,
                            "frac": (b_orient / (orient_ms * 1e-3) / 1e9 / peak) if orient_ms else None,
                            "unit": "GB/s", "peak": peak},
        "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
        "stages_ms_per_step": {k: round(v[0] / steps, 4) for k, v in sorted(stages.items())},
        "autotune": tuned,
        "sparsified": {"kept_edges": sp[1], "kept_triangles": sp[0], "estimate": sp[2],
                       "rel_error": abs(sp[2] - T) / T if T else None},
    }
    state = None
    if keep:
        state = dict(g=g, T=T, n=n, m=m, edges_dev=edges_dev)
    else:
        del edges_dev
    del edges_host
    tri_buf.clear()
    torch.cuda.empty_cache()
    return rec, state


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tc", choices=["tc", "reference"])
    ap.add_argument("--workload", default="ba27", choices=sorted(WORKLOADS))
    ap.add_argument("--also", default="ba24,rmat24",
                    help="more workloads measured the same way, reported under 'workloads' (empty: none)")
    ap.add_argument("--also-steps", type=int, default=5)
    ap.add_argument("--q", type=float, default=0.1)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--also-e2e-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-log-n", type=int, default=20, help="log2 n of the CPU-baseline sample")
    ap.add_argument("--cpu-par-log-n", type=int, default=22,
                    help="log2 n of the all-cores CPU-baseline sample (0: skip)")
    ap.add_argument("--ref-log-n", type=int, default=18, help="log2 n of each reference-arm step")
    ap.add_argument("--batch-graphs", type=int, default=4096,
                    help="graphs of the batched Chung-Lu workload (0 skips the batched measurement)")
    ap.add_argument("--batch-steps", type=int, default=3)
    ap.add_argument("--serve-requests", type=int, default=10000,
                    help="requests measured per arrival rate (0 skips the serving measurement)")
    ap.add_argument("--serve-loads", default="0.5,0.85", help="arrival rates as fractions of measured capacity")
    ap.add_argument("--serve-pool-gb", type=float, default=150.0)
    ap.add_argument("--no-tune", action="store_true", help="skip the tile/block threshold autotuner")
    ap.add_argument("--no-partition", dest="partition", action="store_false",
                    help="skip the load-balancing partition report")
    ap.add_argument("--no-orders", dest="orders", action="store_false",
                    help="skip the node-ordering report (id, degree, random orders)")
    ap.add_argument("--no-sparsify-study", dest="sparsify_study", action="store_false",
                    help="skip the 25-seed sparsification accuracy report")
    ap.add_argument("--no-host-study", dest="host_study", action="store_false",
                    help="skip the count with the CSR in host memory")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)

    import torch
    import torch.distributed as dist
    import paper_1706_05151_gb300 as tc
    from paper_1706_05151_gb300 import build as tcbuild

    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if rank == 0 or world == 1:
        tcbuild.build()
    if world > 1:
        dist.barrier()
    ctx = tc.Context(local_rank)

    def barrier():
        if world > 1:
            dist.barrier()

    head, st = measure_workload(args, tc, ctx, dev, args.workload, args.steps, args.warmup, args.e2e_steps,
                                world, rank, local_rank, barrier, keep=True)
    g, T, n, edges_dev = st["g"], st["T"], st["n"], st["edges_dev"]
    del st
    part = bench_partition(tc, ctx, g, T, dev) if world == 1 and args.partition else None
    orders = bench_orders(tc, ctx, edges_dev, n, T, dev, args.seed) if world == 1 and args.orders else None
    spacc = bench_sparsify_accuracy(tc, ctx, g, T, dev, args.q) if world == 1 and args.sparsify_study else None
    host = bench_host_resident(tc, ctx, g, T, dev) if world == 1 and args.host_study else None
    del g, edges_dev
    torch.cuda.empty_cache()

    others = {}
    for nm in [x for x in args.also.split(",") if x and x != args.workload]:
        others[nm], _ = measure_workload(args, tc, ctx, dev, nm, args.also_steps, args.warmup,
                                         args.also_e2e_steps, world, rank, local_rank, barrier)
    ctx.set_tuning(0, 1)
    ctx.set_hub_min(0)
    ctx.set_kernel_shape(0, 0, 0, 0)

    batched = None
    if args.batch_graphs > 0:
        batched = bench_batched(tc, ctx, dev, args, rank)
    serving = None
    if args.serve_requests > 0 and world == 1:
        torch.cuda.empty_cache()
        serving = bench_serving(tc, dev, args)

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            import synth
            sn = 1 << args.cpu_log_n
            se = synth.ba(sn, 16, args.seed)
            dt, sm, _ = cpu_oracle_pipeline(sn, se, args.q, args.seed)
            cpu = {"value": sm / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"CPU oracle (NodeIterator++, 1 thread) full step on PA(n=2^{args.cpu_log_n}, "
                             f"k=16), m={sm}: adjacency, T, T_v, listing, C_v, sparsified count; {dt:.1f} s"}
            if args.cpu_par_log_n > 0:
                pn = 1 << args.cpu_par_log_n
                pe = synth.ba(pn, 16, args.seed)
                pdt, pm, _, threads = cpu_parallel_pipeline(pn, pe, args.q, args.seed)
                cpu["all_cores"] = {
                    "value": pm / pdt, "unit": UNIT, "cores": threads, "kind": "oracle (OpenMP NodeIteratorN)",
                    "sample": f"parallel CPU oracle (NodeIteratorN, {threads} threads) full step on "
                              f"PA(n=2^{args.cpu_par_log_n}, k=16), m={pm}: adjacency, orientation, T, T_v, "
                              f"listing, C_v, sparsified count; {pdt:.1f} s"}
        out = {
            "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": head["workload"], "n": head["n"], "m": head["m"], "triangles": head["triangles"],
                       "W_sum_d_dhat": head["W_sum_d_dhat"], "q": args.q, "seed": args.seed,
                       "step": "tc_orient + tc_analyze(T, T_v, C_v, triangle list) + tc_sparsify_count(q)",
                       "l2": head["l2"],
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "autotune": head["autotune"]},
            "roofline": head["roofline"],
            "orient_roofline": head["orient_roofline"],
            "e2e": head["e2e"],
            "gpu_launches": head["gpu_launches"],
            "clocks": head["clocks"],
            "stages_ms_per_step": head["stages_ms_per_step"],
            "cpu_baseline": cpu,
            "workloads": others,
            "partition": part,
            "orders": orders,
            "sparsify_accuracy": spacc,
            "host_resident_csr": host,
            "batched": batched,
            "serving": serving,
            "sparsified": head["sparsified"],
        }
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
