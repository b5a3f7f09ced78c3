#!/usr/bin/env python3
"""Benchmark of the traffic-matrix hot path on one B300 (or N replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (default, "stream"): an accumulated packet stream of 2^26 packets in
512 windows of 2^17 -- RMAT scale 32 with (a,b,c,d) = (0.57,0.19,0.19,0.05)
plus 10% uniform background pairs, anonymized by a seeded 32-bit bijection --
with the summed traffic matrix A and its nine Table 2 quantities produced
after every window, one library call per window (plain per-window launches).

One step = reset A, then for each window one ns_window_ingest_stats call:
build + accumulate fused, with the statistics of the updated A written into a
device array by the same launch; the per-window call sequence is captured
into a CUDA graph and replayed.  `value` times K steps with inputs resident in HBM; `e2e`
adds, every step, the host-to-device copy of the step's packets from pinned
memory (in chunks on a copy stream, overlapped with the ingest of earlier
chunks) and the device-to-host copy of the 512 statistics rows.

Prints one JSON line.  Under torchrun (N > 1) every rank runs an independent
replica of the stream on its own GPU (no data-path collective) and rank 0
reports the whole-job throughput over the slowest rank.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "packets/s to traffic matrix+stats, %HBM roofline; batched vs plain; p99 latency"
UNIT = "packets/s"
WINDOWS = 512
WINDOW = 1 << 17
PROFILE = os.path.join(ROOT, "profiles", "k_insert_packets.stream_rmat_window_2p17.md")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2509_03653_b300", "csrc", f)
                  for f in ("ns_hash.cu", "ns_common.cuh")]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=15.0,
                    help="seconds of oracle work for the cpu_baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="stream", choices=["stream", "oneshot", "batched", "serve", "anonymize", "slide"],
                    help="stream: 512 windows of 2^17 with stats after each (default); "
                         "oneshot: one 2^30-packet build, sort path vs hash path; "
                         "batched: 8192 uneven windows, batched launch vs plain per-window launches; "
                         "serve: Poisson arrivals at 80%% of capacity, p50/p99 window-to-stats latency; "
                         "anonymize: distinct addresses, random permutation and gather over the one-shot input; "
                         "slide: the stream's windows with per-window and sliding-window quantities")
    ap.add_argument("--serve-windows", type=int, default=448, help="serve: windows per phase")
    ap.add_argument("--serve-cache", default="off", choices=["auto", "on", "off"],
                    help="serve: per-CTA staging of the service's context (RMAT windows: off)")
    ap.add_argument("--batch-windows", type=int, default=8192, help="batched: number of windows")
    ap.add_argument("--tuner-cache", default=None, help="batched: autotuner cache file (default: none, tune now)")
    ap.add_argument("--packets", type=int, default=1 << 30, help="oneshot / anonymize: packets in the input")
    ap.add_argument("--paths", default="sort,hash", help="oneshot: aggregation paths to run")
    ap.add_argument("--slide-windows", type=int, default=8, help="slide: windows in the sliding sum (K)")
    ap.add_argument("--hash-load", type=float, default=0.25,
                    help="stream: load bound of the accumulated matrix's hash tables (sizes them for 2^26 links)")
    ap.add_argument("--windows", type=int, default=WINDOWS,
                    help="windows in the stream (512 = the full workload; fewer = a small case for profiling)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(values, world, device=None):
    """Element-wise maximum of a list of floats over all ranks (the slowest
    rank's times); identity when world == 1."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def whole_job_rate(units_per_rank, world, ms):
    """Units per second of the whole job: every rank's units over the slowest
    rank's time."""
    return world * units_per_rank / (ms / 1e3)


def workload_config(extra=None, windows=WINDOWS):
    cfg = {
        "workload": "accumulated RMAT stream: 2^26 packets as 512 windows of 2^17, "
                    "stats of the summed A after every window (plain per-window launches)",
        "packets": windows * WINDOW,
        "windows": windows,
        "window_packets": WINDOW,
        "generator": "RMAT scale 32 (0.57,0.19,0.19,0.05) + 10% uniform, seeded bijection",
        "l2": "inputs larger than L2 (512 MiB of packets; the accumulated matrix's tables are GiB-sized)",
    }
    if extra:
        cfg.update(extra)
    return cfg


# ----------------------------------------------------------------- CPU legs

def oracle_stream_rate(src, dst, budget_s=None, windows=None):
    """The CPU oracle as it stands, single thread: for each window build A_t,
    A += A_t, and the nine quantities of A; stops after `windows` windows or
    once `budget_s` seconds have passed.  Returns (packets/s, windows, s)."""
    import oracle
    acc = (np.zeros(0, np.uint64), np.zeros(0, np.uint64))
    t0 = time.perf_counter()
    w = 0
    while w < len(src) // WINDOW:
        sl = slice(w * WINDOW, (w + 1) * WINDOW)
        acc = oracle.accumulate(acc, oracle.build_matrix(src[sl], dst[sl]))
        oracle.stats(*acc)
        w += 1
        el = time.perf_counter() - t0
        if windows is not None and w >= windows:
            break
        if budget_s is not None and el >= budget_s:
            break
    el = time.perf_counter() - t0
    return w * WINDOW / el, w, el


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle on this arm's workload and metric, each
    step a bounded sample (the first 16 windows)."""
    if rank != 0:
        return
    import gen.workloads as W
    sample_windows = 16
    src, dst = W.rmat_stream(sample_windows * WINDOW)
    for _ in range(args.warmup):
        oracle_stream_rate(src, dst, windows=sample_windows)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_stream_rate(src, dst, windows=sample_windows)
    el = time.perf_counter() - t0
    value = args.steps * sample_windows * WINDOW / el
    sample = f"first {sample_windows} windows (2^{int(np.log2(sample_windows * WINDOW))} packets) per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic", "config": workload_config({"sample": sample}),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.rows = []
        self.proc = None
        self.gpu = gpu_index
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), [x.strip() for x in line.split(",")]))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.t:
            self.t.join(timeout=2)

    def summary(self, t0, t1):
        rows = [r for t, r in self.rows if t0 <= t <= t1] or [r for _, r in self.rows[-3:]]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if len(r) > 5 + i and r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------- ours

def kernel_traffic():
    """ncu DRAM bytes per launch of the dominant kernel, if the committed
    profile was taken on the current kernel source; else None."""
    if not os.path.exists(PROFILE):
        return None
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        h.update(open(p, "rb").read())
    got_hash = traffic = None
    for line in open(PROFILE):
        if line.startswith("source_sha256:"):
            got_hash = line.split(":", 1)[1].strip()
        if line.startswith("traffic_bytes_per_launch:"):
            traffic = float(line.split(":", 1)[1].strip())
    return traffic if got_hash == h.hexdigest() else None


def run_ours(args, rank, world, local):
    import torch
    import gen.workloads as W
    import paper_2509_03653_b300 as ns

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    NW = args.windows
    N = NW * WINDOW
    # host input (pinned) and its resident device copy
    h_src = torch.empty(N, dtype=torch.int32).pin_memory()
    h_dst = torch.empty(N, dtype=torch.int32).pin_memory()
    seed = W.seed_of(2) + 1000 * rank  # replicas draw independent streams
    W.rmat_stream(N, src=h_src.numpy().view(np.uint32), dst=h_dst.numpy().view(np.uint32), seed=seed)
    d_src = h_src.to(dev)
    d_dst = h_dst.to(dev)

    ctx = ns.Context(local, path="hash", hash_load=args.hash_load)
    A = ns.Matrix(ctx)
    ns.matrix_reserve(A, N)

    # per-window distinct counts for the roofline bytes (bookkeeping only)
    t_build = ns.Matrix(ctx)
    alg_bytes = 0
    for w in range(NW):
        ns.window_build(ctx, d_src[w * WINDOW:(w + 1) * WINDOW], d_dst[w * WINDOW:(w + 1) * WINDOW], t_build)
        st = ns.network_stats(ctx, t_build)
        alg_bytes += 8 * WINDOW + 16 * st["unique_links"] + 16 * (st["unique_sources"] + st["unique_destinations"])
    t_build.free()
    alg_bytes_per_launch = alg_bytes / NW

    stats_rows = torch.zeros(NW, 16, dtype=torch.int64, device=dev)
    cap_stream = torch.cuda.Stream(dev)

    def step(src, dst, ev=None):
        ns.matrix_clear(A)
        for w in range(NW):
            sl = slice(w * WINDOW, (w + 1) * WINDOW)
            if ev is not None:
                ev[w][0].record()
            ns.window_ingest_stats(ctx, A, src[sl], dst[sl], stats_rows[w])
            if ev is not None:
                ev[w][1].record()

    # eager warm-up, then capture one graph per timed step (each with its own
    # timing events around every ingest launch)
    with torch.cuda.stream(cap_stream):
        step(d_src, d_dst)
    torch.cuda.synchronize()
    graphs, events = [], []
    for k in range(args.steps):
        ev = [(torch.cuda.Event(enable_timing=True, external=True),
               torch.cuda.Event(enable_timing=True, external=True)) for _ in range(NW)]
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cap_stream):
            step(d_src, d_dst, ev)
        graphs.append(g)
        events.append(ev)
    g_plain = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_plain, stream=cap_stream):
        step(d_src, d_dst)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    for _ in range(max(args.warmup, 3)):
        g_plain.replay()
    torch.cuda.synchronize()

    # ---- timed region: K steps of the plain graph, inputs resident in HBM
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    cur = torch.cuda.current_stream()
    tw0 = time.time()
    e0.record(cur)
    for _ in range(args.steps):
        g_plain.replay()
    e1.record(cur)
    torch.cuda.synchronize()
    tw1 = time.time()
    barrier()
    ms = e0.elapsed_time(e1)
    clock_summary = clocks.summary(tw0, tw1)
    # ---- the same K steps again from graphs with an event pair around every
    # ingest launch: per-launch kernel time (the event nodes sit between the
    # launches, so this replay is timed separately)
    torch.cuda.synchronize()
    e0.record(cur)
    for g in graphs:
        g.replay()
    e1.record(cur)
    torch.cuda.synchronize()
    ms_instr = e0.elapsed_time(e1)
    launch_ms = [a.elapsed_time(b) for ev in events for a, b in ev]

    # the random-atomic ceiling of the same access pattern: one window's worth
    # of threads, three random 8-byte atomics each, tables as large as A's
    # link table (no hashing, probing or statistics)
    rand_ceiling_us = ns.diag_random_atomics(1 << 28, WINDOW, 5)

    # correctness guard on the last step (cheap invariant, no oracle)
    last = stats_rows[-1].cpu().numpy().view(np.uint64)
    assert int(last[0]) == N, "valid packets != N"

    # ---- end to end: every step copies its packets from pinned host memory
    # (in chunks of 32 windows on a copy stream, overlapped with the ingest of
    # earlier chunks) and reads the statistics rows back; one captured graph
    e2e = None
    if not args.no_e2e:
        h_stats = torch.empty(NW, 16, dtype=torch.int64).pin_memory()
        copy_stream = torch.cuda.Stream(dev)
        CH = 32
        chunks = [(c, min(c + CH, NW)) for c in range(0, NW, CH)]
        ready = [torch.cuda.Event() for _ in chunks]

        def e2e_step():
            copy_stream.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(copy_stream):
                for (a, b_), ev in zip(chunks, ready):
                    sl = slice(a * WINDOW, b_ * WINDOW)
                    d_src[sl].copy_(h_src[sl], non_blocking=True)
                    d_dst[sl].copy_(h_dst[sl], non_blocking=True)
                    ev.record(copy_stream)
            ns.matrix_clear(A)
            for (a, b_), ev in zip(chunks, ready):
                torch.cuda.current_stream().wait_event(ev)
                for w in range(a, b_):
                    sl = slice(w * WINDOW, (w + 1) * WINDOW)
                    ns.window_ingest_stats(ctx, A, d_src[sl], d_dst[sl], stats_rows[w])
            h_stats.copy_(stats_rows, non_blocking=True)
            torch.cuda.current_stream().wait_stream(copy_stream)

        g_e2e = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g_e2e, stream=cap_stream):
            e2e_step()
        for _ in range(2):
            g_e2e.replay()
        torch.cuda.synchronize()
        barrier()
        e2 = torch.cuda.Event(enable_timing=True)
        e3 = torch.cuda.Event(enable_timing=True)
        e2.record(cur)
        for _ in range(args.steps):
            g_e2e.replay()
        e3.record(cur)
        torch.cuda.synchronize()
        barrier()
        assert int(h_stats[-1].numpy().view(np.uint64)[0]) == N, "e2e: valid packets != N"
        e2e = {"ms": e2.elapsed_time(e3), "h2d": 2 * 4 * N, "d2h": NW * 16 * 8}
    clocks.stop()

    # ---- gather over ranks (max time)
    ms, ms_instr, ms_e2e = max_over_ranks([ms, ms_instr, e2e["ms"] if e2e else 0.0], world, dev)
    if e2e:
        e2e["ms"] = ms_e2e
    if rank != 0:
        return

    value = whole_job_rate(args.steps * N, world, ms)
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(peaks_path)) if os.path.exists(peaks_path) else {}
    peak = peaks.get("hbm_gbs", 6400.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    avg_launch_ms = float(np.mean(launch_ms))
    achieved = alg_bytes_per_launch / (avg_launch_ms / 1e3) / 1e9

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": workload_config({"path": "hash (fused window ingest + statistics, one launch per window)", "graph": "per-window launches "
                                   "captured in one CUDA graph per step", "hash_load": args.hash_load,
                                   "table_gib": round(3 * 16 * (1 << math.ceil(math.log2(N / args.hash_load))) / 2**30, 1),
                                   "parallelism": "replicas" if world > 1 else "single GPU"}, windows=NW),
        "roofline": {
            "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": kernel_traffic(), "kernel": "k_insert_packets",
            "alg_bytes_per_launch": alg_bytes_per_launch, "launch_us_avg": avg_launch_ms * 1e3,
            "launch_us_p50": float(np.percentile(launch_ms, 50)) * 1e3,
            "peak_source": f"{peak_src} (hbm_gbs, copy read+write)",
        },
        "roofline_random_access": {
            "bound": "random 8-byte atomics", "kernel": "k_insert_packets",
            "kernel_us": avg_launch_ms * 1e3, "ceiling_us": rand_ceiling_us,
            "frac": rand_ceiling_us / (avg_launch_ms * 1e3),
            "ceiling": "2^17 threads x 3 random atomics into three 2 GiB tables (measured live)",
        },
        "clocks": clock_summary,
        "gpu_launches": args.steps * NW,
        "ms_per_step_instrumented": ms_instr / args.steps,
    }
    if e2e:
        line["e2e"] = {"value": whole_job_rate(args.steps * N, world, e2e["ms"]), "unit": UNIT,
                       "h2d_bytes_per_step": e2e["h2d"], "d2h_bytes_per_step": e2e["d2h"]}
    if not args.no_cpu_baseline:
        rate, wins, el = oracle_stream_rate(h_src.numpy().view(np.uint32), h_dst.numpy().view(np.uint32),
                                            budget_s=args.cpu_budget)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"first {wins} windows of the same stream ({wins * WINDOW} packets, "
                                          f"{el:.1f} s), stats after each window"}
    print(json.dumps(line), flush=True)


def peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(path)) if os.path.exists(path) else {}
    if "hbm_gbs" in peaks:
        return peaks["hbm_gbs"], "measured (hbm_gbs, copy read+write)"
    return 6400.0, "fallback"


def run_oneshot(args, rank, world, local):
    """One build of N packets (default 2^30; src/dst Zipf(1.2) over 2^24
    addresses under a seeded bijection): A plus the nine quantities, with the
    sort path and the hash path on the same resident input."""
    import torch
    import gen.workloads as W
    import paper_2509_03653_b300 as ns

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    N = args.packets
    h_src = torch.empty(N, dtype=torch.int32).pin_memory()
    h_dst = torch.empty(N, dtype=torch.int32).pin_memory()
    tg = time.time()
    W.large_build(N, src=h_src.numpy().view(np.uint32), dst=h_dst.numpy().view(np.uint32))
    gen_s = time.time() - tg
    d_src = h_src.to(dev)
    d_dst = h_dst.to(dev)
    out = torch.zeros(16, dtype=torch.int64, device=dev)
    peak, peak_src = peak_hbm()
    res = {}
    stats_by_path = {}
    for path in args.paths.split(","):
        ctx = ns.Context(local, path=path)
        M = ns.Matrix(ctx)
        for _ in range(max(args.warmup, 3)):
            ns.window_build(ctx, d_src, d_dst, M)
            st = ns.network_stats(ctx, M)
        stats_by_path[path] = st
        ns.trace_enable(ctx, True)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            ns.window_build(ctx, d_src, d_dst, M)
            ns.network_stats_async(ctx, M, out)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        tr = ns.trace_read(ctx)
        ns.trace_enable(ctx, False)
        U, S, D = st["unique_links"], st["unique_sources"], st["unique_destinations"]
        if path == "sort":
            kname = "k_onesweep<u64 key>"
            kbytes = 16 * N  # one digit pass reads and writes every 8-byte key
            # minimal bytes of each sort-path kernel (N < 2^32: the column
            # side sorts one word per link): histogram 8N; 8 digit passes
            # 16N each; link runs 8N + 16U (pos, keys); link counts 16U; row
            # runs 24U + 16S (reads keys and counts, writes the dst words,
            # pos, psum); row stats 16S; column histogram 8U; 4 digit passes
            # 16U each; column runs 8U + 16D; column stats 16D
            path_bytes = 144 * N + 136 * U + 32 * (S + D)
        else:
            kname = "k_insert_packets"
            kbytes = 8 * N + 16 * U + 16 * (S + D)
            path_bytes = kbytes
        alg_bytes = 8 * N + 16 * U + 16 * U + 16 * (S + D)
        kl, ktot, kmax = tr.get(kname, (0, 0.0, 0.0))
        kavg = ktot / kl if kl else float("nan")
        res[path] = {
            "packets_per_s": N / (ms / 1e3), "ms_per_build": ms,
            "path_bytes_frac": path_bytes / (ms / 1e3) / 1e9 / peak,
            "alg_bytes_frac": alg_bytes / (ms / 1e3) / 1e9 / peak,
            "dominant_kernel": kname, "kernel_ms_avg": kavg,
            "kernel_frac": (kbytes / (kavg / 1e3) / 1e9 / peak) if kl else None,
            "kernels_ms": {k: round(v[1] / args.steps, 4) for k, v in sorted(tr.items(), key=lambda kv: -kv[1][1])},
            "launches_per_build": sum(v[0] for v in tr.values()) / args.steps,
        }
        M.free()
        ctx.close()
        torch.cuda.empty_cache()
    same = len({json.dumps(v, sort_keys=True) for v in stats_by_path.values()}) == 1
    best = max(res, key=lambda p: res[p]["packets_per_s"])
    b = res[best]
    kbytes_best = (16 * N) if best == "sort" else None
    line = {
        "metric": METRIC, "value": b["packets_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": b["ms_per_build"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"large one-shot build: {N} packets, src/dst Zipf(1.2) over 2^24 addresses "
                               "under a seeded bijection; A plus the nine quantities",
                   "path": best, "l2": "inputs larger than L2", "generator_s": round(gen_s, 1)},
        "roofline": {"bound": "hbm", "achieved": b["kernel_frac"] * peak if b["kernel_frac"] else None,
                     "peak": peak, "unit": "GB/s", "frac": b["kernel_frac"], "traffic": None,
                     "kernel": b["dominant_kernel"], "peak_source": peak_src},
        "paths": res, "stats": stats_by_path[best], "paths_agree": same,
    }
    print(json.dumps(line), flush=True)


def run_anonymize(args, rank, world, local):
    """Address anonymization (the paper's "IP Address Anonymization" step) of
    N packets (default 2^30, the one-shot build's Zipf(1.2) input): distinct
    addresses of both columns, a random permutation drawn from counter-based
    random keys, and the gather that relabels every packet."""
    import torch
    import gen
    import gen.workloads as W
    import paper_2509_03653_b300 as ns

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    N = args.packets
    h_src = torch.empty(N, dtype=torch.int32).pin_memory()
    h_dst = torch.empty(N, dtype=torch.int32).pin_memory()
    tg = time.time()
    W.large_build(N, src=h_src.numpy().view(np.uint32), dst=h_dst.numpy().view(np.uint32))
    h_rand = torch.empty(2 * N, dtype=torch.int64).pin_memory()
    gen.random_u64(2 * N, W.seed_of(3), 9, out=h_rand.numpy().view(np.uint64))
    gen_s = time.time() - tg
    d_src, d_dst, d_rand = h_src.to(dev), h_dst.to(dev), h_rand.to(dev)
    o_src = torch.empty_like(d_src)
    o_dst = torch.empty_like(d_dst)
    ctx = ns.Context(local)
    for _ in range(max(args.warmup, 3)):
        _, _, nu = ns.anonymize(ctx, d_src, d_dst, d_rand, o_src, o_dst)
    ns.trace_enable(ctx, True)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        ns.anonymize(ctx, d_src, d_dst, d_rand, o_src, o_dst)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    tr = ns.trace_read(ctx)
    ns.trace_enable(ctx, False)
    peak, peak_src = peak_hbm()
    # minimal bytes: both columns read into the address set (8N); the
    # distinct addresses compacted, sorted (histogram 4 nu + four digit
    # passes 32 nu) and widened (12 nu); the permutation's sort of nu
    # (key, position) pairs (8 digit passes x 32 nu); the gather (8N read +
    # 8N written).  The set's table (mostly L2-resident) is not counted.
    path_bytes = 8 * N + 4 * nu + 32 * nu + 12 * nu + 256 * nu + 16 * N
    kname = "k_set_insert"
    kl, ktot, _ = tr.get(kname, (0, 0.0, 0.0))
    kavg = ktot / kl if kl else float("nan")
    line = {
        "metric": "packets/s anonymized (distinct addresses, random permutation, gather)", "value": N / (ms / 1e3),
        "unit": "packets/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"address anonymization of {N} packets, src/dst Zipf(1.2) over 2^24 addresses "
                               "under a seeded bijection; counter-based random keys",
                   "distinct_addresses": nu, "l2": "inputs larger than L2", "generator_s": round(gen_s, 1)},
        "roofline": {"bound": "hbm", "achieved": path_bytes / (ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": path_bytes / (ms / 1e3) / 1e9 / peak, "traffic": None,
                     "kernel": "whole step (minimal bytes of its passes)", "peak_source": peak_src,
                     "set_insert_frac": (8 * N / (kavg / 1e3) / 1e9 / peak) if kl else None},
        "kernels_ms": {k: round(v[1] / args.steps, 4) for k, v in sorted(tr.items(), key=lambda kv: -kv[1][1])},
    }
    print(json.dumps(line), flush=True)


def run_slide(args, rank, world, local):
    """The stream workload's windows (512 x 2^17 RMAT packets) through a
    slider over the last K windows: every window's own quantities and those
    of the sum of the last K windows, after each window."""
    import torch
    import gen.workloads as W
    import paper_2509_03653_b300 as ns

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    NW, K = args.windows, args.slide_windows
    N = NW * WINDOW
    h_src = torch.empty(N, dtype=torch.int32).pin_memory()
    h_dst = torch.empty(N, dtype=torch.int32).pin_memory()
    W.rmat_stream(N, src=h_src.numpy().view(np.uint32), dst=h_dst.numpy().view(np.uint32))
    d_src, d_dst = h_src.to(dev), h_dst.to(dev)
    # RMAT windows hardly repeat a source or destination: no per-CTA staging
    ctx = ns.Context(local, path="hash", cta_cache="off")
    out_w = torch.zeros(NW, 16, dtype=torch.int64, device=dev)
    out_s = torch.zeros(NW, 16, dtype=torch.int64, device=dev)

    def step(sl):
        for w in range(NW):
            a = w * WINDOW
            ns.slider_push(ctx, sl, d_src[a:a + WINDOW], d_dst[a:a + WINDOW], out_w[w], out_s[w])

    sl = ns.Slider(ctx, K)
    for _ in range(max(args.warmup, 3)):
        step(sl)  # also grows the sliding sum's tables to their final size
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step(sl)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    ns.trace_enable(ctx, True)  # one more step, traced, for the kernel breakdown
    step(sl)
    torch.cuda.synchronize()
    tr = ns.trace_read(ctx)
    ns.trace_enable(ctx, False)
    line = {
        "metric": "packets/s with per-window and sliding-window (last K windows) statistics after every window",
        "value": N / (ms / 1e3), "unit": "packets/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": f"sliding windows: {NW} windows of 2^17 RMAT packets (the stream workload), "
                               f"quantities of each window and of the sum of the last {K}",
                   "windows": NW, "slide_windows": K, "cta_cache": "off", "l2": "inputs larger than L2"},
        "ms_per_window": ms / NW,
        "kernels_ms_traced_step": {k: round(v[1], 4) for k, v in sorted(tr.items(), key=lambda kv: -kv[1][1])},
        "launches_per_step": sum(v[0] for v in tr.values()),
    }
    print(json.dumps(line), flush=True)


def run_batched(args, rank, world, local):
    """Workload 4: 8192 windows, sizes log-uniform in [2^10, 2^20], per-window
    Zipf exponent in [0.8, 1.4] over 2^20 addresses.  Per-window quantities
    plus the running aggregate, as (a) one autotuned batched launch sequence
    and (b) plain per-window launches (build, statistics, accumulate), each
    captured in a CUDA graph and replayed."""
    import torch
    import gen.workloads as W
    import paper_2509_03653_b300 as ns

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    Wn = args.batch_windows
    sizes, svals = W.batched_plan(Wn)
    total = int(sizes.sum())
    off = np.zeros(Wn + 1, np.uint64)
    off[1:] = np.cumsum(sizes)
    h_src = torch.empty(total, dtype=torch.int32).pin_memory()
    h_dst = torch.empty(total, dtype=torch.int32).pin_memory()
    hs, hd = h_src.numpy().view(np.uint32), h_dst.numpy().view(np.uint32)
    tg = time.time()
    for w in range(Wn):
        a, b = int(off[w]), int(off[w + 1])
        W.batched_window(w, b - a, float(svals[w]), src=hs[a:b], dst=hd[a:b])
    gen_s = time.time() - tg
    d_src, d_dst = h_src.to(dev), h_dst.to(dev)

    ctx = ns.Context(local, path="hash", hbm_budget_bytes=96 << 30, tuner_cache=args.tuner_cache)
    acc = ns.Matrix(ctx)
    ns.matrix_reserve_ex(acc, total, 1 << 21)
    batch = ns.Batch(ctx, Wn, total)
    tt = time.time()
    params = ns.batch_tune(ctx, batch, d_src, d_dst, off) if not args.tuner_cache else batch.params
    tune_s = time.time() - tt
    out_b = torch.zeros(Wn * 9, dtype=torch.int64, device=dev)
    out_p = torch.zeros(Wn * 9, dtype=torch.int64, device=dev)
    At = ns.Matrix(ctx)
    cap = torch.cuda.Stream(dev)

    def batched():
        ns.matrix_clear(acc)
        ns.batch_run(ctx, batch, d_src, d_dst, off, out_b, acc)

    def plain():
        ns.matrix_clear(acc)
        for w in range(Wn):
            a, b = int(off[w]), int(off[w + 1])
            ns.window_build(ctx, d_src[a:b], d_dst[a:b], At)
            ns.network_stats_async(ctx, At, out_p[w * 9:(w + 1) * 9])
            ns.accumulate(ctx, acc, At)

    res = {}
    for name, fn in (("plain", plain), ("batched", batched)):
        with torch.cuda.stream(cap):
            fn()  # eager warm-up: sizes the per-window matrix outside capture
        torch.cuda.synchronize()
        stats_eager = ns.network_stats(ctx, acc)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cap):
            fn()
        for _ in range(max(args.warmup, 3)):
            g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        res[name] = {"ms_per_step": ms, "packets_per_s": total / (ms / 1e3),
                     "aggregate": ns.network_stats(ctx, acc), "aggregate_eager": stats_eager}
        del g
    same_rows = bool(torch.equal(out_b, out_p))
    same_acc = res["plain"]["aggregate"] == res["batched"]["aggregate"]
    # per-kernel times of one traced (eager) batched run
    ns.trace_enable(ctx, True)
    batched()
    tr = ns.trace_read(ctx)
    ns.trace_enable(ctx, False)
    rows = out_b.cpu().numpy().view(np.uint64).reshape(Wn, 9)
    sumU, sumS, sumD = int(rows[:, 1].sum()), int(rows[:, 2].sum()), int(rows[:, 3].sum())
    kl, ktot, _ = tr.get("k_batch_insert", (0, 0.0, 0.0))
    kbytes = 8 * total + 16 * sumU + 16 * (sumS + sumD)
    peak, peak_src = peak_hbm()
    frac = (kbytes / (ktot / kl / 1e3) / 1e9 / peak) if kl else None
    b, p_ = res["batched"], res["plain"]
    line = {
        "metric": METRIC, "value": b["packets_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": b["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"batched: {Wn} windows, sizes log-uniform in [2^10, 2^20] ({total} packets), "
                               "per-window Zipf exponent U[0.8,1.4] over 2^20 addresses; per-window stats plus "
                               "running aggregate", "generator_s": round(gen_s, 1), "tune_s": round(tune_s, 1),
                   "batch_params": params, "l2": "inputs larger than L2"},
        "batched_vs_plain": b["packets_per_s"] / p_["packets_per_s"],
        "plain": {"packets_per_s": p_["packets_per_s"], "ms_per_step": p_["ms_per_step"],
                  "launches_per_step": 3 * Wn},
        "results_agree": same_rows and same_acc,
        "roofline": {"bound": "hbm", "achieved": frac * peak if frac else None, "peak": peak, "unit": "GB/s",
                     "frac": frac, "traffic": None, "kernel": "k_batch_insert", "peak_source": peak_src},
        "kernels_ms": {k: round(v[1], 3) for k, v in sorted(tr.items(), key=lambda kv: -kv[1][1])},
        "aggregate": b["aggregate"],
    }
    print(json.dumps(line), flush=True)


def run_serve(args, rank, world, local):
    """Workload 5: windows of log-uniform size in [2^12, 2^22] packets (RMAT
    scale 32 + 10% uniform) arrive from host memory.  Phase 1 measures the
    service's capacity with every window submitted at once (closed loop);
    phase 2 submits a fresh set as a Poisson process at 80% of that rate.
    Latency is the library's submit -> both statistics records on the host."""
    import threading as th
    import torch
    import gen.workloads as W
    import paper_2509_03653_b300 as ns

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    Wn = args.serve_windows
    sizes, _ = W.serving_plan(2 * Wn, 1.0)
    wins = []
    for w in range(2 * Wn):
        s, d = W.serving_window(w, int(sizes[w]))
        wins.append((torch.from_numpy(s.view(np.int32)).pin_memory(), torch.from_numpy(d.view(np.int32)).pin_memory()))
    phase = [wins[:Wn], wins[Wn:]]
    pk = [int(sizes[:Wn].sum()), int(sizes[Wn:].sum())]

    # one service for both phases; RMAT windows hardly repeat a source or
    # destination, so no per-CTA staging (cta_cache "off", --serve-cache)
    ctx = ns.Context(local, path="hash", max_slots=8, hbm_budget_bytes=64 << 30, cta_cache=args.serve_cache)
    acc = ns.Matrix(ctx)
    ns.matrix_reserve(acc, max(pk))
    srv = ns.Server(ctx, acc)

    def restart():  # an empty aggregate between phases (the service is idle)
        srv.clear()

    # every slot sized for the largest window, then a short warm-up
    srv.reserve(int(sizes.max()))
    for t in [ns.stream_submit(srv, s, d, i) for i, (s, d) in enumerate(wins[:16])]:
        ns.stream_wait(srv, t)
    restart()

    # phase 1: closed loop -> capacity
    t0 = time.perf_counter()
    pending, i = [], 0
    while i < Wn or pending:  # keep the queue full; wait in ticket order
        while i < Wn:
            try:
                pending.append(ns.stream_submit(srv, phase[0][i][0], phase[0][i][1], i))
                i += 1
            except ns.NsError as e:
                if e.name != "NS_ERR_BUSY":
                    raise
                break
        if pending:
            ns.stream_wait(srv, pending.pop(0))
    cap_s = time.perf_counter() - t0
    cap_wps = Wn / cap_s
    cap_pps = pk[0] / cap_s
    restart()

    # phase 2: Poisson arrivals at 80% of capacity
    rate = 0.8 * cap_wps
    _, arrivals = W.serving_plan(Wn, rate)
    tickets = [None] * Wn
    busy = [0]

    def submitter():
        start = time.perf_counter()
        for i, (s, d) in enumerate(phase[1]):
            while True:
                dt = start + float(arrivals[i]) - time.perf_counter()
                if dt <= 0:
                    break
                time.sleep(min(dt, 0.0005))
            while True:
                try:
                    tickets[i] = ns.stream_submit(srv, s, d, i)
                    break
                except ns.NsError as e:
                    if e.name != "NS_ERR_BUSY":
                        raise
                    busy[0] += 1
                    time.sleep(0.0001)

    thr = th.Thread(target=submitter)
    thr.start()
    lat, first, last = [], None, None
    for i in range(Wn):
        while tickets[i] is None:
            time.sleep(0.0001)
        _, _, tm = ns.stream_wait(srv, tickets[i])
        lat.append((tm["complete_us"] - tm["submit_us"]) / 1e3)
        first = tm["submit_us"] if first is None else min(first, tm["submit_us"])
        last = tm["complete_us"] if last is None else max(last, tm["complete_us"])
    thr.join()
    srv.close()
    span_s = (last - first) / 1e6
    lat = np.array(lat)
    line = {
        "metric": METRIC, "value": pk[1] / span_s, "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 1,
        "ms_per_step": span_s * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"streaming serving: {Wn} windows per phase, sizes log-uniform in [2^12, 2^22], "
                               "RMAT scale 32 + 10% uniform from pinned host memory, Poisson arrivals at 80% of "
                               "measured capacity, 64 GiB HBM admission budget, 8 slots",
                   "packets": pk[1], "cta_cache": args.serve_cache},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "mean": float(lat.mean()), "max": float(lat.max())},
        "capacity": {"windows_per_s": cap_wps, "packets_per_s": cap_pps},
        "offered_windows_per_s": rate, "busy_retries": busy[0],
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "oneshot":
        if rank == 0:
            run_oneshot(args, rank, world, local)
        return
    if args.workload == "batched":
        if rank == 0:
            run_batched(args, rank, world, local)
        return
    if args.workload == "serve":
        if rank == 0:
            run_serve(args, rank, world, local)
        return
    if args.workload == "anonymize":
        if rank == 0:
            run_anonymize(args, rank, world, local)
        return
    if args.workload == "slide":
        if rank == 0:
            run_slide(args, rank, world, local)
        return
    run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
