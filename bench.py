#!/usr/bin/env python3
"""Benchmark of the traffic-matrix hot path on one B300 (or N replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload headline|oneshot|stream|batched|serve|anonymize|slide]

Default ("headline"): the large one-shot build -- 2^30 packets (8 GiB of
uint32 src/dst), src and dst independently Zipf(1.2) over 2^24 addresses
under a seeded 32-bit bijection -- turned into A's sorted nonzero list and
its nine Table 2 quantities.  One step = one ns_window_build (sort path) plus
the statistics record, inputs resident in HBM (8 GiB, far larger than L2).
`value` is packets/s over K timed steps (CUDA events); the hash path is timed
beside it on the same input.  `e2e` times ns_window_build_host: the host
columns (pinned) copied in, the build, the nine quantities read back.
`cpu_baseline` times the oracle on a sample of the same input, single-threaded
(O1) and on every host core (O2).

The same JSON line carries sub-records, each with its own clock samples:
  stream            2^26 RMAT packets as 512 windows of 2^17, running
                    quantities after every window (plain per-window launches)
  batched_vs_plain  8192 windows of log-uniform size in [2^10, 2^20], one
                    autotuned batched launch sequence vs per-window launches
  serve             windows of log-uniform size in [2^12, 2^22] arriving at
                    80% of capacity: p50/p99 window-to-stats latency, and the
                    same windows through a plain per-window loop

--workload picks one of them alone (for profiling), printing its own line.
Under torchrun (N > 1) every rank builds its own copy of the headline
workload on its own GPU (replicas, no data-path collective) and rank 0
reports the whole-job rate over the slowest rank; the sub-records run at
N = 1 only.
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
CSRC = os.path.join(ROOT, "paper_2509_03653_b300", "csrc")
HEADLINE_WORKLOAD = ("large one-shot build: 2^30 packets, src/dst Zipf(1.2) over 2^24 addresses under a "
                     "seeded bijection; A's sorted nonzero list plus the nine quantities")
CPU_SAMPLE = 1 << 26  # packets of the headline input the oracle is timed on


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="headline",
                    choices=["headline", "oneshot", "stream", "batched", "serve", "anonymize", "slide"],
                    help="headline: the one-shot 2^30 build with the stream, batched and serve sub-records "
                         "(default); the others run one workload alone")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-sub", action="store_true", help="headline without the sub-records")
    ap.add_argument("--packets", type=int, default=1 << 30, help="oneshot / anonymize: packets in the input")
    ap.add_argument("--paths", default="sort,hash", help="oneshot: aggregation paths to run (first = value)")
    ap.add_argument("--sort-split", default="auto", choices=["auto", "on", "off"],
                    help="headline/oneshot: the sort path's hot-key split")
    ap.add_argument("--sort-digits", default="auto", choices=["auto", "8", "wide"],
                    help="oneshot/headline: the sort path's digit plan (auto: the path tuner's choice)")
    ap.add_argument("--no-tune", action="store_true",
                    help="headline/oneshot: skip ns_path_tune before timing the sort path")
    ap.add_argument("--windows", type=int, default=WINDOWS, help="stream: windows (512 = the full workload)")
    ap.add_argument("--hash-load", type=float, default=0.25,
                    help="stream: load bound of the accumulated matrix's hash tables")
    ap.add_argument("--batch-windows", type=int, default=8192, help="batched: number of windows")
    ap.add_argument("--tuner-cache", default=None, help="batched: autotuner cache file (default: tune now)")
    ap.add_argument("--serve-windows", type=int, default=448, help="serve: windows per phase")
    ap.add_argument("--serve-cache", default="off", choices=["auto", "on", "off"],
                    help="serve: per-CTA staging of the service's context (RMAT windows: off)")
    ap.add_argument("--slide-windows", type=int, default=8, help="slide: windows in the sliding sum (K)")
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


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(path)) if os.path.exists(path) else {}
    if "hbm_gbs" in peaks:
        return float(peaks["hbm_gbs"]), "measured (hbm_gbs, copy read+write)"
    return 6400.0, "fallback"


def host_cores():
    try:
        aff = len(os.sched_getaffinity(0))
    except AttributeError:
        aff = os.cpu_count()
    return {"nproc": aff, "cpu_count": os.cpu_count()}


def sources_sha(names):
    h = hashlib.sha256()
    for n in names:
        h.update(open(os.path.join(CSRC, n), "rb").read())
    return h.hexdigest()


def profile_traffic(profile, names):
    """DRAM bytes per launch from a committed ncu summary under profiles/
    (its `traffic_bytes_per_launch` and the `units_per_launch` it was taken
    on), if the summary was taken on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", profile)
    if not os.path.exists(path):
        return None
    got = {}
    for line in open(path):
        for key in ("source_sha256", "traffic_bytes_per_launch", "units_per_launch"):
            if line.startswith(key + ":"):
                got[key] = line.split(":", 1)[1].strip()
    if got.get("source_sha256") != sources_sha(names) or "traffic_bytes_per_launch" not in got:
        return None
    return {"bytes": float(got["traffic_bytes_per_launch"]),
            "units": float(got["units_per_launch"]) if "units_per_launch" in got else None}


def profile_traffic_keyed(profile, names, key):
    """DRAM bytes per unit for one launch configuration from a committed ncu
    summary under profiles/ (its `traffic_per_packet[<key>]` line), if the
    summary was taken on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", profile)
    if not os.path.exists(path):
        return None
    sha, val = None, None
    for line in open(path):
        if line.startswith("source_sha256:"):
            sha = line.split(":", 1)[1].strip()
        if line.startswith(f"traffic_per_packet[{key}]:"):
            val = float(line.split(":", 1)[1])
    return val if sha == sources_sha(names) else None


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
        time.sleep(0.3)

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
        """Median SM clock, max clock and the throttle reasons seen in [t0, t1]
        (the last samples before t1 if the region was shorter than a sample)."""
        rows = [r for t, r in self.rows if t0 <= t <= t1]
        if not rows:
            rows = [r for t, r in self.rows if t <= t1 + 0.2][-2:]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if len(r) > 5 + i and r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def timed(fn, steps, stream=None):
    """CUDA-event time (ms, total) of `steps` calls of fn on the current
    stream, synchronized on both sides; also the wall-clock span."""
    import torch
    cur = stream or torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t0 = time.time()
    e0.record(cur)
    for _ in range(steps):
        fn()
    e1.record(cur)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), t0, time.time()


def kernels_ms(tr, per=1):
    return {k: round(v[1] / per, 4) for k, v in sorted(tr.items(), key=lambda kv: -kv[1][1])}


# ------------------------------------------------------------ CPU baselines

def oracle_rates(src, dst, n):
    """The oracle as it stands on the first n packets: build + nine
    quantities, once single-threaded (O1) and once on every host core (O2).
    Returns ({O1}, {O2})."""
    import oracle
    s, d = src[:n], dst[:n]
    t0 = time.perf_counter()
    k, c = oracle.build_matrix(s, d)
    st1 = oracle.stats(k, c)
    t1 = time.perf_counter() - t0
    del k, c
    t0 = time.perf_counter()
    k, c = oracle.build_matrix_parallel(s, d)
    st2 = oracle.stats_parallel(k, c)
    t2 = time.perf_counter() - t0
    assert st1 == st2, "O1 and O2 disagree"
    threads = oracle.hardware_threads()
    return ({"value": n / t1, "unit": UNIT, "cores": 1, "seconds": round(t1, 2)},
            {"value": n / t2, "unit": UNIT, "cores": threads, "seconds": round(t2, 2)})


def run_reference(args, rank, world):
    """Reference arm: the oracle, on every host core (O2), on the headline
    workload's metric and unit; each step builds A and its quantities for a
    bounded sample (the first 2^26 packets) of the headline input."""
    if rank != 0:
        return
    import gen.workloads as W
    import oracle
    src, dst = W.large_build(CPU_SAMPLE)
    for _ in range(args.warmup):
        oracle.stats_parallel(*oracle.build_matrix_parallel(src, dst))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.stats_parallel(*oracle.build_matrix_parallel(src, dst))
    el = time.perf_counter() - t0
    value = args.steps * CPU_SAMPLE / el
    threads = oracle.hardware_threads()
    sample = (f"first 2^{int(math.log2(CPU_SAMPLE))} packets of the headline input per step (A's nonzero list "
              f"and the nine quantities), oracle on all {threads} host threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic", "config": headline_config(),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                         **host_cores()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------- headline (workload 3)

def headline_config():
    return {"workload": HEADLINE_WORKLOAD, "packets": 1 << 30, "window_packets": 1 << 30,
            "generator": "Zipf(1.2) over 2^24 ranks per column, 4-round Feistel bijection into 32 bits",
            "l2": "inputs larger than L2 (8 GiB of packets)", "parallelism": "single GPU"}


def sort_path_bytes(N, U, S, D, info, passes=8):
    """Minimal bytes of the sort path's passes, kernel by kernel (N < 2^32:
    the column side sorts one u64 word per link).  Without a hot-key split:
    histogram 8N; `passes` digit passes 16N each (eight with 8-bit digits,
    seven with the wide plan); link runs 8N + 16U; link
    counts 16U; row runs 24U + 16S; row statistics 16S; column histogram 8U;
    four column passes 16U each; column runs 8U + 16D; column statistics
    16D.  With the split (C cold packets, H hot keys): the split reads the
    packets and writes the cold keys (8N + 8C); the histogram, digit passes
    and link runs see the C cold keys (8C + 128C + 8C + 16 U_C); the merge
    reads the cold runs and writes the merged list (16 U_C + 16U).  With the
    column side's hot-destination split (W cold column words): it reads the
    U words and writes the cold ones (8U + 8W); the column histogram,
    passes and runs see the W cold words (8W + 64W + 8W); the cold
    destinations' runs and statistics are bounded by 32D."""
    rows = 24 * U + 16 * S + 16 * S
    if "cold_words" in info:
        W = info["cold_words"]
        cols = 8 * U + 8 * W + 8 * W + 64 * W + 8 * W + 32 * D
    else:
        cols = 8 * U + 64 * U + 8 * U + 16 * D + 16 * D
    dp = 16 * passes
    if "cold_packets" not in info:
        return (16 + dp) * N + 32 * U + rows + cols
    C = info["cold_packets"]
    UC = U - info.get("hot_keys", 0)
    return 8 * N + 8 * C + (16 + dp) * C + 16 * UC + 16 * UC + 16 * U + rows + cols


def c3_run(args, rank, world, local, clocks, N):
    """One build of N packets of workload 3, each path in args.paths timed on
    the same resident input; e2e through ns_window_build_host."""
    import torch
    import gen.workloads as W
    import paper_2509_03653_b300 as ns

    dev = torch.device("cuda", local)
    h_src = torch.empty(N, dtype=torch.int32).pin_memory()
    h_dst = torch.empty(N, dtype=torch.int32).pin_memory()
    tg = time.time()
    W.large_build(N, src=h_src.numpy().view(np.uint32), dst=h_dst.numpy().view(np.uint32))
    gen_s = time.time() - tg
    d_src = h_src.to(dev)
    d_dst = h_dst.to(dev)
    out = torch.zeros(16, dtype=torch.int64, device=dev)
    peak, peak_src = peak_hbm()
    res, stats_by_path = {}, {}
    tuned = None
    tuned_file = None
    for path in args.paths.split(","):
        tuner_file = None
        if path == "sort" and not args.no_tune:
            import tempfile
            tuner_file = os.path.join(tempfile.mkdtemp(prefix="ns_tune_"), "tuner.json")
        ctx = ns.Context(local, path=path, sort_split=args.sort_split, tuner_cache=tuner_file,
                         sort_digits=args.sort_digits)
        if tuner_file:
            # the path tuner on this input: the timed builds below take its
            # split and tile choices for this size
            tt = time.time()
            ns.path_tune(ctx, d_src, d_dst)
            entries = json.load(open(tuner_file))
            tuned = {"seconds": round(time.time() - tt, 1), **{k.split("|", 1)[1]: json.loads(v) if isinstance(v, str)
                                                               else v for k, v in entries.items()}}
            tuned_file = tuner_file
        M = ns.Matrix(ctx)
        for _ in range(max(args.warmup, 3)):
            ns.window_build(ctx, d_src, d_dst, M)
        st = ns.network_stats(ctx, M)
        stats_by_path[path] = st
        steps = args.steps if path == args.paths.split(",")[0] else max(1, min(args.steps, 5))

        def step():
            ns.window_build(ctx, d_src, d_dst, M)
            ns.network_stats_async(ctx, M, out)

        barrier(world)
        ms, t0, t1 = timed(step, steps)
        barrier(world)
        ms = ms / steps
        # one more build, traced: per-kernel launch times (events on the
        # launching stream)
        ns.trace_enable(ctx, True)
        step()
        torch.cuda.synchronize()
        tr = ns.trace_read(ctx)
        ns.trace_enable(ctx, False)
        info = {}
        passes = 8
        if path == "sort":
            variant = ns.sort_resolve(ctx, N)
            passes = 7 if variant["digits"] == "wide" else 8
            info["sort_variant"] = {"tile": variant["tile"], "digits": variant["digits"], "digit_passes": passes}
            si = ns.sort_split_info(ctx)
            if si["used"]:
                info.update(hot_keys=si["hot_keys"], cold_packets=si["cold_packets"])
            ci = ns.column_split_info(ctx)
            if ci["used"]:
                info.update(hot_destinations=ci["hot_destinations"], cold_words=ci["cold_words"])
        U, S, D = st["unique_links"], st["unique_sources"], st["unique_destinations"]
        alg_bytes = 8 * N + 32 * U + 16 * (S + D)
        if path == "sort":
            kname = "k_onesweep<u64 key>"
            keys = info.get("cold_packets", N)
            kbytes = 16 * keys  # one digit pass reads and writes every 8-byte key
            path_bytes = sort_path_bytes(N, U, S, D, info, passes)
            traffic = profile_traffic("k_onesweep.oneshot_zipf_2p26.md", ["ns_sort.cu", "ns_common.cuh"])
        else:
            kname = "k_insert_packets"
            kbytes = 8 * N + 16 * U + 16 * (S + D)
            path_bytes = kbytes
            traffic = None
        kl, ktot, _ = tr.get(kname, (0, 0.0, 0.0))
        kavg = ktot / kl if kl else float("nan")
        per_launch_traffic = None
        if traffic and path == "sort":
            units = traffic["units"] or (1 << 26)
            per_launch_traffic = traffic["bytes"] * keys / units  # traffic grows with the keys a pass moves
        res[path] = {
            "packets_per_s": world * N / (ms / 1e3), "ms_per_build": ms, "steps": steps,
            "clocks": clocks.summary(t0, t1),
            "path_bytes_frac": path_bytes / (ms / 1e3) / 1e9 / peak,
            "alg_bytes_frac": alg_bytes / (ms / 1e3) / 1e9 / peak,
            # the minimal passes of the plain sort path (no split, eight
            # 8-bit digit passes) over the measured build time: the bandwidth a
            # build without the splits would need to match it
            "plain_sort_bytes_frac": (sort_path_bytes(N, U, S, D, {}) / (ms / 1e3) / 1e9 / peak
                                      if path == "sort" else None),
            "dominant_kernel": kname, "kernel_ms_avg": kavg, "kernel_launches": kl,
            "kernel_alg_bytes_per_launch": kbytes,
            "kernel_frac": (kbytes / (kavg / 1e3) / 1e9 / peak) if kl else None,
            "kernel_traffic_per_launch": per_launch_traffic,
            "kernels_ms": kernels_ms(tr),
            "launches_per_build": sum(v[0] for v in tr.values()),
            "build_info": info,
        }
        M.free()
        ctx.close()
        torch.cuda.empty_cache()
    same = len({json.dumps(v, sort_keys=True) for v in stats_by_path.values()}) == 1
    first = args.paths.split(",")[0]
    e2e = None
    if not args.no_e2e:
        # the variant the timed builds took (the tuner's record for this size)
        ctx = ns.Context(local, path=first, sort_split=args.sort_split,
                         tuner_cache=tuned_file if first == "sort" else None, sort_digits=args.sort_digits)
        M = ns.Matrix(ctx)
        ns.window_build_host(ctx, h_src, h_dst, M)  # sizes the staging buffers
        steps = max(1, min(args.steps, 5))
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            got = ns.window_build_host(ctx, h_src, h_dst, M)
        el = time.perf_counter() - t0
        (el,) = max_over_ranks([el], world, dev)
        assert got == stats_by_path[first], "e2e statistics differ"
        e2e = {"value": world * steps * N / el, "unit": UNIT, "h2d_bytes_per_step": 8 * N,
               "d2h_bytes_per_step": 72, "steps": steps,
               "call": "ns_window_build_host (pinned host columns in, nine quantities out)"}
        M.free()
        ctx.close()
        torch.cuda.empty_cache()
    return {"res": res, "stats": stats_by_path[first], "paths_agree": same, "gen_s": gen_s, "e2e": e2e, "tuned": tuned,
            "h_src": h_src, "h_dst": h_dst, "peak": peak, "peak_src": peak_src}


def run_headline(args, rank, world, local, oneshot_only=False):
    import torch
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    clocks = ClockSampler(local)
    clocks.start()
    N = args.packets
    r = c3_run(args, rank, world, local, clocks, N)
    res = r["res"]
    first = args.paths.split(",")[0]
    b = res[first]
    (ms,) = max_over_ranks([b["ms_per_build"]], world, dev)
    subs = {}
    if world == 1 and not oneshot_only and not args.no_sub:
        subs["stream"] = c2_record(args, local, clocks)
        torch.cuda.empty_cache()
        subs["batched_vs_plain"] = c4_record(args, local, clocks)
        torch.cuda.empty_cache()
        subs["serve"] = c5_record(args, local, clocks)
    clocks.stop()
    if rank != 0:
        return
    peak = r["peak"]
    kfrac = b["kernel_frac"]
    line = {
        "metric": METRIC, "value": whole_job_rate(N, world, ms), "unit": UNIT, "n_gpus": world, "steps": b["steps"],
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": headline_config() if N == 1 << 30 else dict(headline_config(), packets=N, window_packets=N,
                                                              workload=f"one-shot build of {N} packets"),
        "roofline": {
            "bound": "hbm", "achieved": kfrac * peak if kfrac else None, "peak": peak, "unit": "GB/s",
            "frac": kfrac, "traffic": b["kernel_traffic_per_launch"], "kernel": b["dominant_kernel"],
            "alg_bytes_per_launch": b["kernel_alg_bytes_per_launch"], "launch_ms_avg": b["kernel_ms_avg"],
            "launches_per_build": b["kernel_launches"], "peak_source": r["peak_src"],
            "path_bytes_frac": b["path_bytes_frac"], "alg_bytes_frac": b["alg_bytes_frac"],
            "plain_sort_bytes_frac": b.get("plain_sort_bytes_frac"),
        },
        "clocks": b["clocks"],
        "gpu_launches": b["launches_per_build"] * b["steps"],
        "path": first, "paths": res, "paths_agree": r["paths_agree"], "stats": r["stats"], "path_tuner": r["tuned"],
        "generator_s": round(r["gen_s"], 1),
    }
    if r["e2e"]:
        line["e2e"] = r["e2e"]
    if not args.no_cpu_baseline and rank == 0:
        n = min(CPU_SAMPLE, N)
        o1, o2 = oracle_rates(r["h_src"].numpy().view(np.uint32), r["h_dst"].numpy().view(np.uint32), n)
        line["cpu_baseline"] = {
            "value": o2["value"], "unit": UNIT, "cores": o2["cores"], "kind": "oracle",
            "sample": f"first 2^{int(math.log2(n))} packets of the same input: A's nonzero list and the nine "
                      "quantities; value = all host cores (O2), o1 = one core",
            "o1": o1, "o2": o2, **host_cores()}
    line.update(subs)
    print(json.dumps(line), flush=True)


# ----------------------------------------------------- stream (workload 2)

def c2_record(args, local, clocks, steps=None, windows=None):
    """Workload 2: one ns_window_ingest_stats launch per window (build +
    accumulate + the running quantities), the 512 launches of a step captured
    in one CUDA graph.  Also the per-launch kernel time, the random-atomic
    ceiling it is bound by, and e2e with the packets copied in every step."""
    import torch
    import gen.workloads as W
    import paper_2509_03653_b300 as ns

    dev = torch.device("cuda", local)
    steps = steps or min(args.steps, 20)
    NW = windows or args.windows
    N = NW * WINDOW
    h_src = torch.empty(N, dtype=torch.int32).pin_memory()
    h_dst = torch.empty(N, dtype=torch.int32).pin_memory()
    W.rmat_stream(N, src=h_src.numpy().view(np.uint32), dst=h_dst.numpy().view(np.uint32))
    d_src, d_dst = h_src.to(dev), h_dst.to(dev)
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
    alg_per_launch = alg_bytes / NW
    rows = torch.zeros(NW, 16, dtype=torch.int64, device=dev)
    cap = torch.cuda.Stream(dev)

    def step(ev=None):
        ns.matrix_clear(A)
        for w in range(NW):
            sl = slice(w * WINDOW, (w + 1) * WINDOW)
            if ev is not None:
                ev[w][0].record()
            ns.window_ingest_stats(ctx, A, d_src[sl], d_dst[sl], rows[w])
            if ev is not None:
                ev[w][1].record()

    with torch.cuda.stream(cap):
        step()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=cap):
        step()
    ev = [(torch.cuda.Event(enable_timing=True, external=True),
           torch.cuda.Event(enable_timing=True, external=True)) for _ in range(NW)]
    g_ev = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_ev, stream=cap):
        step(ev)
    for _ in range(max(args.warmup, 3)):
        g.replay()
    ms, t0, t1 = timed(g.replay, steps)
    clk = clocks.summary(t0, t1)
    # per-launch kernel time from a separately replayed graph with an event
    # pair around every launch (the event nodes break the launches'
    # programmatic overlap, so this replay is timed apart)
    g_ev.replay()
    torch.cuda.synchronize()
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    last = rows[-1].cpu().numpy().view(np.uint64)
    assert int(last[0]) == N, "valid packets != N"
    ceiling_us = ns.diag_random_atomics(1 << 28, WINDOW, 5)
    # the same window against the ingest's own two-round-trip structure, and
    # what claiming stale slots (an epoch mark instead of the clear) would add
    slots = 1 << 28  # the link, row and column tables' capacity here (load <= 1/4)
    claim_add_us = ns.diag_random_claims(slots, WINDOW, "claim_add", 5)
    stale_us = ns.diag_random_claims(slots, WINDOW, "claim_stale", 5)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(cap):
        ns.matrix_clear(A)
        e0.record()
        for _ in range(5):
            ns.matrix_clear(A)
        e1.record()
    torch.cuda.synchronize()
    clear_ms = e0.elapsed_time(e1) / 5
    peak, peak_src = peak_hbm()
    kus = float(np.mean(launch_ms)) * 1e3
    rec = {
        "workload": "accumulated RMAT stream: 2^26 packets as 512 windows of 2^17, running quantities "
                    "after every window (plain per-window launches, one CUDA graph per step)",
        "value": steps * N / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
        "gpu_launches": steps * NW, "clocks": clk, "hash_load": args.hash_load,
        "roofline": {"bound": "hbm", "kernel": "k_insert_packets", "alg_bytes_per_launch": alg_per_launch,
                     "launch_us_avg": kus, "achieved": alg_per_launch / (kus / 1e6) / 1e9, "peak": peak,
                     "frac": alg_per_launch / (kus / 1e6) / 1e9 / peak, "peak_source": peak_src,
                     "traffic": (profile_traffic("k_insert_packets.stream_rmat_window_2p17.md",
                                                 ["ns_hash.cu", "ns_common.cuh"]) or {}).get("bytes")},
        "roofline_random_access": {"kernel_us": kus, "ceiling_us": ceiling_us, "frac": ceiling_us / kus,
                                   "ceiling": "2^17 threads x 3 random 8-byte atomics into three 2 GiB tables",
                                   "structure_ceiling_us": claim_add_us, "structure_frac": claim_add_us / kus,
                                   "structure_ceiling": "2^17 threads x 3 random 16-byte CAS claims into three "
                                                        "4 GiB tables, then 2 dependent adds (the ingest's two "
                                                        "round trips)"},
        "clear_vs_epoch": {"clear_ms_per_step": clear_ms, "stale_claim_us": stale_us,
                           "epoch_extra_ms_per_step": NW * max(stale_us - claim_add_us, 0.0) / 1e3,
                           "note": "an epoch mark replaces the per-step clear of the three tables by a second "
                                   "compare-and-swap on every slot's first touch after the clear"},
    }
    if not args.no_e2e:
        h_rows = torch.empty(NW, 16, dtype=torch.int64).pin_memory()
        copy = torch.cuda.Stream(dev)
        CH = 32
        chunks = [(c, min(c + CH, NW)) for c in range(0, NW, CH)]
        ready = [torch.cuda.Event() for _ in chunks]

        def e2e_step():
            copy.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(copy):
                for (a, b_), e in zip(chunks, ready):
                    sl = slice(a * WINDOW, b_ * WINDOW)
                    d_src[sl].copy_(h_src[sl], non_blocking=True)
                    d_dst[sl].copy_(h_dst[sl], non_blocking=True)
                    e.record(copy)
            ns.matrix_clear(A)
            for (a, b_), e in zip(chunks, ready):
                torch.cuda.current_stream().wait_event(e)
                for w in range(a, b_):
                    sl = slice(w * WINDOW, (w + 1) * WINDOW)
                    ns.window_ingest_stats(ctx, A, d_src[sl], d_dst[sl], rows[w])
            h_rows.copy_(rows, non_blocking=True)
            torch.cuda.current_stream().wait_stream(copy)

        g_e2e = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g_e2e, stream=cap):
            e2e_step()
        for _ in range(2):
            g_e2e.replay()
        ms_e, _, _ = timed(g_e2e.replay, steps)
        assert int(h_rows[-1].numpy().view(np.uint64)[0]) == N, "e2e: valid packets != N"
        rec["e2e"] = {"value": steps * N / (ms_e / 1e3), "unit": UNIT, "h2d_bytes_per_step": 8 * N,
                      "d2h_bytes_per_step": NW * 16 * 8}
    A.free()
    ctx.close()
    return rec


# ----------------------------------------------------- batched (workload 4)

def c4_record(args, local, clocks, steps=None):
    """Workload 4: per-window quantities plus the running aggregate, as one
    autotuned batched launch sequence and as plain per-window launches
    (build, statistics, accumulate), each captured in a CUDA graph."""
    import torch
    import gen.workloads as W
    import paper_2509_03653_b300 as ns

    dev = torch.device("cuda", local)
    steps = steps or max(1, min(args.steps, 5))
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
    # the library picks each step's path: windows of up to 2^20 packets take
    # the hash path (plain arm), and the batched arm's empty aggregate over
    # all 1.2e9 packets takes one sort-path build
    ctx = ns.Context(local, path="auto", hbm_budget_bytes=96 << 30, tuner_cache=args.tuner_cache)
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
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cap):
            fn()
        for _ in range(max(args.warmup, 3)):
            g.replay()
        ms, t0, t1 = timed(g.replay, steps)
        res[name] = {"ms_per_step": ms / steps, "packets_per_s": steps * total / (ms / 1e3),
                     "clocks": clocks.summary(t0, t1), "aggregate": ns.network_stats(ctx, acc)}
        del g
    agree = bool(torch.equal(out_b, out_p)) and res["plain"]["aggregate"] == res["batched"]["aggregate"]
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
    # DRAM traffic per launch: the committed ncu summary's bytes per packet for
    # the configuration the tuner picked, times the packets of one launch
    tpp = profile_traffic_keyed("k_batch_insert.batched_1024_windows.md", ["ns_hash.cu", "ns_batch.cu", "ns_common.cuh"],
                                f"{params['tile_packets']},{params['ctas_per_sm']},{params['max_load']:g},"
                                f"{params['cta_cache']}")
    traffic = tpp * total / kl if (tpp and kl) else None
    b, p_ = res["batched"], res["plain"]
    batch.free()
    At.free()
    acc.free()
    ctx.close()
    return {
        "workload": f"batched: {Wn} windows, sizes log-uniform in [2^10, 2^20] ({total} packets), per-window "
                    "Zipf exponent U[0.8,1.4] over 2^20 addresses; per-window quantities plus the running aggregate",
        "value": b["packets_per_s"], "unit": UNIT, "ms_per_step": b["ms_per_step"], "steps": steps,
        "clocks": b["clocks"], "batched_vs_plain": b["packets_per_s"] / p_["packets_per_s"],
        "plain": {"packets_per_s": p_["packets_per_s"], "ms_per_step": p_["ms_per_step"], "clocks": p_["clocks"],
                  "launches_per_step": 3 * Wn},
        "results_agree": agree, "batch_params": params, "tune_s": round(tune_s, 1), "generator_s": round(gen_s, 1),
        "roofline": {"bound": "hbm", "kernel": "k_batch_insert", "alg_bytes_per_launch": kbytes / max(kl, 1),
                     "achieved": frac * peak if frac else None, "peak": peak, "frac": frac, "traffic": traffic,
                     "peak_source": peak_src},
        "kernels_ms": kernels_ms(tr),
        "aggregate": b["aggregate"],
    }


# ----------------------------------------------------- serving (workload 5)

def c5_record(args, local, clocks):
    """Workload 5: windows of log-uniform size in [2^12, 2^22] (RMAT scale
    32 + 10% uniform) from pinned host memory.  Phase 1 measures the
    service's capacity with every window submitted at once (closed loop);
    phase 2 submits fresh windows as a Poisson process at 80% of that rate
    (latency = submit -> both statistics records on the host).  The phase-2
    windows then go through a plain per-window loop (host build with its
    quantities, accumulate, the running quantities; one window at a time)."""
    import threading as th
    import torch
    import gen.workloads as W
    import paper_2509_03653_b300 as ns

    Wn = args.serve_windows
    sizes, _ = W.serving_plan(2 * Wn, 1.0)
    wins = []
    for w in range(2 * Wn):
        s, d = W.serving_window(w, int(sizes[w]))
        wins.append((torch.from_numpy(s.view(np.int32)).pin_memory(), torch.from_numpy(d.view(np.int32)).pin_memory()))
    phase = [wins[:Wn], wins[Wn:]]
    pk = [int(sizes[:Wn].sum()), int(sizes[Wn:].sum())]
    ctx = ns.Context(local, path="hash", max_slots=8, hbm_budget_bytes=64 << 30, cta_cache=args.serve_cache)
    acc = ns.Matrix(ctx)
    ns.matrix_reserve(acc, max(pk))
    srv = ns.Server(ctx, acc)
    srv.reserve(int(sizes.max()))
    for t in [ns.stream_submit(srv, s, d, i) for i, (s, d) in enumerate(wins[:16])]:
        ns.stream_wait(srv, t)
    srv.clear()

    # phase 1: closed loop -> capacity
    t0 = time.perf_counter()
    tw0 = time.time()
    pending, i = [], 0
    while i < Wn or pending:
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
    cap_clk = clocks.summary(tw0, time.time())
    cap_wps, cap_pps = Wn / cap_s, pk[0] / cap_s
    srv.clear()

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

    tw0 = time.time()
    thr = th.Thread(target=submitter)
    thr.start()
    lat, first, last, results = [], None, None, []
    for i in range(Wn):
        while tickets[i] is None:
            time.sleep(0.0001)
        pw, run, tm = ns.stream_wait(srv, tickets[i])
        results.append((pw, run))
        lat.append((tm["complete_us"] - tm["submit_us"]) / 1e3)
        first = tm["submit_us"] if first is None else min(first, tm["submit_us"])
        last = tm["complete_us"] if last is None else max(last, tm["complete_us"])
    thr.join()
    poisson_clk = clocks.summary(tw0, time.time())
    srv.close()
    span_s = (last - first) / 1e6
    lat = np.array(lat)

    # capacity again on a fresh service whose slots are not reserved: they
    # grow on demand, in stream order on their own streams
    ctx_g = ns.Context(local, path="hash", max_slots=8, hbm_budget_bytes=64 << 30, cta_cache=args.serve_cache)
    acc_g = ns.Matrix(ctx_g)
    ns.matrix_reserve(acc_g, max(pk))
    srv_g = ns.Server(ctx_g, acc_g)
    t0 = time.perf_counter()
    pending, i = [], 0
    while i < Wn or pending:
        while i < Wn:
            try:
                pending.append(ns.stream_submit(srv_g, phase[0][i][0], phase[0][i][1], i))
                i += 1
            except ns.NsError as e:
                if e.name != "NS_ERR_BUSY":
                    raise
                break
        if pending:
            ns.stream_wait(srv_g, pending.pop(0))
    grow_s = time.perf_counter() - t0
    srv_g.close()
    acc_g.free()
    ctx_g.close()

    # the same phase-2 windows through a plain per-window loop
    ctx_p = ns.Context(local, path="hash", cta_cache=args.serve_cache)
    acc_p, At = ns.Matrix(ctx_p), ns.Matrix(ctx_p)
    ns.matrix_reserve(acc_p, pk[1])
    ns.matrix_reserve(At, int(sizes.max()))
    ns.window_build_host(ctx_p, phase[1][0][0], phase[1][0][1], At)  # sizes the staging buffers
    torch.cuda.synchronize()
    agree = True
    tw0 = time.time()
    t0 = time.perf_counter()
    for i, (s, d) in enumerate(phase[1]):
        pw = ns.window_build_host(ctx_p, s, d, At)
        ns.accumulate(ctx_p, acc_p, At)
        run = ns.network_stats(ctx_p, acc_p)
        agree &= (pw, run) == results[i]
    plain_s = time.perf_counter() - t0
    plain_clk = clocks.summary(tw0, time.time())
    At.free()
    acc_p.free()
    ctx_p.close()
    acc.free()
    ctx.close()
    return {
        "workload": f"streaming serving: {Wn} windows per phase, sizes log-uniform in [2^12, 2^22], RMAT scale 32 "
                    "+ 10% uniform from pinned host memory, Poisson arrivals at 80% of measured capacity, 64 GiB "
                    "HBM admission budget, 8 slots",
        "value": pk[1] / span_s, "unit": UNIT, "packets": pk[1],
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "mean": float(lat.mean()), "max": float(lat.max())},
        "capacity": {"windows_per_s": cap_wps, "packets_per_s": cap_pps, "clocks": cap_clk},
        "capacity_slots_grow_on_demand": {"windows_per_s": Wn / grow_s, "packets_per_s": pk[0] / grow_s,
                                          "note": "fresh service, no ns_server_reserve (first use of each slot "
                                                  "included)"},
        "offered_windows_per_s": rate, "busy_retries": busy[0], "clocks": poisson_clk,
        "plain_per_window": {"packets_per_s": pk[1] / plain_s, "windows_per_s": Wn / plain_s, "clocks": plain_clk,
                             "loop": "ns_window_build_host + ns_accumulate + ns_network_stats per window, "
                                     "one window at a time",
                             "results_equal_service": bool(agree)},
        "served_vs_plain": cap_pps / (pk[1] / plain_s),
    }


# ------------------------------------------------- single-workload runs

def run_single(args, rank, world, local):
    """One sub-record's workload alone, printed as its own line (rank 0)."""
    import torch
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if rank != 0:
        return
    clocks = ClockSampler(local)
    clocks.start()
    if args.workload == "stream":
        rec = c2_record(args, local, clocks, steps=args.steps)
    elif args.workload == "batched":
        rec = c4_record(args, local, clocks, steps=args.steps)
    elif args.workload == "serve":
        rec = c5_record(args, local, clocks)
    elif args.workload == "anonymize":
        rec = anonymize_record(args, local)
    else:
        rec = slide_record(args, local)
    clocks.stop()
    rec.update({"metric": METRIC if args.workload in ("stream", "batched", "serve") else rec.get("metric"),
                "n_gpus": 1, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u64", "data": "synthetic"})
    print(json.dumps(rec), flush=True)


def anonymize_record(args, local):
    """Address anonymization of N packets (default 2^30, the headline's
    Zipf(1.2) input): distinct addresses of both columns, a random
    permutation drawn from counter-based random keys, and the gather."""
    import torch
    import gen
    import gen.workloads as W
    import paper_2509_03653_b300 as ns

    dev = torch.device("cuda", local)
    N = args.packets
    h_src = torch.empty(N, dtype=torch.int32).pin_memory()
    h_dst = torch.empty(N, dtype=torch.int32).pin_memory()
    W.large_build(N, src=h_src.numpy().view(np.uint32), dst=h_dst.numpy().view(np.uint32))
    h_rand = torch.empty(2 * N, dtype=torch.int64).pin_memory()
    gen.random_u64(2 * N, W.seed_of(3), 9, out=h_rand.numpy().view(np.uint64))
    d_src, d_dst, d_rand = h_src.to(dev), h_dst.to(dev), h_rand.to(dev)
    o_src, o_dst = torch.empty_like(d_src), torch.empty_like(d_dst)
    ctx = ns.Context(local)
    for _ in range(max(args.warmup, 3)):
        _, _, nu = ns.anonymize(ctx, d_src, d_dst, d_rand, o_src, o_dst)
    ms, _, _ = timed(lambda: ns.anonymize(ctx, d_src, d_dst, d_rand, o_src, o_dst), args.steps)
    ms /= args.steps
    ns.trace_enable(ctx, True)
    ns.anonymize(ctx, d_src, d_dst, d_rand, o_src, o_dst)
    tr = ns.trace_read(ctx)
    ns.trace_enable(ctx, False)
    peak, peak_src = peak_hbm()
    # minimal bytes: both columns read into the address set (8N); the
    # distinct addresses compacted, sorted and widened (48 nu); the
    # permutation's pair sort (256 nu); the gather (16N)
    path_bytes = 24 * N + 304 * nu
    return {"metric": "packets/s anonymized (distinct addresses, random permutation, gather)",
            "value": N / (ms / 1e3), "unit": "packets/s", "steps": args.steps, "ms_per_step": ms,
            "workload": f"address anonymization of {N} packets (headline input)", "distinct_addresses": nu,
            "roofline": {"bound": "hbm", "achieved": path_bytes / (ms / 1e3) / 1e9, "peak": peak,
                         "frac": path_bytes / (ms / 1e3) / 1e9 / peak, "peak_source": peak_src},
            "kernels_ms": kernels_ms(tr)}


def slide_record(args, local):
    """The stream workload's windows through a slider over the last K
    windows: each window's own quantities and those of the sliding sum."""
    import torch
    import gen.workloads as W
    import paper_2509_03653_b300 as ns

    dev = torch.device("cuda", local)
    NW, K = args.windows, args.slide_windows
    N = NW * WINDOW
    h_src = torch.empty(N, dtype=torch.int32).pin_memory()
    h_dst = torch.empty(N, dtype=torch.int32).pin_memory()
    W.rmat_stream(N, src=h_src.numpy().view(np.uint32), dst=h_dst.numpy().view(np.uint32))
    d_src, d_dst = h_src.to(dev), h_dst.to(dev)
    ctx = ns.Context(local, path="hash", cta_cache="off")
    out_w = torch.zeros(NW, 16, dtype=torch.int64, device=dev)
    out_s = torch.zeros(NW, 16, dtype=torch.int64, device=dev)
    sl = ns.Slider(ctx, K)

    def step():
        for w in range(NW):
            a = w * WINDOW
            ns.slider_push(ctx, sl, d_src[a:a + WINDOW], d_dst[a:a + WINDOW], out_w[w], out_s[w])

    for _ in range(max(args.warmup, 3)):
        step()
    ms, _, _ = timed(step, args.steps)
    ms /= args.steps
    return {"metric": "packets/s with per-window and sliding-window (last K windows) statistics after every window",
            "value": N / (ms / 1e3), "unit": "packets/s", "steps": args.steps, "ms_per_step": ms,
            "workload": f"sliding windows: {NW} windows of 2^17 RMAT packets, K = {K}", "ms_per_window": ms / NW}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload in ("headline", "oneshot"):
        run_headline(args, rank, world, local, oneshot_only=args.workload == "oneshot")
        return
    run_single(args, rank, world, local)


if __name__ == "__main__":
    main()
