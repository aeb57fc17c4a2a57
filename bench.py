#!/usr/bin/env python
"""Benchmark of the DIST hot path: one step = the whole path on one pair.

Workload: one pair m = n = 4096 over ACGT (i.i.d. by default, or the
correlated variant), full int32 DIST of the whole grid + LCS length + one LCS
by leftmost-argmax traceback.  Metric: GCUPS = m*n cells per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun with one process per GPU; every rank solves its own
pair of the same workload (independent problems, no data-path collective) and
the value is all ranks' cells over the slowest rank's time ("weak" scaling).
The reference arm times the CPU oracle (the only implementation of the
method besides ours) on the host cores, on a bounded sample of each step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Hardware work queues of this process's CUDA context (read once, when the
# context is created, so before torch touches the GPU).  Every batch of the
# serving loop runs on streams of its own; with the default 8 queues, dozens
# of batches in flight share them and a small batch's kernels wait behind
# another batch's long sweeps.  The single-pair solve is unaffected.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

METRIC = "GCUPS (m·n/s) per pair"
UNIT = "GCUPS"
L2_FLUSH_BYTES = 256 << 20


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--variant", choices=["iid", "correlated"], default="iid")
    ap.add_argument("--strip-height", type=int, default=0, help="0: autotuned")
    ap.add_argument("--no-graphs", action="store_true", help="plain launches instead of CUDA-graph replay")
    ap.add_argument("--schedule", choices=["auto", "retain", "depth"], default="auto",
                    help="tree schedule of the 4096 pair's solves (lcs_set_schedule)")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-pair16384", action="store_true", help="skip the m = n = 16384 pair measurement")
    ap.add_argument("--plain-pairs", type=int, default=20000,
                    help="pairs of the batched workload run one lcs_batch_submit each (the plain form)")
    ap.add_argument("--tree-pairs", type=int, default=2000,
                    help="pairs of the batched workload run through lcs_solve one by one (tree path)")
    ap.add_argument("--pair16384-steps", type=int, default=10)
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="serving arrivals per second")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def workload(variant, rank):
    from paper_2309_09072_gb300 import inputs
    a, b = inputs.pair_4096(variant, seed=1 + rank)
    return a, b


def config_dict(variant, m, n):
    """The workload, the same for both arms."""
    return {"workload": "single pair m=n=4096, ACGT %s: int32 DIST of the whole grid + LCS length + "
                        "leftmost-argmax LCS" % variant,
            "m": m, "n": n, "variant": variant, "dist_dtype": "int32",
            "l2": "flushed between steps (256 MiB write outside the timed events)"}


def max_over_ranks(x, world, device=None):
    """Largest value of x over the ranks of the process group (x itself for
    one rank): the job's time is its slowest rank's."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def aggregate_gcups(world, m, n, steps, seconds):
    """Whole-job throughput: every rank solves `steps` pairs of m x n cells,
    over the slowest rank's time."""
    return world * m * n * steps / seconds / 1e9


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index):
        self.lines = []
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + ",".join(self.FIELDS), "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.4)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [l.split(",") for l in out.strip().splitlines() if l.count(",") >= 8]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if "Active" in r[5 + k] and "Not" not in r[5 + k]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ CPU oracle
def oracle_step(a, b, nthreads=0):
    """Time one complete step of the oracle: every one of the n+1 DIST rows
    (the per-source DP, sources spread over the host threads) plus the
    leftmost traceback.  Nothing is extrapolated.  Returns (seconds, threads)."""
    import oracle
    t0 = time.perf_counter()
    oracle.dist(a, b, nthreads)
    oracle.traceback(a, b)
    t = time.perf_counter() - t0
    return t, nthreads or os.cpu_count() or 1


def length_dp_baseline(a, b):
    """The oracle's textbook two-row O(mn) DP (length only) on the host: one
    pair on one core, and one pair per core on all cores at once (the C call
    releases the GIL)."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    m, n = len(a), len(b)
    oracle.lcs_length(a[:64], b[:64])              # loads the library
    t0 = time.perf_counter()
    L = oracle.lcs_length(a, b)
    t1 = time.perf_counter() - t0
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    with ThreadPoolExecutor(cores) as ex:
        list(ex.map(lambda _: oracle.lcs_length(a, b), range(cores)))
    tn = time.perf_counter() - t0
    return {"kind": "oracle two-row O(mn) DP, length only", "unit": UNIT, "length": L,
            "one_core": m * n / t1 / 1e9, "all_cores": cores * m * n / tn / 1e9, "cores": cores,
            "sample": "the whole pair; all cores: one copy of the pair per core"}


def pairs_length_dp(pairs, sample):
    """The oracle's two-row O(mn) DP (length only) over many pairs, spread
    over all host cores (the C call releases the GIL); largest pairs first,
    dealt round-robin into chunks so the pool's tail stays short."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    cores = os.cpu_count() or 1
    oracle.lcs_length(pairs[0][0][:8], pairs[0][1][:8])      # loads the library
    cells = sum(len(x) * len(y) for x, y in pairs)
    order = sorted(range(len(pairs)), key=lambda k: -len(pairs[k][0]) * len(pairs[k][1]))
    chunks = [order[c::cores * 4] for c in range(cores * 4)]

    def run(chunk):
        for k in chunk:
            oracle.lcs_length(pairs[k][0], pairs[k][1])

    t0 = time.perf_counter()
    with ThreadPoolExecutor(cores) as ex:
        list(ex.map(run, chunks))
    t = time.perf_counter() - t0
    return {"kind": "oracle two-row O(mn) DP, length only", "unit": UNIT, "value": cells / t / 1e9,
            "cores": cores, "seconds": t, "pairs": len(pairs), "sample": sample}


def workload_baselines(batched, serve_seconds, serve_rate=2000.0, serve_sample=2000):
    """Host baselines of the batched and serving workloads (the same seeded
    pairs the GPU measurements use)."""
    from paper_2309_09072_gb300 import inputs
    out = {}
    if batched:
        out["batched_length_dp"] = pairs_length_dp(inputs.batch_pairs(), "all 20,000 pairs of the batched workload")
    if serve_seconds > 0:
        import oracle
        _, req = inputs.serving_requests(duration_s=serve_seconds, rate=serve_rate)
        req = req[:serve_sample]
        r = pairs_length_dp(req, "the first %d requests of the serving workload" % len(req))
        big = next(((x, y) for x, y in req if len(x) * len(y) >= 16384 * 16384), None)
        if big is not None:
            t0 = time.perf_counter()
            oracle.lcs_length(big[0], big[1])
            r["pair_16384_one_core_ms"] = (time.perf_counter() - t0) * 1e3
        out["serving_length_dp"] = r
    return out


def cpu_baseline(a, b):
    m, n = len(a), len(b)
    t, threads = oracle_step(a, b)
    return {"value": m * n / t / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
            "seconds": t,
            "sample": "one complete step, timed: the oracle's per-source DIST for all %d rows (all host "
                      "threads) plus the full O(mn) leftmost traceback" % (n + 1),
            "method_rate": method_rate(m, n, t),
            "length_dp": length_dp_baseline(a, b)}


def method_rate(m, n, seconds):
    """The method's own work rate: DIST from every source, m (n+1) n / 2 cell
    updates per pair (each of the n+1 sources sweeps its remaining columns
    over all m rows), per second."""
    return {"value": m * n * (n + 1) / 2 / seconds, "unit": "cell updates/s",
            "per_pair": m * n * (n + 1) / 2}


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    a, b = workload(args.variant, 0)
    m, n = len(a), len(b)
    for _ in range(args.warmup):
        oracle_step(a, b)
    total = 0.0
    threads = 1
    for _ in range(args.steps):
        t, threads = oracle_step(a, b)
        total += t
    ms = total / args.steps * 1e3
    value = m * n * args.steps / total / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": config_dict(args.variant, m, n), "impl": "reference",
            "method_rate": method_rate(m, n, total / args.steps),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": "every step complete and timed: the oracle's per-source DIST for all "
                                       "%d rows (all host threads) + the full leftmost traceback" % (n + 1)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm
def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def recorded_counter(kernel_src, summary, key):
    """A per-launch counter recorded in a committed ncu summary (`key: value`
    lines), or None when the kernel source changed since it was taken."""
    import hashlib
    try:
        sha = hashlib.sha256(open(os.path.join(ROOT, kernel_src), "rb").read()).hexdigest()[:16]
        fields = {}
        for line in open(os.path.join(ROOT, "profiles", summary)):
            if ":" in line and not line.startswith((" ", "|", "#")):
                k, v = line.split(":", 1)
                fields[k.strip()] = v.strip()
        if fields.get("source_sha256_prefix") != sha:
            return None
        return float(fields[key])
    except (OSError, KeyError, ValueError):
        return None


def recorded_traffic(kernel_src, summary):
    """DRAM bytes per launch from a committed ncu summary (or None)."""
    return recorded_counter(kernel_src, summary, "traffic_bytes_per_launch")


def roofline(profile, peaks, peaks_src, int_peak):
    """Dominant kernel (largest share of device time) against its bound."""
    if not profile:
        return None
    kind, p = max(profile.items(), key=lambda kv: kv[1]["ms"])
    per_launch_ms = p["ms"] / p["launches"]
    share = p["ms"] / sum(v["ms"] for v in profile.values())
    if kind == "strip":
        achieved = p["ops"] / p["launches"] / (per_launch_ms * 1e-3) / 1e9
        return {"kernel": kind, "bound": "alu", "achieved": achieved, "peak": int_peak["derived_gops"],
                "unit": "Gop/s", "frac": achieved / int_peak["derived_gops"], "traffic": None,
                "peak_source": "152 SMs x 128 INT32 lanes/clk x 2070 MHz (derived)",
                "measured_int32_gops": int_peak["measured_gops"], "share_of_device_time": share,
                "ms_per_launch": per_launch_ms, "launches": p["launches"]}
    achieved = p["bytes"] / p["launches"] / (per_launch_ms * 1e-3) / 1e9
    peak = peaks["hbm_gbs"]
    traffic = None
    out = {}
    if kind == "merge_tile":
        src, summ = "paper_2309_09072_gb300/csrc/merge.cu", "merge_tile_dpx_pair4096.md"
        traffic = recorded_traffic(src, summ)
        alu = recorded_counter(src, summ, "alu_pipe_pct_of_peak_active")
        if alu is not None:
            # The counted bound is HBM (algorithmic bytes); the kernel itself is
            # bound by the (max,+) arithmetic: the DPX issue pipe, from ncu.
            out["measured_bound"] = {"pipe": "alu (DPX max-plus)", "pct_of_peak_active": alu,
                                     "source": "profiles/" + summ}
    return {"kernel": kind, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "peak_source": "hbm_gbs of %s" % peaks_src,
            "algorithmic_bytes_per_launch": p["bytes"] / p["launches"],
            "share_of_device_time": share, "ms_per_launch": per_launch_ms, "launches": p["launches"], **out}


def pair16384_measure(B, torch, peaks, peaks_src, steps=10):
    """The m = n = 16384 pair (20 letters, Zipf(1.1)): int16 DIST of the whole
    grid + length + LCS, autotuned, CUDA-graph replay, timed with CUDA events
    on the launching stream (its 0.5 GB output and ~10 GB of merge operands
    exceed L2); the merge tiles' share and HBM roofline from a profiled pass."""
    from paper_2309_09072_gb300 import inputs
    a, b = inputs.pair_16384()
    m, n = len(a), len(b)
    dev = torch.device("cuda")
    ctx = B.lcs_create(torch.cuda.current_device(), 0)
    try:
        ad = torch.from_numpy(a.copy()).to(dev)
        bd = torch.from_numpy(b.copy()).to(dev)
        ld = ((n + 1) * 2 + 15) // 16 * 16 // 2
        dist = torch.empty((n + 1, ld), dtype=torch.int16, device=dev)
        lcs = torch.empty(min(m, n), dtype=torch.uint8, device=dev)
        ln = torch.empty(1, dtype=torch.int64, device=dev)
        tuned = B.lcs_autotune(ctx, ad, bd, dist=dist, out_lcs=lcs)
        B.lcs_set_graphs(ctx, True)
        stream = torch.cuda.current_stream(dev)
        for _ in range(2):
            B.lcs_solve(ctx, ad, bd, dist=dist, out_lcs=lcs, out_len=ln, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        B.lcs_sync(ctx, stream)
        e0.record(stream)
        for _ in range(steps):
            B.lcs_solve(ctx, ad, bd, dist=dist, out_lcs=lcs, out_len=ln, stream=stream)
        e1.record(stream)
        B.lcs_sync(ctx, stream)
        ms = e0.elapsed_time(e1) / steps
        B.lcs_set_profiling(ctx, True)
        B.lcs_solve(ctx, ad, bd, dist=dist, out_lcs=lcs, out_len=ln, stream=stream)
        B.lcs_sync(ctx, stream)
        profile = B.lcs_get_profile(ctx)
        B.lcs_set_profiling(ctx, False)
        stats = B.lcs_get_stats(ctx)
        L = int(ln.item())
        # Device memory of the chosen configuration alone: a fresh context
        # (the autotuner's candidates grew this one's workspace) for one solve.
        ctx2 = B.lcs_create(torch.cuda.current_device(), 0)
        try:
            B.lcs_set_strip_height(ctx2, stats["strip_height"])
            B.lcs_set_merge_kernel(ctx2, tuned["merge_kernel"])
            B.lcs_solve(ctx2, ad, bd, dist=dist, out_lcs=lcs, out_len=ln, stream=stream)
            B.lcs_sync(ctx2, stream)
            mem = B.lcs_get_stats(ctx2)
        finally:
            B.lcs_destroy(ctx2)
        # End to end through lcs_solve_host: a and b from pinned host memory,
        # the 0.5 GB int16 DIST, the LCS and the length back every step.
        del dist
        ah = torch.from_numpy(a.copy()).pin_memory()
        bh = torch.from_numpy(b.copy()).pin_memory()
        dh = torch.empty((n + 1, ld), dtype=torch.int16).pin_memory()
        lh = torch.empty(min(m, n), dtype=torch.uint8).pin_memory()
        B.lcs_solve_host(ctx, ah, bh, dist_host=dh, lcs_host=lh, dtype=B.LCS_I16, stream=stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            Lh = B.lcs_solve_host(ctx, ah, bh, dist_host=dh, lcs_host=lh, dtype=B.LCS_I16, stream=stream)
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / steps
        e2e = {"value": m * n / e2e_s / 1e9, "unit": "GCUPS", "ms_per_step": e2e_s * 1e3, "steps": steps,
               "h2d_bytes_per_step": m + n, "d2h_bytes_per_step": (n + 1) * (n + 1) * 2 + Lh + 16,
               "api": "lcs_solve_host (pinned host buffers, int16 DIST)"}
        mt = profile.get("merge_tile")
        merge = None
        if mt:
            per = mt["ms"] / mt["launches"]
            achieved = mt["bytes"] / mt["launches"] / (per * 1e-3) / 1e9
            merge = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "peak_source": "hbm_gbs of %s" % peaks_src,
                     "algorithmic_bytes_per_launch": mt["bytes"] / mt["launches"], "ms_per_launch": per,
                     "launches": mt["launches"]}
        return {"workload": "single pair m=n=16384, 20 letters Zipf(1.1): int16 DIST of the whole grid + LCS "
                            "length + leftmost-argmax LCS", "value": m * n / (ms * 1e-3) / 1e9, "unit": "GCUPS",
                "ms_per_step": ms, "steps": steps, "method_rate": method_rate(m, n, ms * 1e-3), "e2e": e2e,
                "strip_height": stats["strip_height"],
                "merge_kernel": {1: "exact", 2: "dpx"}.get(tuned["merge_kernel"], "auto"),
                "lcs_length": L, "peak_workspace_bytes": mem["peak_workspace_bytes"],
                "schedule": {"depth_first": bool(mem["depth_first"]), "chunk_strips": mem["chunk_strips"],
                             "plan_bytes": mem["plan_bytes"],
                             "peak": "device workspace of a fresh context for one solve of the chosen "
                                     "configuration (the DIST output is the caller's, 0.54 GB, not counted)"},
                "kernels": {k: {"launches": v["launches"], "ms": v["ms"]} for k, v in profile.items()},
                "merge_roofline": merge}
    finally:
        B.lcs_destroy(ctx)


def batched_measure(B, torch, plain_pairs, tree_pairs, reps=3):
    """The batched form (one lcs_batch_submit of the 20,000-pair workload,
    one LCS per pair) against the plain per-pair form of the same
    computation: the same pairs, one lcs_batch_submit + lcs_batch_poll per
    pair, one after another.  Separately labelled: lcs_solve pair by pair
    (the strip tree with every source's DIST, a different algorithm) on the
    first `tree_pairs` pairs.  All through the library's C entry points on
    strings already on the device."""
    import ctypes
    import numpy as np
    from paper_2309_09072_gb300 import inputs
    pairs = inputs.batch_pairs()
    sizes = [(len(x), len(y)) for x, y in pairs]
    dbuf = torch.from_numpy(np.concatenate([np.concatenate([x, y]) for x, y in pairs])).cuda()
    base = dbuf.data_ptr()
    arr = (B.lcs_pair * len(pairs))()
    off = 0
    for k, (m, n) in enumerate(sizes):
        arr[k].a, arr[k].m = base + off, m
        arr[k].b, arr[k].n = base + off + m, n
        arr[k].flags = B.LCS_WANT_STRING
        off += m + n
    res = (B.lcs_result * len(pairs))()
    lib = B.load()
    ctx = B.lcs_create(0, 0)
    ticket, done = ctypes.c_uint64(), ctypes.c_int64()

    def one_batch():
        B._check(ctx, lib.lcs_batch_submit(ctx, arr, len(pairs), ctypes.byref(ticket)))
        B._check(ctx, lib.lcs_batch_poll(ctx, ticket.value, res, len(pairs), ctypes.byref(done), -1))
        B._check(ctx, lib.lcs_batch_release(ctx, ticket.value))

    for _ in range(2):
        one_batch()
    times = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        one_batch()
        times.append(time.perf_counter() - t0)
    bad = sum(1 for k in range(len(pairs)) if res[k].status != B.LCS_OK)
    cells = sum(m * n for m, n in sizes)
    batch_s = sorted(times)[len(times) // 2]
    # Plain per-pair form: the same kernels, one pair per submission.
    k_plain = min(plain_pairs, len(pairs))
    one = (B.lcs_result * 1)()

    def one_pair(k):
        B._check(ctx, lib.lcs_batch_submit(ctx, ctypes.byref(arr[k]), 1, ctypes.byref(ticket)))
        B._check(ctx, lib.lcs_batch_poll(ctx, ticket.value, one, 1, ctypes.byref(done), -1))
        B._check(ctx, lib.lcs_batch_release(ctx, ticket.value))
        return one[0].status

    for k in range(20):
        one_pair(k)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain_bad = sum(1 for k in range(k_plain) if one_pair(k) != B.LCS_OK)
    plain_s = time.perf_counter() - t0
    plain_cells = sum(m * n for m, n in sizes[:k_plain])
    # The tree path per pair (lcs_solve).
    k_tree = min(tree_pairs, len(pairs))
    views = []
    off = 0
    for m, n in sizes[:k_tree]:
        views.append((dbuf[off:off + m], dbuf[off + m:off + m + n]))
        off += m + n
    out = torch.empty(2048, dtype=torch.uint8, device="cuda")
    ln = torch.zeros(1, dtype=torch.int64, device="cuda")
    for a, b in views[:20]:
        B.lcs_solve(ctx, a, b, out_lcs=out[:max(1, min(a.numel(), b.numel()))], out_len=ln)
    B.lcs_sync(ctx)
    t0 = time.perf_counter()
    for a, b in views:
        B.lcs_solve(ctx, a, b, out_lcs=out[:max(1, min(a.numel(), b.numel()))], out_len=ln)
    B.lcs_sync(ctx)
    tree_s = time.perf_counter() - t0
    tree_cells = sum(m * n for m, n in sizes[:k_tree])
    B.lcs_destroy(ctx)
    bv, pv, tv = cells / batch_s / 1e9, plain_cells / plain_s / 1e9, tree_cells / tree_s / 1e9
    return {"workload": "20,000 pairs, m and n log-uniform in [32, 2048], ACGT i.i.d., one LCS per pair",
            "value": bv, "unit": UNIT, "ms_per_batch": batch_s * 1e3, "pairs_failed": bad,
            "api": "lcs_batch_submit + lcs_batch_poll (strings resident on the device; host wall time of submit "
                   "to completion, median of %d)" % reps,
            "plain_value": pv,
            "plain_api": "the same computation one pair at a time: lcs_batch_submit of one pair, "
                         "lcs_batch_poll until done, lcs_batch_release, pair after pair",
            "plain_sample": "%d pairs of the same workload" % k_plain, "plain_pairs_failed": plain_bad,
            "batched_over_plain": bv / pv,
            "tree_path_per_pair": {"value": tv, "unit": UNIT, "sample": "first %d pairs" % k_tree,
                                   "api": "lcs_solve per pair: strip tree with DIST from every source, "
                                          "merges and traceback (a different algorithm from the batch's "
                                          "one-strip sweep from source 0)",
                                   "batched_over_tree_path": bv / tv}}


def serving_measure(B, torch, seconds, rate=2000.0):
    """The serving workload (Poisson arrivals at `rate` pairs/s, 20 letters,
    lengths log-uniform in [128, 8192], every 50th pair 16384 x 16384, 30%
    correlated) for `seconds` seconds of arrivals through continuous batching
    (serve.py over lcs_batch_submit/poll), strings resident on the device."""
    from paper_2309_09072_gb300 import inputs, serve
    times, pairs = inputs.serving_requests(duration_s=seconds, rate=rate)
    dev = [(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()) for a, b in pairs]
    ctx = B.lcs_create(0, 0)
    serve.serve(ctx, dev[:50], times[:50] - times[0])          # warm-up on the first requests
    out = serve.serve(ctx, dev, times)
    B.lcs_destroy(ctx)
    summ = serve.summary(out, [(len(a), len(b)) for a, b in pairs])
    summ.update({"workload": "serving: Poisson %s pairs/s for %.0f s, 20 letters, lengths log-uniform "
                             "[128, 8192], every 50th pair 16384 x 16384, 30%% correlated; one LCS per pair"
                             % (format(int(rate), ","), seconds),
                 "latency": "p50_ms/p99_ms/max_ms: device completion of the request's batch minus its "
                            "arrival; host_*: the loop's receipt of the result (after the poll and the "
                            "string copy to the host) minus its arrival"})
    return summ


def run_ours(args):
    import numpy as np
    import torch
    from paper_2309_09072_gb300 import binding as B

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    a, b = workload(args.variant, rank)
    m, n = len(a), len(b)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    ctx = B.lcs_create(local, 0)
    B.lcs_set_strip_height(ctx, args.strip_height)
    B.lcs_set_schedule(ctx, {"auto": B.LCS_SCHED_AUTO, "retain": B.LCS_SCHED_RETAIN,
                             "depth": B.LCS_SCHED_DEPTH}[args.schedule], 0)
    ad = torch.from_numpy(a.copy()).to(dev)
    bd = torch.from_numpy(b.copy()).to(dev)
    ld = ((n + 1) * 4 + 15) // 16 * 16 // 4
    dist_out = torch.empty((n + 1, ld), dtype=torch.int32, device=dev)
    lcs_out = torch.empty(min(m, n), dtype=torch.uint8, device=dev)
    len_out = torch.empty(1, dtype=torch.int64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    tuned = {"merge_kernel": 0}
    if args.strip_height == 0:
        tuned = B.lcs_autotune(ctx, ad, bd, dist=dist_out, out_lcs=lcs_out, stream=stream)
    graphs = not args.no_graphs
    B.lcs_set_graphs(ctx, graphs)

    def step():
        B.lcs_solve(ctx, ad, bd, dist=dist_out, out_lcs=lcs_out, out_len=len_out, stream=stream)

    for _ in range(max(3, args.warmup)):
        step()
    B.lcs_sync(ctx, stream)
    stats = B.lcs_get_stats(ctx)
    int_gops, int_mhz = B.lcs_measure_int32_peak(local)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    int_peak = {"measured_gops": int_gops, "measured_mhz": int_mhz,
                "derived_gops": sms * 128 * 2070e6 / 1e9}

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    barrier()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    barrier()
    clock_info = clocks.stop()
    B.lcs_sync(ctx, stream)
    total_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    # Per-kernel times: a second pass of the same steps with an event pair
    # around every launch (the events also stop consecutive kernels from
    # overlapping their launches, so this pass is not the timed one).
    prof_steps = min(args.steps, 50)
    B.lcs_set_profiling(ctx, True)
    for k in range(prof_steps):
        flush.fill_(k & 0xFF)
        step()
    B.lcs_sync(ctx, stream)
    profile = B.lcs_get_profile(ctx)
    B.lcs_set_profiling(ctx, False)
    total_ms = max_over_ranks(total_ms, world, dev)
    value = aggregate_gcups(world, m, n, args.steps, total_ms * 1e-3)

    # End to end through the public host API: H2D of a, b and D2H of DIST,
    # the LCS and the length every step.
    ah = torch.from_numpy(a.copy()).pin_memory()
    bh = torch.from_numpy(b.copy()).pin_memory()
    dh = torch.empty((n + 1, ld), dtype=torch.int32).pin_memory()
    lh = torch.empty(min(m, n), dtype=torch.uint8).pin_memory()
    L = 0
    for _ in range(2):
        L = B.lcs_solve_host(ctx, ah, bh, dist_host=dh, lcs_host=lh, stream=stream)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        L = B.lcs_solve_host(ctx, ah, bh, dist_host=dh, lcs_host=lh, stream=stream)
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, world, dev)
    e2e = {"value": aggregate_gcups(world, m, n, args.e2e_steps, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": m + n, "d2h_bytes_per_step": (n + 1) * (n + 1) * 4 + L + 16,
           "steps": args.e2e_steps, "api": "lcs_solve_host (pinned host buffers)"}

    peaks, peaks_src = load_peaks()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": config_dict(args.variant, m, n),
            "tuning": {"strip_height": stats["strip_height"], "cuda_graphs": graphs,
                       "merge_kernel": {1: "exact", 2: "dpx"}.get(tuned["merge_kernel"], "auto"),
                       "chosen_by": "lcs_autotune" if args.strip_height == 0 else "--strip-height",
                       "depth_first": bool(stats["depth_first"]), "plan_bytes": stats["plan_bytes"]},
            "e2e": e2e, "gpu_launches": stats["kernel_launches"] * args.steps,
            "method_rate": method_rate(m, n, total_ms * 1e-3 / args.steps / world),
            "roofline": roofline(profile, peaks, peaks_src, int_peak),
            "clocks": clock_info,
            "kernels": {k: {"launches": v["launches"], "ms": v["ms"]} for k, v in profile.items()},
            "kernels_steps": prof_steps,
            "lcs_length": L, "workspace_bytes": stats["peak_workspace_bytes"]}
    B.lcs_destroy(ctx)
    if rank == 0 and not args.no_pair16384:
        line["pair_16384"] = pair16384_measure(B, torch, peaks, peaks_src, args.pair16384_steps)
    if rank == 0 and not args.no_batched:
        line["batched"] = batched_measure(B, torch, args.plain_pairs, args.tree_pairs)
    if rank == 0 and args.serve_seconds > 0:
        line["serving"] = serving_measure(B, torch, args.serve_seconds, args.serve_rate)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(a, b)
        line["cpu_baseline"].update(workload_baselines(not args.no_batched, args.serve_seconds, args.serve_rate))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
