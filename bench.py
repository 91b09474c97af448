"""Benchmark: binary64 arguments checked per second on the plain exp workload.

Workload (one step): exp over a contiguous 2^36-argument slice of the
binary64 binade [1/2, 1) (seeded block-aligned start), degree-3 Taylor blocks
of 2^24 arguments in 192-bit fixed point, sub-intervals of N = 2^14
arguments, threshold m = 40: packet starts, tabulated-difference stepping,
Algorithm 4 filter, exact resolution and compaction over all 2^22 lines.

  value    device throughput of the batched form: the persistent work-queue
           kernel replayed as a CUDA graph, plan and tables resident in HBM
           when the timed region starts; arguments / s, whole job over all
           ranks.
  plain    the same work as one fused per-job launch (tmd_search).
  unfused  the same work as two launches (generate lines to HBM, then search
           them).
  e2e      the public C-ABI call from host job descriptors to the sorted
           host candidate list, every step: host planning (output-binade
           cuts), the host->device copy of the job records, the device
           planning and correctly rounded table kernels, the search kernel,
           the device->host read of the count and records.

Further sections of the same line (each skippable by its flag): Lefevre's
filter on the same slice (Table 4's comparison), the sound mode on Table 2's
domain (exp on [1, 1+2^-13[, 2^39 arguments), the sound mode on exp's binade
[128, 256) with both filters and the phase counts of Table 7, a 64-job
mixed batch against per-job launches, the large 2^16-job batch, a
Poisson-arrival serving stream, and the whole binade [1, 2) of exp in sound
mode through the public API (Table 4's workload).

Between timed steps a 256 MiB buffer (> the 129 MB L2) is written so that no
step starts with a warm L2.  `--impl reference` times the CPU oracle instead
(exact enclosures, direct Horner, brute force over every argument) on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

METRIC = "binary64 args checked/s (exp, binade slice) batched vs plain; % int-pipe peak"
UNIT = "args/s"

# Integer/FP32 issue ceiling: 152 SMs x 4 schedulers x 32 lanes per clock at
# the 2070 MHz maximum SM clock (every instruction of the path is a 32-bit
# integer, logic, conversion or FP32 operation; one warp instruction per
# scheduler per clock).
SMS, LANES_PER_SM, SM_MAX_HZ = 152, 128, 2.070e9
ISSUE_PEAK_OPS = SMS * LANES_PER_SM * SM_MAX_HZ

# Algorithmic 32-bit operations (a fixed cost model of Algorithm 4):
#   per line:       tabulated stepping (2d-1) W-bit adds = 2 (2d-1) L 32-bit
#                   add-with-carry, plus 4 to form the search words;
#   per half-step:  35 (divisor and dividend to FP32, reciprocal, two
#                   quotient estimates, two 64x32 multiply-subtracts, two
#                   corrections, the u/v update, the exit test).
OPS_PER_HALF_STEP = 35

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# k_persistent<3,3> on this 2^36 workload, from one single-pass ncu capture of
# the kernel as it stands; None until the kernel's current form is captured,
# and reset to None whenever that kernel changes.
TRAFFIC_BYTES_PER_LAUNCH = 1_416_704


def ops_per_line(job) -> int:
    return 2 * (2 * job.d - 1) * job.limbs + 4


# The method's own count (the paper's work per partial quotient, Sect. III-B,
# Algorithm 4): one quotient and one reduction of d (two 64-bit divisions),
# two 64-bit multiply-subtracts and two adds/compares per half-step, each
# counted as one operation -- the useful-work fraction beside the cost model.
METHOD_OPS_PER_HALF_STEP = 6


def roofline_of(tmd, jobs, stats, ms: float) -> dict:
    """Integer-issue roofline of one timed launch (or step) over `jobs`:
    algorithmic operations from the cost model (stepping per line, 35 per
    continued-fraction half-step counted live by the kernel) divided by the
    step time, against the derived issue ceiling."""
    lines = [tmd.tmd_plan(j)["n_subints"] for j in jobs]
    gen = sum(n * ops_per_line(j) for n, j in zip(lines, jobs))
    alg = gen + stats["half_steps"] * OPS_PER_HALF_STEP
    method = gen + stats["half_steps"] * METHOD_OPS_PER_HALF_STEP
    sec = ms / 1e3
    return {"bound": "alu", "achieved": alg / sec / 1e12, "peak": ISSUE_PEAK_OPS / 1e12, "unit": "Tops/s",
            "frac": alg / sec / ISSUE_PEAK_OPS, "frac_method": method / sec / ISSUE_PEAK_OPS,
            "half_steps_per_line": stats["half_steps"] / max(1, stats["lines"]),
            "filter_fail_per_line": stats["filter_fail"] / max(1, stats["lines"])}


def rank_info():
    r = int(os.environ.get("RANK", "0"))
    w = int(os.environ.get("WORLD_SIZE", "1"))
    lr = int(os.environ.get("LOCAL_RANK", str(r)))
    return r, w, lr


def rank_job(job, rank: int):
    """Weak scaling: rank r searches the r-th neighbouring 2^36 slice."""
    span = (1 << (job.p - 1))
    start = (job.start + rank * job.count) % (span - job.count)
    start -= start % (1 << job.log2_T)
    return job.replace(start=start)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while it runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cuda_index(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_rank < len(ids) and ids[local_rank].isdigit():
            return int(ids[local_rank])
    return local_rank


# ------------------------------------------------------------ oracle timing
def oracle_sample(job, seconds_target: float = 12.0, threads: int = 0):
    """Time the CPU oracle on consecutive blocks of the job until about
    `seconds_target` seconds of work; returns (args, seconds, blocks, threads)."""
    from oracle import candidates as oc
    from oracle import plan
    oc.build_brute() if not os.path.exists(os.path.join(ROOT, "oracle", "_brute.so")) else None
    lib = oc._brute_lib()
    nthreads = threads or (os.cpu_count() or 1)
    blocks = plan.blocks(job)
    t0 = time.perf_counter()
    done_args, nb = 0, 0
    for blk in blocks:
        oc.job_candidates(job, blocks=[blk], threads=nthreads)
        done_args += blk.length
        nb += 1
        if time.perf_counter() - t0 >= seconds_target:
            break
    dt = time.perf_counter() - t0
    used = lib.oracle_threads_available() if lib is not None else 1
    return done_args, dt, nb, min(used, nthreads)


def run_reference(args):
    r, w, _ = rank_info()
    if w > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group("gloo")
        if r != 0:
            dist.barrier()
            return
    job = wl.plain_job()
    per_step = []
    sample = None
    # the whole reference run stays within a few minutes: each step is a
    # bounded sample (at least one Taylor block) of the workload
    target = min(args.ref_seconds, 150.0 / (args.warmup + args.steps))
    for k in range(args.warmup + args.steps):
        a, dt, nb, th = oracle_sample(job, seconds_target=target)
        if k >= args.warmup:
            per_step.append((a, dt))
            sample = (nb, th)
    args_total = sum(a for a, _ in per_step)
    t_total = sum(d for _, d in per_step)
    value = args_total / t_total
    nb, th = sample
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": w,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / len(per_step),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": "exp binary64 [1/2,1) 2^36-arg slice, d=3, W=192, N=2^14, m=40",
                   "sample": f"{nb} Taylor blocks of 2^24 args per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": th, "kind": "oracle",
                         "sample": f"first {nb} blocks (2^24 args each) of the 2^36 slice per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    if w > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------- served form
SERVER_CFG = dict(max_inflight=4, chunk_tasks=0, cand_cap=1 << 16, max_batch=1024, device_budget=8 << 30)


def run_serving(tmd, ctx, jobs, rate_per_s, seed=2012):
    """Serve `jobs` arriving with exponential gaps (rate_per_s; inf = all at
    once), replayed by the server's clock (tmd_server_submit_many), and
    collect every result.  Returns (seconds from the first arrival to the
    last completion, latencies in s, total args, total records, server
    counters)."""
    n = len(jobs)
    delays = [0.0] * n if math.isinf(rate_per_s) else wl.arrival_times(n, rate_per_s, seed)
    lat, recs, t_first, t_last = [], 0, float("inf"), 0.0
    with tmd.Server(ctx, **SERVER_CFG) as srv:
        srv.submit_many(jobs, list(range(n)), delays)
        done = 0
        while done < n:
            for r, rr in srv.poll(cap=4096, rec_cap=1 << 18, wait_ms=50):
                assert r["status"] == 0, r
                lat.append(r["t_done"] - r["t_submit"])
                t_first = min(t_first, r["t_submit"])
                t_last = max(t_last, r["t_done"])
                recs += r["count"]
                done += 1
        st = srv.stats()
    return t_last - t_first, lat, sum(j.count for j in jobs), recs, st


def percentile(xs, q):
    ys = sorted(xs)
    return ys[min(len(ys) - 1, int(q * (len(ys) - 1) + 0.5))]


# ------------------------------------------------------------- native arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--ref-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--m", type=int, default=40)
    ap.add_argument("--mixed-jobs", type=int, default=64,
                    help="jobs of the seeded mixed batch for batched vs per-job launches (0 = skip)")
    ap.add_argument("--large", type=int, default=1,
                    help="run the large batch: 2^x, 2^40 args in 2^16 uneven jobs (0 = skip)")
    ap.add_argument("--serve-jobs", type=int, default=10000,
                    help="jobs of the seeded serving stream to serve (0 = skip)")
    ap.add_argument("--count-log2", type=int, default=36,
                    help="slice size (smaller only for profiling captures)")
    ap.add_argument("--sound", type=int, default=1,
                    help="also time the sound-mode search of exp on [1, 1+2^-13[ (0 = skip)")
    ap.add_argument("--lefevre", type=int, default=1,
                    help="also time the same slice with Lefevre's filter (0 = skip)")
    ap.add_argument("--binade128", type=int, default=1,
                    help="also time the sound search of exp on [128, 256), Table 7's regime (0 = skip)")
    ap.add_argument("--binade128-log2", type=int, default=36,
                    help="arguments of the [128, 256) slice (smaller only for profiling captures)")
    ap.add_argument("--binade-full", type=int, default=1,
                    help="also search the whole binade [1, 2) of exp, Table 4's workload (0 = skip)")
    ap.add_argument("--binade-full-chunks", type=int, default=1024,
                    help="2^42-argument calls of the whole-binade run (1024 = all of [1, 2))")
    ap.add_argument("--twins", type=int, default=1,
                    help="also time the dense twins (m = 20 / 20 / 22) of the plain, mixed and large workloads")
    ap.add_argument("--tiling", default="auto",
                    help="'auto' (tmd_autotune picks it) or 'nu,ctas_per_sm[,lanes[,unroll]]' for the batched form")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import paper_1211_3056_gb300 as tmd

    rank, world, local_rank = rank_info()
    torch.cuda.set_device(local_rank)
    dev = f"cuda:{local_rank}"
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    job = rank_job(wl.plain_job(m=args.m, count_log2=args.count_log2), rank)
    stream = torch.cuda.current_stream()
    ctx = tmd.Context(local_rank)
    cap = 1 << 16
    d_cand, d_count = tmd.alloc_candidates(cap, local_rank)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    # resident plan and tables (host work happens here, outside the timed region)
    tmd.tmd_search(ctx, [job], None, d_cand, d_count)
    torch.cuda.synchronize()
    need = tmd.tmd_generate(ctx, [job], None)
    d_lin = torch.empty(need // 8, dtype=torch.int64, device=dev)

    def fused_step():
        tmd.tmd_search(ctx, [job], None, d_cand, d_count)

    # batched form: the persistent work-queue kernel, captured once as a
    # graph, with the tiling the autotuner picks for this batch (untimed)
    if args.tiling == "auto":
        tuned = tmd.tmd_autotune(ctx, [job])
        tiling = None
    else:
        tl = [int(v) for v in args.tiling.split(",")] + [1, 1]
        tuned = {"nu": tl[0], "ctas_per_sm": tl[1], "lanes": tl[2], "unroll": tl[3], "ms": None}
        tiling = tuple(tl[:4])
    d_cand_b, d_count_b = tmd.alloc_candidates(cap, local_rank)
    batch = tmd.Batch(ctx, [job], d_cand_b, d_count_b, tiling=tiling)

    def batched_step():
        batch.launch()

    def plain_step():
        tmd.tmd_generate(ctx, [job], d_lin)
        tmd.tmd_search(ctx, [job], d_lin, d_cand, d_count)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            flush.fill_(1)
            fn()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        barrier()
        torch.cuda.synchronize()
        for e0, e1 in evs:
            flush.fill_(1)
            e0.record(stream)
            fn()
            e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return [e0.elapsed_time(e1) for e0, e1 in evs]

    # measured issue rates of the pipes (lane-operations per SM per clock)
    pipe_rates = tmd.tmd_pipe_rates(local_rank)

    sampler = ClockSampler(cuda_index(local_rank))
    sampler.start()
    batched_ms = timed(batched_step, args.steps, args.warmup)
    fused_ms = timed(fused_step, args.steps, args.warmup)
    clocks = sampler.stop()
    stats = batch.stats()
    recs_b, count_b = tmd.tmd_candidates(ctx, d_cand_b, d_count_b)
    recs, count = tmd.tmd_candidates(ctx, d_cand, d_count)
    assert (recs_b, count_b) == (recs, count), "batched and plain forms disagree"
    plain_ms = timed(plain_step, max(args.steps // 4, 3), args.warmup)

    def max_over_ranks(x: float) -> float:
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    ms = max_over_ranks(statistics.mean(batched_ms))
    ms_fused = max_over_ranks(statistics.mean(fused_ms))
    ms_plain = max_over_ranks(statistics.mean(plain_ms))
    total_args = job.count * world
    value = total_args / (ms / 1e3)
    fused_value = total_args / (ms_fused / 1e3)
    plain_value = total_args / (ms_plain / 1e3)

    # end to end through the C ABI: host descriptors in, host records out
    e2e_times = []
    h2d = 0
    for k in range(args.e2e_steps + 1):
        tmd.tmd_evict(ctx)
        flush.fill_(1)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        tmd.tmd_search(ctx, [job], None, d_cand, d_count)
        got, n = tmd.tmd_candidates(ctx, d_cand, d_count)
        t1 = time.perf_counter()
        if k > 0:
            e2e_times.append(t1 - t0)
    e2e_s = max_over_ranks(statistics.mean(e2e_times))
    h2d = tmd.tmd_stats_read(ctx)["upload_bytes"]
    d2h = 8 + 4 + n * tmd.CANDIDATE_BYTES

    # roofline of the persistent kernel (the step is that one launch plus two
    # 8-byte memsets in the same graph)
    alg_ops = stats["lines"] * ops_per_line(job) + stats["half_steps"] * OPS_PER_HALF_STEP
    achieved = alg_ops / (statistics.mean(batched_ms) / 1e3)
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": ISSUE_PEAK_OPS / 1e12,
                "unit": "Tops/s", "frac": achieved / ISSUE_PEAK_OPS,
                "traffic": TRAFFIC_BYTES_PER_LAUNCH if args.count_log2 == 36 else None,
                "traffic_unit": "bytes per launch (ncu DRAM read + write)",
                "peak_note": ("derived: 152 SMs x 128 lanes x 2.07 GHz (one warp instruction per "
                              "scheduler per clock; issue ceiling, of derived); the measured rates below "
                              "(lane-ops per SM per clock) reach 128 for 32-bit add and FP32 FMA, 64 for "
                              "logic and integer multiply-add"),
                "measured_pipe_rates": pipe_rates,
                "half_steps_per_line": stats["half_steps"] / max(1, stats["lines"]),
                "filter_fail_per_line": stats["filter_fail"] / max(1, stats["lines"]),
                "frac_method": (stats["lines"] * ops_per_line(job) + stats["half_steps"] * METHOD_OPS_PER_HALF_STEP)
                / (statistics.mean(batched_ms) / 1e3) / ISSUE_PEAK_OPS,
                "frac_method_note": ("useful-work fraction: 6 operations per half-step (two 64-bit divisions, two "
                                     "multiply-subtracts, two adds/compares: the method's count) instead of the "
                                     "cost model's 35")}

    # the dense twin of the same slice (m = 20: about 1.3e5 records), batched
    # the same way: the exact resolution and compaction at scale
    twin = None
    if args.twins:
        tjob = job.replace(m=20)
        d_cand_t, d_count_t = tmd.alloc_candidates(1 << 18, local_rank)
        tmd.tmd_autotune(ctx, [tjob])
        tb = tmd.Batch(ctx, [tjob], d_cand_t, d_count_t)
        t_ms = max_over_ranks(statistics.mean(timed(tb.launch, 10, 3)))
        tst = tb.stats()
        _, t_n = tmd.tmd_candidates(ctx, d_cand_t, d_count_t)
        twin = {"m": 20, "value": total_args / (t_ms / 1e3), "ms_per_step": t_ms, "candidates": t_n,
                "roofline": roofline_of(tmd, [tjob], tst, t_ms),
                "form": "batched, autotuned tiling; flagged lines resolved exactly and compacted"}
        tb.close()

    # Lefevre's filter (Algorithm 3) on the same slice, batched the same way
    # (Table 4's comparison of the two searches; identical records)
    lefevre = None
    if args.lefevre:
        ljob = job.replace(flags=job.flags | wl.FLAG_LEFEVRE)
        d_cand_l, d_count_l = tmd.alloc_candidates(cap, local_rank)
        ltune = tmd.tmd_autotune(ctx, [ljob])
        lbatch = tmd.Batch(ctx, [ljob], d_cand_l, d_count_l)
        lef_ms = max_over_ranks(statistics.mean(timed(lbatch.launch, max(args.steps // 4, 5), args.warmup)))
        lst = lbatch.stats()
        lrecs = tmd.tmd_candidates(ctx, d_cand_l, d_count_l)
        assert lrecs == (recs, count), "the two filters must give the same records"
        lefevre = {"value": total_args / (lef_ms / 1e3), "ms_per_step": lef_ms,
                   "regular_over_lefevre_time": lef_ms / ms,
                   "iterations_per_line": lst["half_steps"] / max(1, lst["lines"]),
                   "filter_fail_per_line": lst["filter_fail"] / max(1, lst["lines"]),
                   "tiling": {k: ltune[k] for k in ("nu", "ctas_per_sm", "lanes", "unroll")},
                   "form": "batched, Lefevre's lower bound (Algorithm 3) as the filter"}
        lbatch.close()

    # sound mode on Table 2's domain: exp on [1, 1+2^-13[ (2^39 binary64
    # arguments), directed (53, 2^-32) cases: filter at eps1, exhaustive
    # phase at eps3 (Sect. II-A / III-A), one batched launch
    sound_run = None
    if args.sound:
        sjob = tmd.sound_job(wl.Job(wl.FUNC_EXP, 1, 53, 32, 15, 3, 24, 3, 0, 1 << 39, wl.FLAG_BP_DIRECTED))
        d_cand_s, d_count_s = tmd.alloc_candidates(1 << 16, local_rank)
        sb = tmd.Batch(ctx, [sjob], d_cand_s, d_count_s)
        s_ms = max_over_ranks(statistics.mean(timed(sb.launch, 10, 3)))
        sst = sb.stats()
        _, s_count = tmd.tmd_candidates(ctx, d_cand_s, d_count_s)
        sound_run = {"workload": "exp binary64 [1, 1+2^-13[ (2^39 args), directed (53, 2^-32) cases, "
                                 "d=3, W=192, N=2^15", "value": sjob.count / (s_ms / 1e3), "unit": UNIT,
                     "ms_per_step": s_ms, "listed_arguments": s_count,
                     "eps1_log2": math.log2(sjob.eps1) - 64, "eps3_log2": math.log2(sjob.eps3) - 64,
                     "filter_fail_per_line": sst["filter_fail"] / max(1, sst["lines"]),
                     "phase3_args": sst["refined_args"], "one_by_one_args": sst["exhaustive_args"],
                     "form": "batched: filter at eps1, exact line minimum, 32 refined pieces per failing "
                             "line at eps2 (phase 2); phase 3 on the failing pieces: 32 sub-pieces each "
                             "tested against their own half-width, Horner at every argument of the failing ones"}
        recs_s = tmd.tmd_candidates(ctx, d_cand_s, d_count_s)
        sb.close()
        # the same job with Lefevre's filter (Table 6's comparison of the two
        # searches' phase shares on a binade where exp is nearly linear)
        sjl = sjob.replace(flags=sjob.flags | wl.FLAG_LEFEVRE)
        sbl = tmd.Batch(ctx, [sjl], d_cand_s, d_count_s)
        sl_ms = max_over_ranks(statistics.mean(timed(sbl.launch, 10, 3)))
        stl = sbl.stats()
        assert tmd.tmd_candidates(ctx, d_cand_s, d_count_s) == recs_s, "the two filters must give the same records"
        sbl.close()
        sound_run["lefevre"] = {"value": sjob.count / (sl_ms / 1e3), "ms_per_step": sl_ms,
                                "filter_fail_per_line": stl["filter_fail"] / max(1, stl["lines"]),
                                "phase3_args": stl["refined_args"], "one_by_one_args": stl["exhaustive_args"]}

    # Table 7's second binade: exp on [128, 256), where the degree-1 lines'
    # truncation error is far above eps: a 2^36-argument slice at a seeded
    # block-aligned start, sound (53, 2^-32) cases with N = 2^16, the
    # regular and Lefevre's filter; the phases' argument counts are the
    # table's rows (phase 2 = lines failing the first filter times N)
    binade128 = None
    if args.binade128:
        import random
        bstart = random.Random(128256).randrange(0, (1 << 52) - (1 << 36), 1 << 20)
        bjob = wl.Job(wl.FUNC_EXP, 8, 53, 32, 16, 3, 20, 3, bstart, 1 << args.binade128_log2)
        binade128 = {"workload": f"exp binary64 [128, 256), 2^{args.binade128_log2}-arg slice at Random(128256) "
                                 "block-aligned start, sound (53, 2^-32) cases, d=3, W=192, N=2^16, T=2^20",
                     "start": bstart, "unit": UNIT}
        d_cand_b, d_count_b = tmd.alloc_candidates(1 << 16, local_rank)
        recs_b = None
        for name, flags in (("regular", 0), ("lefevre", wl.FLAG_LEFEVRE)):
            sj = tmd.sound_job(bjob.replace(flags=bjob.flags | flags))
            bb = tmd.Batch(ctx, [sj], d_cand_b, d_count_b)
            b_ms = max_over_ranks(statistics.mean(timed(bb.launch, 10, 3)))
            bst = bb.stats()
            got_b = tmd.tmd_candidates(ctx, d_cand_b, d_count_b)
            if recs_b is None:
                recs_b = got_b
            assert got_b == recs_b, "the two filters must give the same records"
            nl = max(1, bst["lines"])
            binade128[name] = {"value": sj.count / (b_ms / 1e3), "ms_per_step": b_ms,
                               "phase1_args": sj.count,
                               "phase2_args": bst["filter_fail"] << sj.log2_N,
                               "phase3_args": bst["refined_args"],
                               "one_by_one_args": bst["exhaustive_args"],
                               "phase2_fraction": bst["filter_fail"] / nl,
                               "phase3_fraction": bst["refined_args"] / sj.count,
                               "eps1_log2": math.log2(sj.eps1) - 64, "eps3_log2": math.log2(sj.eps3) - 64}
            bb.close()
        binade128["listed_arguments"] = recs_b[1]
        binade128["form"] = ("batched: filter at eps1, exact line minimum, 32 refined pieces per failing line "
                             "at eps2 (phase 2); phase 3 on the failing pieces: 32 sub-pieces each tested "
                             "against their own half-width, Horner at every argument of the failing ones")

    # Table 4's workload: the whole binade [1, 2) of exp, 2^52 binary64
    # arguments, sound (53, 2^-32) directed cases (Table 2's parameters), as
    # 1024 calls of the public API on 2^42-argument slices: host job record
    # in, plan, correctly rounded tables and fused search on the device,
    # host records out, every call (wall clock around the whole loop)
    binade_full = None
    if args.binade_full and world == 1:
        try:
            d_cand_f, d_count_f = tmd.alloc_candidates(1 << 16, local_rank)
            chunk_log2 = 42
            n_chunks = min(args.binade_full_chunks, 1 << (52 - chunk_log2))
            listed = 0
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for c in range(n_chunks):
                fj = tmd.sound_job(wl.Job(wl.FUNC_EXP, 1, 53, 32, 15, 3, 24, 3, c << chunk_log2,
                                          1 << chunk_log2, wl.FLAG_BP_DIRECTED))
                tmd.tmd_search(ctx, [fj], None, d_cand_f, d_count_f)
                _, nf = tmd.tmd_candidates(ctx, d_cand_f, d_count_f)
                listed += nf
            secs = time.perf_counter() - t0
            args_done = n_chunks << chunk_log2
            binade_full = {"workload": f"exp binary64 [1, 2), {n_chunks} x 2^{chunk_log2} arguments "
                                       f"({'the whole binade' if args_done == 1 << 52 else 'part of the binade'}), "
                                       "sound (53, 2^-32) directed cases, d=3, W=192, N=2^15",
                           "value": args_done / secs, "unit": UNIT, "seconds": secs,
                           "listed_arguments": listed,
                           "form": "one tmd_search + tmd_candidates call per slice from host job records "
                                   "(plan, tables, fused search, records back), wall clock"}
        except Exception as e:  # report, do not lose the rest of the line
            binade_full = {"error": repr(e)}

    mixed = None
    if args.mixed_jobs > 0:
        mjobs = wl.batched_jobs(njobs=args.mixed_jobs)
        margs = sum(j.count for j in mjobs)
        dmc, dmn = tmd.alloc_candidates(cap, local_rank)
        mtuned = tmd.tmd_autotune(ctx, mjobs)
        t0 = time.perf_counter()
        mb = tmd.Batch(ctx, mjobs, dmc, dmn)
        t_plan = time.perf_counter() - t0
        singles = [tmd.Batch(ctx, [j], dmc, dmn) for j in mjobs]
        ms_b = statistics.mean(timed(mb.launch, 10, 3))
        st_b = mb.stats()
        roof_b = roofline_of(tmd, mjobs, st_b, ms_b)

        def per_job():
            for sb in singles:
                sb.launch()
        ms_p = statistics.mean(timed(per_job, 5, 2))
        mixed = {"jobs": len(mjobs), "args": margs, "lines": st_b["lines"],
                 "batched": {"value": margs / (ms_b / 1e3), "ms_per_step": ms_b,
                             "form": "one persistent graph launch over all jobs",
                             "tiling": {k: mtuned[k] for k in ("nu", "ctas_per_sm", "lanes", "unroll")},
                             "roofline": roof_b},
                 "plain": {"value": margs / (ms_p / 1e3), "ms_per_step": ms_p,
                           "form": "one launch per job, plans resident",
                           "roofline": roofline_of(tmd, mjobs, st_b, ms_p)},
                 "plan_and_tables_s": t_plan}
        for sb in singles:
            sb.close()
        mb.close()
        if args.twins:
            tj = [j.replace(m=20) for j in mjobs]
            tmd.tmd_autotune(ctx, tj)
            dtc, dtn = tmd.alloc_candidates(1 << 20, local_rank)
            tb = tmd.Batch(ctx, tj, dtc, dtn)
            t_ms = statistics.mean(timed(tb.launch, 10, 3))
            tst = tb.stats()
            _, t_n = tmd.tmd_candidates(ctx, dtc, dtn)
            mixed["twin"] = {"m": 20, "value": margs / (t_ms / 1e3), "ms_per_step": t_ms, "candidates": t_n,
                             "roofline": roofline_of(tmd, tj, tst, t_ms)}
            tb.close()

    large = None
    if args.large:
        ljobs = wl.large_jobs()
        largs = sum(j.count for j in ljobs)
        dlc, dln = tmd.alloc_candidates(cap, local_rank)
        ltuned = tmd.tmd_autotune(ctx, ljobs)
        t0 = time.perf_counter()
        lb = tmd.Batch(ctx, ljobs, dlc, dln)
        t_plan = time.perf_counter() - t0
        ms_l = statistics.mean(timed(lb.launch, 5, 3))
        st_l = lb.stats()
        _, n_l = tmd.tmd_candidates(ctx, dlc, dln)
        large = {"jobs": len(ljobs), "args": largs, "lines": st_l["lines"], "candidates": n_l,
                 "batched": {"value": largs / (ms_l / 1e3), "ms_per_step": ms_l,
                             "form": "one persistent graph launch over all 2^16 jobs",
                             "tiling": {k: ltuned[k] for k in ("nu", "ctas_per_sm", "lanes", "unroll")},
                             "roofline": roofline_of(tmd, ljobs, st_l, ms_l)},
                 "plan_and_tables_s": t_plan, "upload_bytes": lb.upload_bytes}
        lb.close()
        if args.twins:
            tj = [j.replace(m=22) for j in ljobs]
            tmd.tmd_autotune(ctx, tj)
            dtc, dtn = tmd.alloc_candidates(1 << 20, local_rank)
            tb = tmd.Batch(ctx, tj, dtc, dtn)
            t_ms = statistics.mean(timed(tb.launch, 5, 3))
            tst = tb.stats()
            _, t_n = tmd.tmd_candidates(ctx, dtc, dtn)
            large["twin"] = {"m": 22, "value": largs / (t_ms / 1e3), "ms_per_step": t_ms, "candidates": t_n,
                             "roofline": roofline_of(tmd, tj, tst, t_ms)}
            tb.close()

    serving = None
    if rank == 0 and args.serve_jobs > 0:
        sjobs = wl.serving_jobs()[: args.serve_jobs]
        sargs = sum(j.count for j in sjobs)
        mean_size = sargs / len(sjobs)
        w_sat, lat_sat, a_sat, _, st_sat = run_serving(tmd, ctx, sjobs, float("inf"))
        sat = a_sat / w_sat
        rate = 0.8 * sat / mean_size
        reps = []
        for rep in range(3):
            w, lat, a, nrec, st = run_serving(tmd, ctx, sjobs, rate)
            reps.append({"p50_ms": 1e3 * percentile(lat, 0.50), "p99_ms": 1e3 * percentile(lat, 0.99),
                         "args_per_s": a / w, "seconds": w, "records": nrec, "groups": st["groups"]})
        # the same jobs as one batch (one persistent graph launch, plans and
        # tables resident): the ceiling of the served form
        dsc, dsn = tmd.alloc_candidates(1 << 18, local_rank)
        sb = tmd.Batch(ctx, sjobs, dsc, dsn)
        sb_ms = statistics.mean(timed(sb.launch, 3, 3))
        sbst = sb.stats()
        sb.close()
        roof_sat = roofline_of(tmd, sjobs, st_sat, 1e3 * w_sat)
        serving = {"jobs": len(sjobs), "arrival_rate_jobs_per_s": rate, "mean_job_args": mean_size,
                   "p50_ms": statistics.median(r["p50_ms"] for r in reps),
                   "p99_ms": statistics.median(r["p99_ms"] for r in reps),
                   "args_per_s": statistics.median(r["args_per_s"] for r in reps),
                   "repeats": reps,
                   "saturated_args_per_s": sat, "saturated_seconds": w_sat, "saturated_groups": st_sat["groups"],
                   "saturated_roofline": roof_sat,
                   "batched_same_jobs": {"value": sargs / (sb_ms / 1e3), "ms_per_step": sb_ms,
                                         "roofline": roofline_of(tmd, sjobs, sbst, sb_ms)},
                   "records": reps[0]["records"],
                   "form": ("continuous batching: arrived jobs admitted up to 1024 per group into 4 slots "
                            "(plan, tables, one fused launch per kernel class per group); Poisson arrivals "
                            "at 0.8 x the saturated rate replayed by the server clock; 3 repeats"),
                   "latency": "t_done - t_submit per job (arrival to results ready on the host)"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        a, dt, nb, th = oracle_sample(job, seconds_target=args.ref_seconds)
        cpu = {"value": a / dt, "unit": UNIT, "cores": th, "kind": "oracle",
               "sample": f"first {nb} Taylor blocks (2^24 args each) of the slice, {dt:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": f"exp binary64 [1/2,1) 2^{args.count_log2}-arg slice per GPU, "
                                   f"d=3, W=192, N=2^14, m={args.m}",
                       "l2": "256 MiB flush before every step",
                       "form": "batched: persistent work-queue kernel replayed as a CUDA graph",
                       "tiling": {"nu": tuned["nu"], "ctas_per_sm": tuned["ctas_per_sm"],
                                  "lanes": tuned.get("lanes", 1), "unroll": tuned.get("unroll", 1),
                                  "picked_by": ("tmd_autotune (4 replays per candidate, the three fastest again with 16)"
                                                if args.tiling == "auto" else "--tiling")},
                       "candidates": count},
            "plain": {"value": fused_value, "ms_per_step": ms_fused,
                      "form": "per-job fused launch (tmd_search)"},
            "unfused": {"value": plain_value, "ms_per_step": ms_plain,
                        "form": "generate lines to HBM, then search them (two launches)"},
            "e2e": {"value": total_args / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_s * 1e3},
            "gpu_launches": args.steps * 1,
            "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks, "dense_twin": twin, "lefevre": lefevre,
            "sound_table2": sound_run,
            "binade_128_256": binade128,
            "binade_1_2_whole": binade_full,
            "mixed_batch": mixed,
            "large_batch": large,
            "serving": serving,
        }
        print(json.dumps(line), flush=True)
    batch.close()
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
