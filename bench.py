#!/usr/bin/env python
"""Benchmark of the profile-likelihood hot path on B300.

Metric: profile log-likelihood evaluations per second at n = 4000 (one
evaluation = one correlation-parameter point omega, its n x n Matern matrix
built, factored and solved against 9 Box-Cox columns + 3 covariates, giving
l_p at all 9 lambdas), with p50/p99 latency of end-to-end steps.

Workload ("mixed4000"): n = 4000 sites uniform on [0,20]^2, p = 3, M = 9
lambdas in [-0.5, 1.5], K = 1024 omega (960 Halton points of the parameter box
+ 64 ill-conditioned points).  A step is one batch of `--batch` points of that
grid (cycling through it) through the whole path: Box-Cox rows, build,
blocked Cholesky with the bordered right-hand side, closed form.  Inputs are
synthetic (paper_2305_04318_b300.synth), resident in HBM when the timed region
starts; each step's tile workspace is several GB, far larger than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
  python bench.py --impl reference      # the FP64 CPU oracle on the host cores

Under torchrun (N > 1) every rank evaluates its own slice of points (weak
scaling, no data-path collective); the step time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

# DRAM traffic model of the dominant mixed-path kernel, k_trail_pipe<5> (the
# 5-slice trailing update), per kind of launch, in bytes per work item (a
# half tile for the data rows, a whole tile for the right-hand-side row, over
# all points of the part): the data triangle (four panels per item; each operand image is
# re-read by many items, mostly from L2), one tile column's data rows (the
# group's earlier panels: every item reads its own operand images, so they
# come from DRAM: a term per item and panel) and the right-hand-side row (its
# epilogue moves only M + p rows).  Fitted by least squares to
# dram__bytes_read.sum + dram__bytes_write.sum of every k_trail_pipe<5> launch
# in one ncu capture (a one-pass metric set) of the small case
# `python bench.py --precision mixed --n 2000 --batch 148 --steps 1 --warmup 1
# --no-cpu-baseline --no-e2e`, then evaluated on the bench's own launches (the
# full-size workload exceeds the capture-size rule).  Points that the early
# verdict stops skip their items, so at full size this is an upper bound.
# Valid for the kernel source it was taken on (SHA-256 below), else traffic is
# null.
TRAIL_TRAFFIC = {"tri_item": 184226.6, "col_item": 115869.1, "col_item_panel": 84528.1, "rhs_item": 191195.1,
                 "fit_rel_rms": 0.081,
                 "sources_sha256": "64e808de636ca4a592c060a2fc52f9cd2a5a26704e425e440f6342611c489c63"}

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "profile-logL evals/s at n=4000 (FP64 vs mixed, |ΔlogL|≤1e-3); p50/p99 latency"
UNIT = "evals/s"
# arithmetic the path computes in: FP64 mode is FP64 throughout; mixed mode
# splits the trailing updates and panel solves into exact bf16 slice products
# on the tensor cores (FP32 accumulation), keeps the trailing matrix, the
# first-pass build and the diagonal tiles in double-float FP32 (two floats per
# value), and the log-determinant and closed form in FP64
DTYPE = {"fp64": "f64", "mixed": "bf16 split products (5/7 slices) + f32 pairs + f64"}
WORKLOAD = ("mixed4000: n=4000 sites on [0,20]^2, p=3, M=9 lambdas in [-0.5,1.5], "
            "K=1024 omega (960 Halton + 64 ill-conditioned), anisotropic Matern")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", "fp64", "mixed"])
    ap.add_argument("--batch", type=int, default=0, help="omega points per step (default: 1776 = 12 x 148 mixed, 128 fp64)")
    ap.add_argument("--n", type=int, default=4000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=0, help="oracle points in the CPU sample (default: cores)")
    ap.add_argument("--workload", default="mixed4000", choices=["mixed4000", "uneven", "serving", "pipeline", "iso100", "aniso1000"],
                    help="mixed4000: the metric's n=4000 workload (default); uneven: 256 datasets of "
                         "n in [200,3000] x 512 points through the job scheduler; serving: Poisson "
                         "stream of profile jobs over a pool of resident datasets; pipeline: Steps 1-6 of "
                         "the method on one dataset (MLE, representative points, evaluation, profiles); "
                         "iso100 / aniso1000: the two smaller configurations, both precisions against the oracle")
    ap.add_argument("--datasets", type=int, default=0, help="uneven/serving: number of datasets (default 256 / 32)")
    ap.add_argument("--points", type=int, default=512, help="uneven: points per dataset")
    ap.add_argument("--item-batch", type=int, default=0,
                    help="uneven: points per scheduled batch (default 0: chosen by the autotuner per dataset size)")
    ap.add_argument("--jobs", type=int, default=40, help="serving: jobs per load level")
    ap.add_argument("--job-grid", type=int, default=16,
                    help="serving: grid values of the profiled parameter (the full job: 64)")
    ap.add_argument("--job-sub", type=int, default=2,
                    help="serving: sub-grid values of each other parameter (the full job: 4)")
    ap.add_argument("--serve-batch", type=int, default=16, help="serving: points per scheduled batch")
    ap.add_argument("--capacity-jobs", type=int, default=6, help="serving: jobs run one after another for the capacity")
    ap.add_argument("--level-seconds", type=float, default=0.0,
                    help="serving: run each load level for this long (arrivals stop then, the jobs in flight finish) "
                         "instead of a fixed number of jobs")
    ap.add_argument("--streams", type=int, default=4, help="uneven/serving: scheduler streams")
    ap.add_argument("--policy", default="largest", choices=["fifo", "largest"],
                    help="uneven: which job a free scheduler stream serves next (largest dataset first, or oldest)")
    ap.add_argument("--graph", type=int, default=0,
                    help="uneven, iso100, aniso1000: launch batches as CUDA graphs (1) or eagerly (0, default)")
    ap.add_argument("--pipe-counters", action="store_true",
                    help="diagnostic: one mixed step of the n=4000 workload through the library built with the "
                         "trailing update's wait-cycle counters (libplk_counters.so); prints their breakdown")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the raw samples go to PLK_CLOCKS_DIR (default: the system temp folder);
        # the JSON line carries their summary
        d = os.environ.get("PLK_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"clocks_rank_gpu{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path))
    except Exception:
        return {}


def probe_fp64_peak():
    """Live FP64 FMA-pipe throughput (TFLOP/s) on this GPU."""
    import ctypes as C
    from paper_2305_04318_b300 import build
    L = C.CDLL(build.build_probe())
    L.plk_probe_fp64_fma_tflops.restype = C.c_double
    L.plk_probe_fp32_fma_tflops.restype = C.c_double
    return L.plk_probe_fp64_fma_tflops(5), L.plk_probe_fp32_fma_tflops(5)


def probe_pipes():
    """Live throughputs (TFLOP/s) of the pipes the design chooses between:
    FP64 FMA (DFMA), FP64 tensor MMA (DMMA, mma.sync m8n8k4), FP32 FMA, and
    tcgen05 bf16 MMA with both operands in shared memory at N = 64, 128, 256."""
    import ctypes as C
    from paper_2305_04318_b300 import build
    L = C.CDLL(build.build_probe())
    for f in ("plk_probe_fp64_fma_tflops", "plk_probe_fp32_fma_tflops", "plk_probe_fp64_mma_tflops",
              "plk_probe_tcgen05_bf16_tflops"):
        getattr(L, f).restype = C.c_double
    L.plk_probe_tcgen05_bf16_tflops.argtypes = [C.c_int, C.c_int]
    out = {"fp64_fma": L.plk_probe_fp64_fma_tflops(5), "fp64_dmma": L.plk_probe_fp64_mma_tflops(5),
           "fp32_fma": L.plk_probe_fp32_fma_tflops(5)}
    for N in (64, 128, 256):
        out[f"tcgen05_bf16_n{N}"] = L.plk_probe_tcgen05_bf16_tflops(N, 5)
    return {k: round(v, 2) for k, v in out.items()}


def probe_fp64_lanes():
    """SM cycles per FP64 FMA warp instruction of a dependent chain, for 1 and
    4 warps in one block and 1 or 32 active lanes: whether FP64 issue cost
    depends on the active lanes (it decides how FP64 work is laid out)."""
    import ctypes as C
    from paper_2305_04318_b300 import build
    L = C.CDLL(build.build_probe())
    f = L.plk_probe_fp64_cycles_per_warp_fma
    f.restype, f.argtypes = C.c_double, [C.c_int, C.c_int]
    return {f"warps{w}_lanes{a}": round(f(w, a), 2) for w in (1, 4) for a in (1, 32)}


def trailing_flops(n, q, TB=128):
    """Algorithmic flops of the trailing updates, per omega, per step J of the
    blocked factorisation: the rank-TB update of the lower triangle of the true
    (unpadded) r x r trailing matrix (TB r^2) plus the q right-hand-side rows
    (2 TB q r).  Summed over J this is n^3/3 + n^2 q to leading order."""
    nb = -(-n // TB)
    out = []
    for J in range(nb):
        r = max(0, n - (J + 1) * TB)
        out.append(TB * r * r + 2 * TB * q * r)
    return out


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle
# ---------------------------------------------------------------------------

def oracle_rate(ds, P, lambdas, npts, threads, full=False):
    import oracle
    t0 = time.perf_counter()
    r = oracle.profile_batch(ds.coords, ds.y, ds.X, P[:npts], lambdas, nthreads=threads)
    dt = time.perf_counter() - t0
    return (npts / dt, dt, r["threads"], r) if full else (npts / dt, dt, r["threads"])


def oracle_sample_indices(K, npts, n_ill=64):
    """Points of the n=4000 grid in the CPU-baseline sample: the first Halton
    points and, for a quarter of the sample, ill-conditioned points of the
    grid's last 64 (kappa = 8, phi_X = 40, all four nuggets, both ratios), so
    that the per-result errors cover them."""
    k_ill = min(npts // 4, n_ill)
    ill_pick = [56, 58, 61, 63, 48, 50, 53, 55, 40, 42, 45, 47, 32, 34, 37, 39][:k_ill]
    return np.array(list(range(npts - k_ill)) + [K - n_ill + i for i in ill_pick])


def per_result_errors(g, o, lam, prefix=""):
    """Largest errors of GPU results g against the oracle's o on the same points:
    |Delta l_p| (abs), sigma^2 (rel), beta (abs, relative to the largest |beta|),
    log|V| and log|X'V^-1X| (abs), the status agreement, and the 95 % likelihood
    CI of lambda from the profile over these points (endpoint error relative to
    the oracle CI's width)."""
    import oracle
    st = g["status"] & 15
    ok = (st == 0) & (o["status"] == 0)
    r = {"points": int(len(st)), "compared": int(ok.sum()), "status_agree": int((st == o["status"]).sum())}
    if ok.any():
        d = np.abs(g["logL"][ok] - o["logL"][ok])
        r["max_abs_dlogL"] = float(d.max())
        r["max_rel_dlogL"] = float((d / np.abs(o["logL"][ok])).max())
        r["max_rel_dsigma2"] = float(np.abs(g["sigma2"][ok] / o["sigma2"][ok] - 1).max())
        r["max_dbeta_rel_to_max_beta"] = float(np.abs(g["beta"][ok] - o["beta"][ok]).max() / np.abs(o["beta"][ok]).max())
        r["max_abs_dlogdet"] = float(np.abs(g["logdet"][ok] - o["logdet"][ok]).max())
        from paper_2305_04318_b300 import native as nv
        gp = np.nanmax(np.where(ok[:, None], g["logL"], np.nan), axis=0)
        op = oracle.profile_max(np.where(ok[:, None], o["logL"], np.nan).T)
        gci, oci = nv.profile_ci(lam, gp, 0.95), oracle.profile_ci(lam, op, 0.95)
        width = oci["hi"] - oci["lo"]
        if width > 0:
            r["lambda_ci95_oracle"] = [oci["lo"], oci["hi"]]
            r["max_ci_endpoint_err_rel_to_width"] = float(max(abs(gci["lo"] - oci["lo"]), abs(gci["hi"] - oci["hi"])) / width)
    return r


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2305_04318_b300 import synth
    w = synth.mixed4000(n=args.n)
    ds, P, lam = w.datasets[0], w.params[0], w.lambdas
    cores = cpu_cores()
    npts = args.cpu_sample or cores
    for s in range(args.warmup):   # untimed warm-up steps (same sample size)
        idx = (np.arange(npts) + (args.steps + s) * npts) % P.shape[0]
        oracle_rate(ds, P[idx], lam, npts, cores)
    rates, times = [], []
    for s in range(args.steps):
        idx = (np.arange(npts) + s * npts) % P.shape[0]
        r, dt, used = oracle_rate(ds, P[idx], lam, npts, cores)
        rates.append(r)
        times.append(dt)
    value = npts * len(times) / sum(times)
    sample = f"{npts} omega points per step of the n=4000 workload, one per thread"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "precision": "fp64", "device": "cpu"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_uneven(args):
    """Config 4: 256 datasets with n log-uniform in [200, 3000] and p in {2,3,5},
    512 points each, all submitted at once to one context; the scheduler
    interleaves their batches over the stream pool (continuous batching).  The
    points per batch come from the library's autotuner (plk_autotune), run once
    per half-octave of n before the timed region, unless --item-batch is set.
    Under torchrun every rank takes whole datasets, balanced by points x n^3
    (shard.balance_by_cost); the time is the max over ranks."""
    import torch
    import torch.distributed as dist
    from paper_2305_04318_b300 import native as nv, shard, synth
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    D = args.datasets or 256
    w = synth.uneven(D=D, per=args.points)
    owner = shard.balance_by_cost([len(P) * float(d.n) ** 3 for d, P in zip(w.datasets, w.params)], world)
    mine = [i for i in range(D) if owner[i] == rank]
    prec = nv.MIXED if args.precision in ("auto", "mixed") else nv.FP64
    M = len(w.lambdas)
    free, _ = torch.cuda.mem_get_info()
    arena_bytes = int(min(free - (8 << 30), 200e9))
    arena = torch.empty((arena_bytes,), dtype=torch.uint8, device="cuda")
    tune = {}

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    with nv.Context(arena_bytes, device=local, arena=arena, n_streams=args.streams) as ctx:
        ctx.set_schedule_policy(nv.SCHED_LARGEST_FIRST if args.policy == "largest" else nv.SCHED_FIFO)
        t_tune = time.perf_counter()
        if args.item_batch <= 0:
            buckets = sorted({int(round(2 * math.log2(w.datasets[i].n))) for i in mine})
            for b in buckets:
                n_rep = int(round(2 ** (b / 2)))
                bb, rate = ctx.autotune(n_rep, 3, M, prec)
                tune[str(n_rep)] = {"batch": bb, "points_per_s": round(rate, 1)}
        t_tune = time.perf_counter() - t_tune
        ids = {i: ctx.create_dataset(w.datasets[i].coords, w.datasets[i].y, w.datasets[i].X) for i in mine}
        # warm-up: one small job
        if mine:
            j = ctx.submit(ids[mine[0]], w.params[mine[0]][:4], w.lambdas, precision=prec, batch=4)
            ctx.poll(j, w.datasets[mine[0]].p)
        barrier()
        t0 = time.perf_counter()
        gflag = nv.FLAG_GRAPH if args.graph else 0
        jobs = {i: ctx.submit(ids[i], w.params[i], w.lambdas, precision=prec, batch=max(0, args.item_batch),
                              flags=gflag) for i in mine}
        res = [ctx.poll(jobs[i], w.datasets[i].p) for i in mine]
        dt = time.perf_counter() - t0
        barrier()
        _, high = ctx.memory_stats()
    if world > 1:
        t = torch.tensor([dt], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dt = float(t.item())
    npts = sum(len(P) for P in w.params)
    st = np.concatenate([r["status"] for r in res]) if res else np.zeros(0, dtype=np.int32)
    ns = np.array([d.n for d in w.datasets])
    line = {"metric": "profile-logL evals/s, batched uneven datasets", "value": npts / dt, "unit": UNIT,
            "n_gpus": world, "steps": 1, "warmup": 1, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": DTYPE["mixed" if prec == nv.MIXED else "fp64"],
            "data": "synthetic",
            "config": {"workload": f"uneven: {D} datasets, n log-uniform in [200,3000] (median {int(np.median(ns))}), "
                                   f"p in {{2,3,5}}, {args.points} points each, 9 lambdas",
                       "precision": "mixed" if prec == nv.MIXED else "fp64", "streams": args.streams,
                       "mixed_tolerance": nv.get_mixed_tolerance(),
                       "batch_per_item": args.item_batch if args.item_batch > 0 else "autotuned",
                       "cuda_graphs": bool(args.graph), "arena_gb": arena_bytes / 1e9,
                       "schedule_policy": args.policy,
                       "parallelism": f"datasets balanced by points x n^3 over {world} rank(s)"},
            "autotune": {"seconds": round(t_tune, 2), "by_n": tune,
                         "what": "plk_autotune per half-octave of n, before the timed region (rank 0's)"},
            "points": int(npts), "points_not_ok_rank0": int(((st & 15) != 0).sum()),
            "points_7slice_rank0": int(((st & 16) != 0).sum()), "points_fp64_rank0": int(((st & 32) != 0).sum()),
            "hbm_high_water_gb": high / 1e9, "e2e": {"value": npts / dt, "unit": UNIT,
            "h2d_bytes_per_step": int(sum(P.nbytes for P in w.params)), "d2h_bytes_per_step": int(
                sum(r["logL"].nbytes + r["sigma2"].nbytes + r["beta"].nbytes + r["logdet"].nbytes + r["status"].nbytes
                    for r in res) * world)}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_serving(args):
    """Config 5: a Poisson stream of profile jobs over a pool of device-resident
    datasets (n log-uniform in [500, 8000]).  A job profiles one parameter:
    G grid values x sub^4 values of the other four x 9 lambdas, then the
    profile maximum and the likelihood CI on the device.  Jobs arrive at an
    offered load of 0.5 and 0.9 of the measured single-stream capacity."""
    import torch
    from paper_2305_04318_b300 import native as nv, synth
    D = args.datasets or 32
    G, sub = args.job_grid, args.job_sub   # default 16 x 2^4 (the full job, 64 x 4^4, takes ~25 s each)
    pool = synth.serving_pool(D=D)
    lam = synth.LAMBDA_GRID_9
    prec = nv.MIXED if args.precision in ("auto", "mixed") else nv.FP64
    rng = np.random.default_rng(55)
    grids = [synth.profile_job_grid(which, G=G, sub=sub) for which in range(5)]
    arena_bytes = int(args.streams * nv.workspace_bytes(8000, 3, 9, args.serve_batch, prec) * 1.1 + (4 << 30))
    arena = torch.empty((arena_bytes,), dtype=torch.uint8, device="cuda")
    results = {}
    with nv.Context(arena_bytes, arena=arena, n_streams=args.streams) as ctx:
        ids = [ctx.create_dataset(d.coords, d.y, d.X) for d in pool]

        def job_spec(k):
            return int(rng.integers(D)), k % 5

        def finish(job, ds_i, which):
            r = ctx.poll(job, 3)
            gv, _ = grids[which]
            vals = torch.as_tensor(r["logL"].reshape(G, -1), device="cuda")
            prof = nv.profile_max_device(vals)
            ci = nv.profile_ci_device(torch.as_tensor(gv, device="cuda"), prof, 0.95).cpu().numpy()
            return r, ci

        # capacity: jobs one after another
        t0 = time.perf_counter()
        cap_jobs = args.capacity_jobs
        for k in range(cap_jobs):
            d_i, which = job_spec(k)
            jb = ctx.submit(ids[d_i], grids[which][1], lam, precision=prec, batch=args.serve_batch)
            finish(jb, d_i, which)
        cap = cap_jobs / (time.perf_counter() - t0)
        levels = {}
        for rho in (0.5, 0.9):
            rate = rho * cap
            if args.level_seconds > 0:   # arrivals for level_seconds, then drain
                arr = np.cumsum(rng.exponential(1.0 / rate, size=int(rate * args.level_seconds * 3) + 10))
                arrivals = arr[arr <= args.level_seconds]
            else:
                arrivals = np.cumsum(rng.exponential(1.0 / rate, size=args.jobs))
            njobs = len(arrivals)
            lat = []
            pending = []
            t0 = time.perf_counter()
            k = 0
            done = 0
            while done < njobs:
                now = time.perf_counter() - t0
                while k < njobs and arrivals[k] <= now:
                    d_i, which = job_spec(k)
                    jb = ctx.submit(ids[d_i], grids[which][1], lam, precision=prec, batch=args.serve_batch)
                    pending.append((jb, d_i, which, t0 + arrivals[k]))
                    k += 1
                still = []
                for jb, d_i, which, ta in pending:
                    r = ctx.poll(jb, 3, timeout_ms=0)
                    if r is None:
                        still.append((jb, d_i, which, ta))
                        continue
                    gv, _ = grids[which]
                    prof = nv.profile_max_device(torch.as_tensor(r["logL"].reshape(G, -1), device="cuda"))
                    nv.profile_ci_device(torch.as_tensor(gv, device="cuda"), prof, 0.95).cpu()
                    lat.append(time.perf_counter() - ta)
                    done += 1
                pending = still
                time.sleep(0.001)
            span = time.perf_counter() - t0
            levels[str(rho)] = {"offered_jobs_per_s": rate, "jobs": njobs, "seconds": span,
                                "throughput_jobs_per_s": njobs / span, "evals_per_s": njobs * G * sub ** 4 / span,
                                "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                                "max_ms": 1e3 * float(np.max(lat))}
        _, high = ctx.memory_stats()
    top = levels["0.9"]
    line = {"metric": "profile jobs: throughput and p50/p99 job latency (serving)", "value": top["evals_per_s"],
            "unit": UNIT, "n_gpus": 1, "steps": top["jobs"], "warmup": cap_jobs, "ms_per_step": top["p50_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE["mixed" if prec == nv.MIXED else "fp64"], "data": "synthetic",
            "config": {"workload": f"serving: {D} resident datasets, n log-uniform in [500,8000], p=3; job = one "
                                   f"parameter's {G}-point profile x {sub}^4 sub-grid x 9 lambdas ({G * sub ** 4} omega), "
                                   "then profile max + 95% CI on the device; Poisson arrivals",
                       "precision": "mixed" if prec == nv.MIXED else "fp64", "streams": args.streams,
                       "mixed_tolerance": nv.get_mixed_tolerance(),
                       "batch_per_item": args.serve_batch},
            "capacity_jobs_per_s": cap, "levels": levels, "hbm_high_water_gb": high / 1e9,
            "latency_ms": {"p50": top["p50_ms"], "p99": top["p99_ms"], "what": "job latency at offered load 0.9"}}
    print(json.dumps(line), flush=True)


def run_pipeline(args):
    """Steps 1-6 of the method on one synthetic dataset shaped like the paper's
    rainfall example (n = 100 sites on the unit square, p = 2): Step 1 the MLE
    and two fits with kappa held at 0.5 and 10 (batched Newton iterations on the
    GPU), Step 2 the representative points (5-D cloud of 726 points x 11
    contour levels around the MLE, 4-D clouds of 120 x 11 around the two
    constrained fits) and 30 lambdas, Step 3 all of them on the GPU, Steps 4-6
    the profiles of lambda, of phi_X (upper hull of the cloud), of beta_1 and of
    sigma on the device.  Reports the time of every step."""
    import torch
    from paper_2305_04318_b300 import native as nv, synth
    n = args.n if args.n != 4000 else 100
    prec = nv.MIXED if args.precision == "mixed" else nv.FP64
    ds = synth.simulate_dataset(101, n, math.sqrt(n / 100.0), 2, beta=(1.0, 0.5), sigma=1.0, kappa=1.0, phi_x=0.2,
                                nug=0.1, phi_r=1.5, phi_a=0.5, lam=0.5, name="pipeline")
    dev = torch.device("cuda")
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)
    arena = torch.empty((16 << 30,), dtype=torch.uint8, device=dev)
    times = {}
    with nv.Context(arena.numel(), arena=arena, n_streams=2) as ctx:
        did = ctx.create_dataset(ds.coords, ds.y, ds.X)
        w0 = np.array([0.3, 1.0, 0.2, 1.2, 0.3])
        nv.fit_mle(ctx, did, w0, 0.3, precision=prec, max_iter=2)          # warm-up
        torch.cuda.synchronize()
        t = time.perf_counter()
        fit = nv.fit_mle(ctx, did, w0, 0.3, precision=prec)
        fits_k = [nv.fit_mle(ctx, did, w0, fit["lam"], precision=prec, kappa_fixed=True, kappa=k) for k in (0.5, 10.0)]
        times["step1_mle_s"] = time.perf_counter() - t
        t = time.perf_counter()
        c5 = nv.quadratic_cloud(ctx, did, fit["omega"], fit["lam"], precision=prec, n_lambda=30, seed=1)
        ck = [nv.quadratic_cloud(ctx, did, f["omega"], f["lam"], precision=prec, kappa_fixed=True, n_lambda=0, seed=2 + i)
              for i, f in enumerate(fits_k)]
        P = np.vstack([c5["params"]] + [c["params"] for c in ck])
        lam = c5["lambdas"]
        times["step2_points_s"] = time.perf_counter() - t
        ctx.release_dataset(did)
    del arena
    torch.cuda.synchronize()
    K, M = P.shape[0], len(lam)
    coords, y, X, lamd, Pd = T(ds.coords), T(ds.y), T(ds.X), T(lam), T(P)
    nv.eval_device(coords, y, X, lamd, Pd[:64], precision=prec, with_ssq=True)   # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out = nv.eval_device(coords, y, X, lamd, Pd, precision=prec, with_ssq=True)
    e1.record()
    torch.cuda.synchronize()
    times["step3_eval_s"] = e0.elapsed_time(e1) * 1e-3

    def profiles():
        lam_prof = nv.profile_lambda_device(out["logL"])
        lam_ci = nv.profile_ci_device(lamd, lam_prof, 0.95)
        best = nv.profile_max_device(out["logL"])                     # max over lambda per point
        ok = torch.isfinite(best)
        xq = T(np.exp(np.linspace(np.log(P[:, 0].min()), np.log(P[:, 0].max()), 64)))
        hull, _ = nv.profile_hull_device(Pd[:, 0][ok].contiguous(), best[ok].contiguous(), xq)
        phi_ci = nv.profile_ci_device(xq, hull, 0.95)
        bgrid = T(np.linspace(-1.0, 2.0, 64))
        bprof = nv.profile_beta_device(y, lamd, out["ssq_yx"], out["logdet"], out["status"], 1, bgrid)
        beta_ci = nv.profile_ci_device(bgrid, bprof, 0.95)
        sgrid = T(np.linspace(0.05, 3.0, 64))
        sprof = nv.profile_sigma_device(y, lamd, out["ssq_yx"], out["logdet"], out["status"], sgrid)
        sig_ci = nv.profile_ci_device(sgrid, sprof, 0.95)
        return {k: v.cpu().numpy()[:2].tolist() for k, v in
                dict(lambda_=lam_ci, phi_x=phi_ci, beta_1=beta_ci, sigma=sig_ci).items()}

    profiles()                                                  # warm-up (first use of these kernels)
    torch.cuda.synchronize()
    t = time.perf_counter()
    cis = profiles()
    torch.cuda.synchronize()
    times["steps4_6_profiles_s"] = time.perf_counter() - t
    st = out["status"].cpu().numpy()
    total = sum(times.values())
    line = {"metric": "profile-likelihood method, Steps 1-6 on one dataset", "value": K * M / times["step3_eval_s"],
            "unit": "(omega, lambda) evals/s in Step 3", "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": 1e3 * total, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE["mixed" if prec == nv.MIXED else "fp64"], "data": "synthetic",
            "config": {"workload": f"pipeline: n={n} sites on a square of side {math.sqrt(n / 100.0):.2f}, p=2, "
                                   "truth kappa=1, phi_X=0.2, nu^2=0.1, ratio 1.5, lambda 0.5",
                       "precision": "mixed" if prec == nv.MIXED else "fp64", "K": int(K), "M": int(M),
                       "mixed_tolerance": nv.get_mixed_tolerance()},
            "times_s": {k: round(v, 4) for k, v in times.items()},
            "mle": {"omega": fit["omega"].tolist(), "lambda": fit["lam"], "logL": fit["logL"],
                    "iterations": fit["iterations"],
                    "kappa_fixed": [{"kappa": k, "logL": f["logL"], "iterations": f["iterations"]}
                                    for k, f in zip((0.5, 10.0), fits_k)]},
            "ci95": cis, "points_not_ok": int(((st & 15) != 0).sum())}
    print(json.dumps(line), flush=True)


def run_small_config(args):
    """Configs 1-2: iso100 (n = 100, K = 100 grid points, lambda = 0) and
    aniso1000 (n = 1000, K = 4096 Halton points, 9 lambdas), all K points per
    step in FP64 and in mixed precision; the oracle on the host cores on all
    (iso100) or a sample (aniso1000) of the points, which also gives the
    largest relative |Delta l_p| of each precision."""
    import torch
    from paper_2305_04318_b300 import native as nv, synth
    import oracle
    w = synth.iso100() if args.workload == "iso100" else synth.aniso1000()
    ds, P, lam = w.datasets[0], w.params[0], w.lambdas
    K, n, M = P.shape[0], ds.n, len(lam)
    dev = torch.device("cuda")
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)
    coords, y, X, lamd, Pd = T(ds.coords), T(ds.y), T(ds.X), T(lam), T(P)
    cores = cpu_cores()
    sample = np.arange(K) if K <= 128 else np.linspace(0, K - 1, 4 * cores).astype(int)
    t0 = time.perf_counter()
    o = oracle.profile_batch(ds.coords, ds.y, ds.X, P[sample], lam, nthreads=cores)
    t_or = time.perf_counter() - t0
    peaks = measured_peaks()
    fp64_peak, _ = probe_fp64_peak()
    out = {}
    for name, prec in (("fp64", nv.FP64), ("mixed", nv.MIXED)):
        batch = min(K, 1184 if n <= 1500 else 296)
        wsb = nv.workspace_bytes(n, ds.p, M, batch, prec)
        ws = torch.empty((wsb,), dtype=torch.uint8, device=dev)
        gflag = nv.FLAG_GRAPH if args.graph else 0
        outs = nv.eval_device(coords, y, X, lamd, Pd, precision=prec, batch=batch, workspace=ws, flags=gflag)
        for _ in range(args.warmup):
            nv.eval_device(coords, y, X, lamd, Pd, precision=prec, batch=batch, workspace=ws, outputs=outs, flags=gflag)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            r = nv.eval_device(coords, y, X, lamd, Pd, precision=prec, batch=batch, workspace=ws, outputs=outs,
                               flags=gflag)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        # per-kernel-class times from one more step with event timing around every launch
        nv.kernel_timing(reset=True)
        nv.eval_device(coords, y, X, lamd, Pd, precision=prec, batch=batch, workspace=ws, flags=nv.FLAG_KERNEL_TIMING)
        torch.cuda.synchronize()
        tm = nv.kernel_timing(reset=True)
        g = {k: v.cpu().numpy() for k, v in r.items()}
        st = g["status"] & 15
        ok = (st[sample] == 0) & (o["status"] == 0)
        err = np.abs(g["logL"][sample][ok] - o["logL"][ok])
        rel = err / np.abs(o["logL"][ok])
        dom = max(tm, key=lambda k: tm[k][0])
        entry = {"evals_per_s": K / (ms * 1e-3), "ms_per_step": ms, "batch": batch,
                 "max_rel_dlogL_vs_oracle": float(rel.max()) if rel.size else None,
                 "max_abs_dlogL_vs_oracle": float(err.max()) if err.size else None,
                 "status_mismatch": int(((st[sample] != 0) != (o["status"] != 0)).sum()),
                 "compared": int(ok.sum()), "dominant_kernel": dom,
                 "kernel_share": {k: round(v[0] / max(1e-9, sum(x[0] for x in tm.values())), 4)
                                  for k, v in tm.items() if v[1]}}
        if dom == "trailing_gemm":
            tf = sum(trailing_flops(n, ds.p + M)) * K
            ach = tf / (tm[dom][0] * 1e-3) / 1e12
            entry["roofline"] = {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                                 "frac": ach / fp64_peak, "kernel": "k_gemm_nt<1> (FP64 trailing update)",
                                 "peak_source": "FP64 FMA pipe measured live"}
        elif dom == "build":
            # Matern entries per second against the FP64 pipe: ~14 FP64 operations per entry
            ent = n * (n - 1) / 2 * K / (tm[dom][0] * 1e-3)
            entry["roofline"] = {"bound": "alu", "achieved": ent * 14 * 2 / 1e12, "peak": fp64_peak, "unit": "TFLOP/s",
                                 "frac": ent * 14 * 2 / 1e12 / fp64_peak, "kernel": "k_build (Matern tiles)",
                                 "achieved_is": "14 FP64 ops per lower-triangle entry, counted as 2 flops each "
                                                "(FMA-equivalent), over the build's event time",
                                 "entries_per_s": ent}
        out[name] = entry
        del ws
        torch.cuda.empty_cache()
    line = {"metric": f"profile-logL evals/s, {args.workload}", "value": out["fp64"]["evals_per_s"], "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": out["fp64"]["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: n={n}, p={ds.p}, K={K}, M={M}", "precision": "fp64 (headline), mixed",
                       "mixed_tolerance": nv.get_mixed_tolerance(),
                       "cuda_graphs": bool(args.graph)},
            "fp64": out["fp64"], "mixed": out["mixed"], "fp64_warp_fma_cycles": probe_fp64_lanes(),
            "cpu_baseline": {"value": len(sample) / t_or, "unit": UNIT, "cores": o["threads"], "kind": "oracle",
                             "sample": f"{len(sample)} of the {K} points ({t_or:.1f} s wall)"}}
    print(json.dumps(line), flush=True)


def trail_kernel_sha256(root):
    """SHA-256 of the trailing-update kernel's source (its configuration, the
    kernel and the PTX wrappers it uses)."""
    import hashlib
    with open(os.path.join(root, "paper_2305_04318_b300/csrc/plk_mixed.cu"), "rb") as fh:
        src = fh.read()
    a = src.index(b"namespace pipe {")
    z = src.index(b"// Panel solve with 7 exact groups", a)
    h = hashlib.sha256(src[a:z])
    with open(os.path.join(root, "paper_2305_04318_b300/csrc/plk_tc.cuh"), "rb") as fh:
        h.update(fh.read())
    return h.hexdigest()


def trail_launches(n, part, TB=128, GP=4):
    """(items, panels, mode) of every k_trail_pipe<5> launch of the 5-slice pass over
    one part of `part` points at n sites: the schedule of launch_mixed_steps
    (panels in groups of GP: before each panel its column's data rows with the
    group's earlier panels, after it the right-hand-side row, after the group
    the data triangle with all its panels)."""
    nb = -(-n // TB)
    out = []

    def add(mode, Klo, Ihi, P):
        m = Ihi - Klo + 1
        if m <= 0:
            return
        T = m * (m + 1) // 2 if mode == 0 else m
        # 0: data triangle, 1: one column's data rows (half-tile items);
        # 2: right-hand-side row (whole-tile items, run transposed)
        out.append((part * T * (1 if mode == 2 else 2), P, mode))
    for J0 in range(0, nb, GP):
        G = min(GP, nb - J0)
        Jend = J0 + G
        for J in range(J0, Jend):
            if J > J0:
                add(1, J, nb - 1, J - J0)
            add(2, J + 1, nb, 1)
        add(0, Jend, nb - 1, G)
    return out


def first_pass_parts(B, part=296):
    if B < 256:
        return [B]
    k = max(2, -(-B // part))
    return [B * (i + 1) // k - B * i // k for i in range(k)]


def trail_traffic(n, B):
    """Modelled DRAM bytes per k_trail_pipe<5> launch of this workload (mean over
    the launches of one evaluation), or None when the kernel sources differ
    from the ones the counters were taken on."""
    root = os.path.dirname(os.path.abspath(__file__))
    if TRAIL_TRAFFIC["sources_sha256"] is None or trail_kernel_sha256(root) != TRAIL_TRAFFIC["sources_sha256"]:
        return None
    L = [x for c in first_pass_parts(B) for x in trail_launches(n, c)]
    t = TRAIL_TRAFFIC

    def launch_bytes(it, P, mode):
        if mode == 0:
            return t["tri_item"] * it
        if mode == 1:
            return t["col_item"] * it + t["col_item_panel"] * it * P
        return t["rhs_item"] * it
    return sum(launch_bytes(*x) for x in L) / len(L)


def split_pairs(S):
    return S * (S + 1) // 2


def run_pipe_counters(args):
    """Where the 5-slice trailing update's roles wait, per launch mode: one
    warm-up and one counted mixed evaluation of a bench step (the n=4000
    workload's points tiled to the step batch) through the diagnostic build."""
    from paper_2305_04318_b300 import build
    os.environ["PLK_LIBRARY"] = build.build_counters()
    import torch
    from paper_2305_04318_b300 import native as nv, synth
    w = synth.mixed4000()
    ds, P = w.datasets[0], w.params[0]
    B = args.batch or 1776
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")
    xs = (T(ds.coords), T(ds.y), T(ds.X), T(w.lambdas), T(np.resize(P, (B, 5))))
    nv.eval_device(*xs, precision=nv.MIXED, batch=B)
    torch.cuda.synchronize()
    nv.pipe_counters(reset=True)
    nv.eval_device(*xs, precision=nv.MIXED, batch=B)
    torch.cuda.synchronize()
    c = nv.pipe_counters(reset=True)
    out = {}
    for mode, v in c.items():
        loop, items = v["loop_cycles"], max(v["items"], 1)
        out[mode] = {"items": v["items"], "cycles_per_item": round(loop / items),
                     "share_of_loop": {k: round(v[k] / loop, 4) for k in nv.PIPE_COUNTER_NAMES[2:]} if loop else {},
                     "per_item": {k: round(v[k] / items) for k in nv.PIPE_COUNTER_NAMES[2:]}}
    print(json.dumps({"diagnostic": "trailing-update wait cycles (k_trail_pipe<5>, one thread block per SM; "
                                    "MMA waits are the MMA thread's, epilogue waits its first thread's)",
                      "workload": f"mixed4000: n={ds.n}, p={ds.p}, M={len(w.lambdas)}, batch={B}",
                      "modes": out}))


def main():
    args = parse()
    if args.pipe_counters:
        run_pipe_counters(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "uneven":
        run_uneven(args)
        return
    if args.workload == "serving":
        run_serving(args)
        return
    if args.workload == "pipeline":
        run_pipeline(args)
        return
    if args.workload in ("iso100", "aniso1000"):
        run_small_config(args)
        return
    import torch
    import torch.distributed as dist
    from paper_2305_04318_b300 import native as nv, shard, synth

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    head = "mixed" if args.precision in ("auto", "mixed") else "fp64"
    w = synth.mixed4000(n=args.n)
    ds, P, lam = w.datasets[0], w.params[0], w.lambdas
    K = P.shape[0]
    n, p, M = ds.n, ds.p, len(lam)
    q = M + p
    nb = -(-n // 128)
    dev = torch.device("cuda", local)
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)
    coords, y, X, lamd, Pd = T(ds.coords), T(ds.y), T(ds.X), T(lam), T(P)
    stream = torch.cuda.current_stream()
    peaks = measured_peaks()

    def outputs(B):
        return dict(logL=torch.empty((B, M), dtype=torch.float64, device=dev),
                    sigma2=torch.empty((B, M), dtype=torch.float64, device=dev),
                    beta=torch.empty((B, M, p), dtype=torch.float64, device=dev),
                    logdet=torch.empty((B, 2), dtype=torch.float64, device=dev),
                    status=torch.empty((B,), dtype=torch.int32, device=dev),
                    err_bound=torch.empty((B,), dtype=torch.float64, device=dev))

    def step_params(s, B):
        # rank r evaluates its own slice of the grid (shard.step_indices)
        idx = torch.as_tensor(shard.step_indices(s, rank, world, B, K), device=dev)
        return Pd.index_select(0, idx).contiguous()

    def measure(prec_name, B, steps, warmup, sample_clocks, batches=None):
        precision = nv.MIXED if prec_name == "mixed" else nv.FP64
        wsb = nv.workspace_bytes(n, p, M, B, precision)
        workspace = torch.empty((wsb,), dtype=torch.uint8, device=dev)
        if batches is None:
            batches = [step_params(s, B) for s in range(warmup + steps)]
        outs = [outputs(B) for _ in range(warmup + steps)]

        def one(s, flags=0):
            nv.eval_device(coords, y, X, lamd, batches[s], precision=precision, batch=B, workspace=workspace,
                           stream=stream, outputs=outs[s], flags=flags)

        for s in range(warmup):
            one(s)
        barrier()
        clocks = ClockSampler(local) if sample_clocks else None
        if clocks:
            clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record(stream)
        for s in range(warmup, warmup + steps):
            one(s)
        e1.record(stream)
        barrier()
        clk = clocks.stop() if clocks else None
        ms_total = max_over_ranks(e0.elapsed_time(e1))
        status = np.concatenate([outs[s]["status"].cpu().numpy() for s in range(warmup, warmup + steps)])
        first = {k: v.cpu().numpy() for k, v in outs[warmup].items()}
        gather = None
        if world > 1 and sample_clocks:
            # the ranks' per-point results of the timed steps to every rank in
            # one all_gather (after the timed region)
            g0 = time.perf_counter()
            idx = np.concatenate([shard.step_indices(s, rank, world, B, K) for s in range(warmup, warmup + steps)])
            mine = {k: np.concatenate([outs[s][k].cpu().numpy() for s in range(warmup, warmup + steps)])
                    for k in shard.RESULT_KEYS}
            merged, covered, mism = shard.gather_results(idx, mine, K, M, p, device=dev, strict=False)
            gather = {"points_covered": covered, "of": K, "ms": 1e3 * (time.perf_counter() - g0),
                      "repeated_points_with_different_results": mism,
                      "what": "shard.gather_results of the timed steps' per-point results (one all_gather)"}
        # per-kernel-class times: the same steps once more, outside the timed
        # region, with CUDA events around every launch on its stream
        nv.kernel_timing(reset=True)
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for s in range(warmup, warmup + steps):
            one(s, flags=nv.FLAG_KERNEL_TIMING)
        f1.record(stream)
        barrier()
        timing = nv.kernel_timing(reset=True)
        res = dict(value=world * B * steps / (ms_total * 1e-3), ms_per_step=ms_total / steps, timing=timing,
                   instrumented_ms_per_step=f0.elapsed_time(f1) / steps,
                   clocks=clk, status=status, wsb=wsb, B=B, steps=steps, warmup=warmup,
                   first=first, first_params=batches[warmup], gather=gather)
        del workspace
        torch.cuda.empty_cache()
        return res

    Bm = args.batch or (1776 if head == "mixed" else 128)   # mixed: 12 x 148 points per step, parts of 296
    main_res = measure(head, Bm, args.steps, args.warmup, True)
    fp64_res = None
    if head == "mixed":
        # the FP64 path on 128-point slices of the mixed run's timed steps (its
        # first timed step starts with the first 128 points of the mixed run's)
        fs = max(1, min(args.steps, 2))
        src = [step_params(args.warmup + s, Bm) for s in range(fs)]
        fB = min(128, Bm)
        fb = [src[0][:fB].contiguous()] + [src[s][:fB].contiguous() for s in range(fs)]
        fp64_res = measure("fp64", fB, fs, 1, False, batches=fb)

    timing = main_res["timing"]
    dom = max(timing, key=lambda k: timing[k][0])
    dom_ms = timing[dom][0]
    launches = int(sum(c for _, c in timing.values()))
    pipes = probe_pipes()
    fp64_peak, fp32_peak = pipes["fp64_fma"], pipes["fp32_fma"]
    tf = sum(trailing_flops(n, q))   # algorithmic trailing-update flops per omega
    roof = None
    st = main_res["status"]
    n_pts = len(st)
    if dom in ("trailing_gemm",):
        achieved = tf * n_pts / (dom_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak, "traffic": None, "kernel": "k_gemm_nt<1> (FP64 trailing update)",
                "peak_source": "FP64 FMA pipe measured live by libplk_probe (no FP64 figure in MEASURED_PEAKS.json)"}
    elif dom == "trailing_split":
        n7 = int(((st & nv.POINT_RETRIED) != 0).sum())
        n64 = int(((st & nv.POINT_FP64) != 0).sum())
        # every point enters the 5-slice pass (this kernel); a point that is
        # re-evaluated with 7 slices (in separate kernels, trailing_split7) leaves
        # it early once its partial error bound passes the tolerance, so only the
        # points that complete it are counted (a lower bound: the retried
        # points' partial work is left out)
        n5 = n_pts - n7
        # per panel J: the data tiles (m (m - 1) / 2, m = nb - J) are 128 x 128 x 128
        # products; the m right-hand-side tiles run transposed with N = the
        # right-hand-side rows rounded up to 8, then to 32
        nr = -(-(-(-q // 8) * 8) // 32) * 32
        cols = sum((nb - J) * (nb - J - 1) // 2 * 128 + (nb - J) * nr for J in range(nb))
        executed = 2.0 * 128 ** 2 * cols * split_pairs(5) * n5
        peak = peaks.get("bf16_tflops_sustained") or 1341.1
        alg = tf * n5 / (dom_ms * 1e-3) / 1e12
        roof = {"bound": "tensor", "achieved": alg, "peak": peak, "unit": "TFLOP/s", "frac": alg / peak,
                "traffic": trail_traffic(n, Bm), "kernel": "k_trail_pipe (5-slice split-bf16 trailing update, tcgen05, persistent)",
                "achieved_is": "algorithmic FP64-equivalent trailing-update flops (n^3/3 + n^2 q per omega, omega that complete the 5-slice pass) / kernel time",
                "executed_bf16_tflops": executed / (dom_ms * 1e-3) / 1e12,
                "executed_frac": executed / (dom_ms * 1e-3) / 1e12 / peak,
                "executed_is": "bf16 MMA flops issued by this kernel for the omega that complete the 5-slice pass: 15 slice products per multiply-add, 128x128 data tiles, 128 x NR right-hand-side tiles (NR = M + p rounded up to 32)",
                "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (kernel timed inside a long step)",
                "fp64_equivalent_over_fp64_fma_peak": alg / fp64_peak,
                "points_7slice": n7, "points_fp64": n64}
    share_tot = max(1e-9, sum(x[0] for x in timing.values()))
    kernel_share = {k: round(v[0] / share_tot, 4) for k, v in timing.items() if v[1]}

    # agreement of mixed with the FP64 path on the same points
    agree = None
    if fp64_res is not None:
        gm, gf = main_res["first"], fp64_res["first"]
        m = min(len(gf["status"]), len(gm["status"]))
        okp = ((gm["status"][:m] & 15) == 0) & (gf["status"][:m] == 0)
        d = np.abs(gm["logL"][:m][okp] - gf["logL"][:m][okp])
        agree = {"points": int(m), "compared": int(okp.sum()), "max_abs_dlogL_vs_fp64": float(d.max()) if d.size else None,
                 "status_mismatch": int((((gm["status"][:m] & 15) != 0) != (gf["status"][:m] != 0)).sum())}
        if d.size:
            s2 = np.abs(gm["sigma2"][:m][okp] / gf["sigma2"][:m][okp] - 1.0)
            bd = np.abs(gm["beta"][:m][okp] - gf["beta"][:m][okp]) / np.abs(gf["beta"][:m][okp]).max()
            ld = np.abs(gm["logdet"][:m][okp] - gf["logdet"][:m][okp])
            agree.update({"max_rel_dsigma2_vs_fp64": float(s2.max()), "max_dbeta_rel_to_max_beta_vs_fp64": float(bd.max()),
                          "max_abs_dlogdet_vs_fp64": float(ld.max()),
                          "what": "per-result errors of the mixed path against the FP64 path on the same points"})

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    lat = None
    if not args.no_e2e:
        precision = nv.MIXED if head == "mixed" else nv.FP64
        B = Bm
        wsb = nv.workspace_bytes(n, p, M, B, precision)
        arena = torch.empty((wsb + (256 << 20),), dtype=torch.uint8, device=dev)
        ctx = nv.Context(arena.numel(), device=local, arena=arena, n_streams=1)
        hostP = [np.ascontiguousarray(step_params(s, B).cpu().numpy()) for s in range(args.warmup + args.steps)]

        def e2e_step(s):
            t0 = time.perf_counter()
            did = ctx.create_dataset(ds.coords, ds.y, ds.X)
            job = ctx.submit(did, hostP[s], lam, precision=precision, batch=B)
            r = ctx.poll(job, p)
            ctx.release_dataset(did)
            return time.perf_counter() - t0, r

        for s in range(args.warmup):
            e2e_step(s)
        barrier()
        times = []
        for s in range(args.warmup, args.warmup + args.steps):
            dt, r = e2e_step(s)
            times.append(dt)
        tot = max_over_ranks(sum(times))
        ctx.close()
        del arena
        h2d = ds.coords.nbytes + ds.y.nbytes + ds.X.nbytes + hostP[0].nbytes + lam.nbytes
        d2h = r["logL"].nbytes + r["sigma2"].nbytes + r["beta"].nbytes + r["logdet"].nbytes + r["status"].nbytes
        e2e = {"value": world * B * args.steps / tot, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}
        lat = {"p50": 1e3 * float(np.percentile(times, 50)), "p99": 1e3 * float(np.percentile(times, 99)),
               "what": f"end-to-end latency of one {B}-point job (host inputs -> host results)"}

    # ---- CPU baseline (oracle on the host cores), rank 0 at N = 1 only ----
    cpu = None
    vs_oracle = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = cpu_cores()
        npts = args.cpu_sample or cores
        sidx = oracle_sample_indices(K, npts)
        r, dt, used, o = oracle_rate(ds, P[sidx], lam, npts, cores, full=True)
        cpu = {"value": r, "unit": UNIT, "cores": used, "kind": "oracle",
               "sample": f"{npts} omega points of the n=4000 workload: the first {int((sidx < K - 64).sum())} "
                         f"Halton points and {int((sidx >= K - 64).sum())} ill-conditioned ones (kappa=8, phi_X>=23; "
                         f"the oracle stops early on the points it finds not positive definite) "
                         f"({dt:.1f} s wall, one point per thread)"}
        # per-result errors of both GPU paths against the oracle on these points
        Ps = T(P[sidx])
        vs_oracle = {"points": [int(i) for i in sidx],
                     "what": "largest errors of each GPU path against the FP64 CPU oracle on the CPU-baseline sample"}
        for name, prec in (("mixed", nv.MIXED), ("fp64", nv.FP64)):
            g = nv.eval_device(coords, y, X, lamd, Ps, precision=prec, batch=len(sidx))
            torch.cuda.synchronize()
            vs_oracle[name] = per_result_errors({k: v.cpu().numpy() for k, v in g.items()}, o, lam)

    if rank == 0:
        fp64_line = None
        if fp64_res is not None:
            tm = fp64_res["timing"]
            gms = tm.get("trailing_gemm", (0.0, 0))[0]
            ach = tf * len(fp64_res["status"]) / (gms * 1e-3) / 1e12 if gms else None
            fp64_line = {"value": fp64_res["value"], "unit": UNIT, "ms_per_step": fp64_res["ms_per_step"],
                         "batch_per_step": fp64_res["B"], "steps": fp64_res["steps"],
                         "trailing_gemm_tflops": ach, "trailing_gemm_frac_of_fp64_peak": (ach / fp64_peak) if ach else None}
        line = {"metric": METRIC, "value": main_res["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": main_res["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[head], "data": "synthetic",
                "config": {"workload": WORKLOAD, "precision": head, "batch_per_step": Bm, "n": n, "p": p, "M": M,
                           "mixed_tolerance": nv.get_mixed_tolerance(),
                           "l2": f"inputs larger than L2: {main_res['wsb'] / 1e9:.1f} GB workspace per step",
                           "parallelism": f"omega-sharded x{world}"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "latency_ms": lat,
                "gpu_launches": launches, "kernel_ms": {k: round(v[0], 3) for k, v in timing.items() if v[1]},
                "kernel_share": kernel_share, "clocks": main_res["clocks"],
                "fp64_path": fp64_line, "mixed_vs_fp64": agree, "vs_oracle": vs_oracle,
                "rank_gather": main_res["gather"],
                "instrumented_ms_per_step": main_res["instrumented_ms_per_step"],
                "kernel_timing_is": "kernel_ms, kernel_share and the roofline's kernel time come from the timed "
                                    "steps run once more after the timed region with CUDA events around every "
                                    "launch (instrumented_ms_per_step); value and ms_per_step are uninstrumented",
                "fp64_fma_peak_tflops": fp64_peak, "fp32_fma_peak_tflops": fp32_peak, "pipe_probes_tflops": pipes,
                "points_not_ok": int(((st & 15) != 0).sum()), "points_evaluated": int(n_pts),
                "points_retried_7slice": int(((st & nv.POINT_RETRIED) != 0).sum()),
                "points_fp64_tier": int(((st & nv.POINT_FP64) != 0).sum())}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
