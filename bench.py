#!/usr/bin/env python3
"""Benchmark of the pole-batched exp(A)V hot path on the 1D Laplacian workload.

Workload (one "step" = one evaluation of exp(T)V ~ R_16(T)V):
  T = 100 * tridiag(1, -2, 1), N = 2^20 rows (spectrum in (-400, 0)),
  V = 2^20 x 8 Gaussian block (float64), degree 16 -> 8 conjugate pole pairs,
  64 complex shifted tridiagonal systems of length 2^20, residue sum fused.

Printed: one JSON line (rank 0).  ``value`` is evaluations per second of the
binary64 path with inputs resident in HBM; ``mixed`` is the float-float path;
``e2e`` goes through the C interface with pinned HOST buffers, so the library's
host<->device copies are inside the timed region.  Each timed step is bracketed
by CUDA events on the launch stream; a 256 MB buffer is rewritten between steps
to flush the 129 MB L2 (outside the step's events).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --peaks        # FMA-throughput probe of the FP64/FP32 pipes

Under torchrun (N > 1) every rank evaluates its own independent instance
(weak scaling, no collective on the data path); the time is the max over ranks.
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
import tempfile
import time

# Host-side linear algebra here (input generation, oracle, closed forms) parallelises over
# independent problems with its own threads; one BLAS thread per caller avoids
# oversubscribing the cores.  Must be set before numpy loads its BLAS.
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "exp(A)V evals/s + p99 latency, mixed vs FP64 path at rel err ≤1e-8; % roofline"
N_ROWS = 1 << 20
NRHS = 8
DEGREE = 16
# nominal FP64 FMA rate of a GB300 SM: 1.25 TFLOP/s / (152 SMs x 2.07 GHz) = 4 flop/clk/SM
SMS = 152
FP64_FLOP_PER_CLK_SM = 4
SM_MAX_MHZ = 2070.0
# algorithmic flops per (system, column, row) of the dominant kernel (tri_block_solve),
# whose forward substitution runs on z = W d' with the residue weight folded into its
# coefficients: forward 10 (z = a v - b z_prev: a v 2, b z_prev 6, subtraction 2), back 8
# (x = z - c' x+: product 6, subtraction 2); Re(W x) is then Re(x) and costs nothing (the
# reduce-scatter addition over the systems, < 1 per element, is not counted)
FLOPS_K3 = 18
# FP32 flops per (system, column, row) of the mixed path's dominant kernel (mx_main: pass 0
# of the binary32 + refinement path), an FMA counting 2: the forward recurrence twice
# (checkpoint pass and chunk recompute, 10 each), the back substitution with c' = e' g (10),
# the float-float residual r_1 (8 error-free products with compensated sums, 129), Re(W x_0)
# as a float pair with its share of the reduce-scatter (24), the last-row spike dot (16), the
# bottom-up sweep for the first-row end value (10), the two norms (6)
FLOPS_MX_MAIN = 215
FP32_FLOP_PER_CLK_SM = 256


def _hbm_peak() -> float:
    """Measured copy bandwidth of this GPU pool (GB/s), else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0


HBM_GBS = _hbm_peak()


def _bf16_peak() -> tuple:
    """Measured dense bf16 TFLOP/s (burst, sustained) from MEASURED_PEAKS.json, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["bf16_tflops"]), float(d["bf16_tflops_sustained"]), "measured"
    except (OSError, KeyError, ValueError):
        return 1900.0, 1700.0, "fallback"
# the binary32 + refinement path: one correction pass at most, stopping test 1e-10
MIXED_OPTS = dict(tol=1e-10, max_refine=1)
# algorithmic HBM bytes of one evaluation: d, e, V read, Y written (binary64)
# dram bytes (read + write) per launch of tri_block_solve<f64> at N = 2^20: one ncu
# capture at N = 2^19 (1.4247 GB: 857.7 MB read + 567.0 MB write) scaled by 2, the
# traffic being proportional to N; valid while the kernel's source text hashes to
# TRAFFIC_SRC_SHA (otherwise reported as null)
TRAFFIC_K3 = 2.8495e9
TRAFFIC_SRC_SHA = "b5a5c00d7042b497"
# dram bytes (read + write) per launch of mx_main<8> at N = 2^20: one ncu capture at
# N = 2^19 (395.8 MB: 114.1 MB read + 281.7 MB write) scaled by 2, the traffic being
# proportional to N; valid while tridiag_mixed.cu hashes to TRAFFIC_MX_SHA
TRAFFIC_MX = 7.917e8
TRAFFIC_MX_SHA = "901bd1b081954068"


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--peaks", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other configurations' sub-objects (dense small, dense 4096, uneven batch, "
                         "served stream)")
    ap.add_argument("--rows", type=int, default=N_ROWS,
                    help="rows of the Laplacian (smaller cases are for profiling only)")
    ap.add_argument("--fp64-only", action="store_true",
                    help="time only the binary64 path (profiling runs)")
    ap.add_argument("--mixed-only", action="store_true",
                    help="time only the binary32 + refinement path (profiling runs)")
    ap.add_argument("--workload", default="laplacian",
                    choices=["laplacian", "dense", "batched", "served", "laplacian2d", "dense_small"],
                    help="laplacian: the headline line; the others print their own lines "
                         "(dense 4096 Hermitian x 256 RHS; 4096-instance uneven batch; served stream; "
                         "dense 64 x 64 degree 12, --steps evaluations per path)")
    ap.add_argument("--dense-n", type=int, default=4096)
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--served-requests", type=int, default=2000)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(vals, world, device=None):
    """Element-wise maximum of per-rank timings over all ranks (the slowest rank sets the
    job's time); the process group must be initialised when world > 1."""
    if world <= 1:
        return [float(v) for v in vals]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def shard_columns(r, rank, world):
    """Right-hand-side columns [c0, c1) of `rank` when one evaluation's r columns are split
    over `world` ranks: the columns of eq. expAx are independent, so each rank evaluates
    its block with the whole operator and the result is the concatenation (no exchange
    until the gather)."""
    base, extra = divmod(r, world)
    c0 = rank * base + min(rank, extra)
    return c0, c0 + base + (1 if rank < extra else 0)


def shard_instances(sizes, world):
    """Instances of an uneven batch assigned to `world` ranks: longest first, each to the
    rank with the least work so far (n^3 per instance); one ascending index list per rank."""
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for i in sorted(range(len(sizes)), key=lambda j: (-sizes[j], j)):
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += float(sizes[i]) ** 3
    return [sorted(x) for x in out]


def whole_job_value(world, steps, max_seconds):
    """Evaluations per second of the whole job: every rank runs `steps` evaluations of its
    own replica (weak scaling) in at most `max_seconds`."""
    return world * steps / max_seconds


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s in sm if s > 0.5 * max(sm)]
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def kernel_sha() -> str:
    """Hash of the source text of the tri_block_solve kernel template."""
    src = open(os.path.join(ROOT, "paper_2306_16778_gb300", "csrc", "tridiag.cu")).read()
    i = src.index("__global__ void __launch_bounds__(128) tri_block_solve(")
    i = src.rindex("template <class R, int LG>", 0, i)
    j = src.index("\n}\n", i) + 3
    return hashlib.sha256(src[i:j].encode()).hexdigest()[:16]


def mixed_sha() -> str:
    """Hash of the mixed tridiagonal path's source file."""
    src = open(os.path.join(ROOT, "paper_2306_16778_gb300", "csrc", "tridiag_mixed.cu")).read()
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def run_peaks():
    import ctypes
    import __graft_entry__
    lib = ctypes.CDLL(__graft_entry__._build_module().build_probe())
    lib.expm_probe_fma_tflops.restype = ctypes.c_double
    lib.expm_probe_fma_tflops.argtypes = [ctypes.c_int] * 4
    out = {}
    for kind, name, iters in ((0, "fp64", 200), (1, "fp32", 4000), (2, "fp32x2", 2000)):
        for bps in (4, 8, 16):
            tf = lib.expm_probe_fma_tflops(kind, iters, bps, 5)
            out[f"{name}_tflops_bps{bps}"] = round(tf, 4)
    print(json.dumps({"probe": "fma_throughput", **out}))


# the headline configuration, identical on both arms
CONFIG = {"workload": "1D Laplacian 100*tridiag(1,-2,1), N=2^20, 8 Gaussian RHS, degree 16, FP64",
          "N": N_ROWS, "nrhs": NRHS, "degree": DEGREE, "systems": (DEGREE // 2) * NRHS,
          "l2": "256 MB buffer rewritten between timed steps (outside the step events)"}


def cpu_oracle_eval(w, workers):
    from oracle import coeffs, matrix
    th, a = coeffs.theta(DEGREE), coeffs.residues(DEGREE)
    t0 = time.perf_counter()
    Y, _ = matrix.apply_tridiag(w["d"], w["e"], w["V"], th, a, workers=workers)
    return Y, time.perf_counter() - t0


def run_ours(args):
    import torch
    import paper_2306_16778_gb300 as P
    import workloads

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    rows = args.rows
    w = workloads.laplacian_1d(N=rows, nrhs=NRHS, offset=1 + rank)
    plan = P.Plan(degree=DEGREE)
    d, e, V = (torch.from_numpy(x).to(dev) for x in (w["d"], w["e"], w["V"]))
    Y = torch.empty_like(V)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)   # 256 MB > 129 MB L2
    S = DEGREE // 2
    K, W = args.steps, args.warmup

    def timed_loop(prec, steps, **kw):
        for _ in range(W):
            P.expm_apply_tridiag(plan, d, e, V, Y, prec=prec, want_info=False, **kw)
        torch.cuda.synchronize()
        P.expm_profile_enable(plan, True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        barrier()
        torch.cuda.synchronize()
        for a, b in ev:
            flush.zero_()
            a.record()
            P.expm_apply_tridiag(plan, d, e, V, Y, prec=prec, want_info=False, **kw)
            b.record()
        torch.cuda.synchronize()
        barrier()
        ms = [a.elapsed_time(b) for a, b in ev]
        prof = P.expm_profile_read(plan)
        P.expm_profile_enable(plan, False)
        return ms, prof

    if args.mixed_only:
        msmx, profmx = timed_loop(P.EXPM_MIXED_FP32, K, **MIXED_OPTS)
        if rank == 0:
            print(json.dumps({"mixed_only": True, "rows": rows, "ms_per_step": sum(msmx) / K,
                              "kernels_ms": {k: v[1] / v[0] for k, v in profmx.items()}}), flush=True)
        plan.close()
        return
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
    ms64, prof64 = timed_loop(P.EXPM_FP64, K)
    clocks = sampler.stop() if sampler else None
    Y64 = Y.cpu().numpy() if rank == 0 else None
    if args.fp64_only:
        if rank == 0:
            print(json.dumps({"fp64_only": True, "rows": rows, "ms_per_step": sum(ms64) / K,
                              "kernels_ms": {k: v[1] / v[0] for k, v in prof64.items()}}), flush=True)
        plan.close()
        return
    msff, profff = timed_loop(P.EXPM_MIXED_F32X2, K)
    Yff = Y.cpu().numpy() if rank == 0 else None
    # binary32 factors + refinement: the asynchronous timed calls do not read the
    # refinement state back; one call with info afterwards reports it
    msmx, profmx = timed_loop(P.EXPM_MIXED_FP32, K, **MIXED_OPTS)
    infomx = P.expm_apply_tridiag(plan, d, e, V, Y, prec=P.EXPM_MIXED_FP32, check=False, **MIXED_OPTS)
    Ymx = Y.cpu().numpy() if rank == 0 else None

    # end to end through the C interface with pinned host buffers (synchronous call)
    hd, he, hV = (torch.from_numpy(x).pin_memory() for x in (w["d"], w["e"], w["V"]))
    hY = torch.empty_like(hV).pin_memory()
    Ke = max(5, K // 10)
    for _ in range(3):
        P.expm_apply_tridiag(plan, hd, he, hV, hY)
    barrier()
    t0 = time.perf_counter()
    for _ in range(Ke):
        P.expm_apply_tridiag(plan, hd, he, hV, hY)
    e2e_s = time.perf_counter() - t0
    barrier()

    tot64 = sum(ms64) / 1e3
    totff = sum(msff) / 1e3
    totmx = sum(msmx) / 1e3
    tot64, totff, totmx, e2e_s = max_over_ranks([tot64, totff, totmx, e2e_s], world, dev)
    if rank != 0:
        return

    def pct(xs, q):
        xs = sorted(xs)
        return xs[min(len(xs) - 1, int(math.ceil(q / 100.0 * len(xs))) - 1)]

    value = whole_job_value(world, K, tot64)
    # dominant kernel of the binary64 step and its roofline
    top = max(prof64.items(), key=lambda kv: kv[1][1])
    kname, (klaunch, kms) = top
    kavg_s = kms / klaunch / 1e3
    flops = FLOPS_K3 * S * NRHS * rows
    achieved = flops / kavg_s / 1e12
    peak = SMS * FP64_FLOP_PER_CLK_SM * SM_MAX_MHZ * 1e6 / 1e12
    traffic = TRAFFIC_K3 if (TRAFFIC_K3 is not None and TRAFFIC_SRC_SHA == kernel_sha()) else None
    hbm_bytes = 8 * (rows + (rows - 1) + 2 * rows * NRHS)

    # the mixed path's dominant kernel on the FP32 pipe
    mx_name = "tri_mixed_main"
    mx_roof = None
    if mx_name in profmx:
        mxl, mxms = profmx[mx_name]
        mx_ach = FLOPS_MX_MAIN * S * NRHS * rows / (mxms / mxl / 1e3) / 1e12
        mx_peak = SMS * FP32_FLOP_PER_CLK_SM * SM_MAX_MHZ * 1e6 / 1e12
        mx_traffic = TRAFFIC_MX if (TRAFFIC_MX is not None and TRAFFIC_MX_SHA == mixed_sha()) else None
        mx_roof = {"kernel": "mx_main<8> (pass 0: binary32 solve, float-float residual, Y update)", "bound": "alu",
                   "achieved": round(mx_ach, 3), "peak": round(mx_peak, 3), "unit": "TFLOP/s",
                   "frac": round(mx_ach / mx_peak, 4), "traffic": mx_traffic,
                   "peak_source": "derived: 152 SMs x 256 FP32 flop/clk x 2070 MHz (probe: 78.4 TFLOP/s)",
                   "algorithmic": f"{FLOPS_MX_MAIN} FP32 flop per (system, column, row) x {S}x{NRHS}x{rows}"}
    line = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": "evals/s",
        "n_gpus": world,
        "steps": K,
        "warmup": W,
        "ms_per_step": round(tot64 * 1e3 / K, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": dict(CONFIG, parallelism=f"replicas{world}"),
        "latency_ms": {"p50": round(pct(ms64, 50), 4), "p99": round(pct(ms64, 99), 4)},
        "mixed": {"prec": "binary32 factors and solves + float-float-residual refinement (EXPM_MIXED_FP32, "
                          f"tol {MIXED_OPTS['tol']:g}, max_refine {MIXED_OPTS['max_refine']})",
                  "value": round(whole_job_value(world, K, totmx), 3), "unit": "evals/s",
                  "ms_per_step": round(totmx * 1e3 / K, 4),
                  "latency_ms": {"p50": round(pct(msmx, 50), 4), "p99": round(pct(msmx, 99), 4)},
                  "speedup_vs_fp64": round(tot64 / totmx, 3),
                  "refine_passes": infomx.refine_iters_max, "resid_rel": infomx.resid_rel_max,
                  "status": infomx.status_worst,
                  "hbm_effective": {"achieved_gbs": round(hbm_bytes * K / totmx / 1e9, 2), "peak_gbs": HBM_GBS,
                                    "frac": round(hbm_bytes * K / totmx / 1e9 / HBM_GBS, 5)},
                  "roofline": mx_roof,
                  "kernels_ms": {k: round(v[1] / v[0], 4) for k, v in profmx.items()}},
        "mixed_f32x2": {"prec": "float-float (EXPM_MIXED_F32X2)",
                        "value": round(whole_job_value(world, K, totff), 3),
                        "unit": "evals/s", "ms_per_step": round(totff * 1e3 / K, 4),
                        "latency_ms": {"p50": round(pct(msff, 50), 4), "p99": round(pct(msff, 99), 4)},
                        "kernels_ms": {k: round(v[1] / v[0], 4) for k, v in profff.items()}},
        "hbm_effective": {"achieved_gbs": round(hbm_bytes * K / tot64 / 1e9, 2), "peak_gbs": HBM_GBS,
                          "frac": round(hbm_bytes * K / tot64 / 1e9 / HBM_GBS, 5),
                          "bytes_per_eval": hbm_bytes, "note": "algorithmic bytes (d, e, V in; Y out) / step time"},
        "kernels_ms": {k: round(v[1] / v[0], 4) for k, v in prof64.items()},
        "roofline": {"kernel": kname, "bound": "alu", "achieved": round(achieved, 4),
                     "peak": round(peak, 4), "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                     "traffic": traffic,
                     "peak_source": "derived: 152 SMs x 4 FP64 flop/clk x 2070 MHz (nominal 1.25 TFLOP/s)",
                     "algorithmic": f"{FLOPS_K3} flop per (system, column, row) x {S}x{NRHS}x{N_ROWS}"},
        "e2e": {"value": round(whole_job_value(world, Ke, e2e_s), 3), "unit": "evals/s",
                "h2d_bytes_per_step": int(8 * (N_ROWS + (N_ROWS - 1) + N_ROWS * NRHS)),
                "d2h_bytes_per_step": int(8 * N_ROWS * NRHS)},
        "gpu_launches": sum(v[0] for v in prof64.values()),
        "clocks": clocks,
    }
    if world == 1 and not args.no_cpu_baseline:
        workers = min(16, os.cpu_count() or 1)
        Yo, t = cpu_oracle_eval(w, workers)
        from oracle import matrix
        line["cpu_baseline"] = {"value": round(1.0 / t, 5), "unit": "evals/s", "cores": workers, "kind": "oracle",
                                "sample": f"one full evaluation (N=2^20, 8 RHS, all 16 poles, LAPACK banded LU "
                                          f"per pole on {workers} threads): {t:.2f} s"}
        line["parity"] = {"fp64_rel_err": matrix.rel_err(Y64, Yo), "mixed_rel_err": matrix.rel_err(Ymx, Yo),
                          "mixed_f32x2_rel_err": matrix.rel_err(Yff, Yo),
                          "tolerance": {"fp64": 1e-12, "mixed": 1e-8}}
    if world == 1 and not args.no_configs:
        plan.close()
        del d, e, V, Y, flush
        torch.cuda.empty_cache()
        line["configs"] = bench_configs()
        print(json.dumps(line), flush=True)
        return
    print(json.dumps(line), flush=True)
    plan.close()


def bench_configs():
    """The other configurations, each bounded so that the default run stays within minutes:
    steps and request counts are stated in each sub-object."""
    out = {}
    for key, fn in (("dense_small_64", lambda: cfg_dense_small(300)),
                    ("dense_hermitian_4096", lambda: cfg_dense(4096, 2)),
                    ("uneven_batch_4096", lambda: cfg_batched(4096, 3)),
                    ("served_stream", lambda: cfg_served(600, (0.5, 0.9, 1.2), 12, 200))):
        t0 = time.perf_counter()
        try:
            out[key] = fn()
        except Exception as ex:  # a failing configuration is reported, the headline line still prints
            out[key] = {"error": f"{type(ex).__name__}: {ex}"}
        out[key]["wall_s"] = round(time.perf_counter() - t0, 1)
        log(f"config {key}: {out[key]['wall_s']} s")
    return out


def run_reference(args):
    """The reference arm: the oracle (the paper's method written plainly: one LAPACK banded
    solve per pole for all 16 poles, summed in long double) evaluating the full headline
    workload in every step on the host's cores."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import workloads
    from oracle import coeffs, matrix
    workers = min(16, os.cpu_count() or 1)
    w = workloads.laplacian_1d(N=N_ROWS, nrhs=NRHS, offset=1)
    th, a = coeffs.theta(DEGREE), coeffs.residues(DEGREE)
    for _ in range(args.warmup):
        matrix.apply_tridiag(w["d"], w["e"], w["V"], th, a, workers=workers)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        matrix.apply_tridiag(w["d"], w["e"], w["V"], th, a, workers=workers)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = args.steps / tot
    sample = (f"every step one full evaluation (N=2^20, 8 RHS, all 16 poles, LAPACK banded LU per pole on "
              f"{workers} threads)")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(tot * 1e3 / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(CONFIG, parallelism=f"replicas{world}"),
            "latency_ms": {"p50": round(1e3 * statistics.median(times), 3), "p99": round(1e3 * max(times), 3)},
            "cpu_baseline": {"value": round(value, 5), "unit": "evals/s", "cores": workers, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 5), "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _time_calls(fn, steps, warmup):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    return ts


def _pcts(ts):
    xs = sorted(ts)
    return xs[len(xs) // 2], xs[min(len(xs) - 1, int(math.ceil(0.99 * len(xs))) - 1)]


def _queue_small(P, plan, A, V, prec, steps, Yo, nreq=8192, cap=512):
    """The same evaluation through the device-fed queue (expm_queue_*): latency of one
    request at a time (submit -> completion seen by poll), and throughput with up to `cap`
    requests in flight (nreq requests, each with its own output buffer from a pool of cap)."""
    import torch
    from oracle import matrix
    q = P.Queue(plan, k=1, prec=prec, capacity=cap, idle_ms=2000.0)
    Y = torch.empty_like(V)
    lat = []
    for i in range(steps + 20):
        t0 = time.perf_counter()
        tk = q.submit(A, V, Y)
        while (r := q.poll(tk)) is None:
            pass
        if i >= 20:
            lat.append(time.perf_counter() - t0)
        assert r[0] == 0
    y0 = Y.cpu().numpy()
    pool = [torch.empty_like(V) for _ in range(cap)]
    torch.cuda.current_stream().synchronize()  # not the device: that waits for the idle consumer
    pending, done, nxt = [], 0, 0
    t0 = time.perf_counter()
    while done < nreq:
        while nxt < nreq and len(pending) < cap:
            tk = q.submit(A, V, pool[nxt % cap])
            if tk is None:
                break
            pending.append(tk)
            nxt += 1
        while pending and (r := q.poll(pending[0])) is not None:
            assert r[0] == 0
            pending.pop(0)
            done += 1
    wall = time.perf_counter() - t0
    same = all(torch.equal(y, pool[0]) for y in pool[1:])
    st = q.state()
    q.close()
    p50, p99 = _pcts(lat)
    return {"latency_us": {"p50": round(p50 * 1e6, 2), "p99": round(p99 * 1e6, 2)},
            "throughput": {"requests": nreq, "in_flight_max": cap, "evals_per_s": round(nreq / wall, 1)},
            "clusters": st["clusters"], "kernel_launches": st["launches"],
            "rel_err_vs_oracle": matrix.rel_err(y0, Yo), "all_outputs_identical": bool(same)}


def cfg_dense_small(steps=300):
    """The small plain configuration: real symmetric 64 x 64, spectrum U[-20, 0], one Gaussian
    vector, degree 12 (12 poles, 6 conjugate pairs).  Latency of one evaluation through
    expm_apply_dense and through a captured graph (one launch), binary64 and mixed; parity
    against the oracle and the eigen closed form of R_n(A)v; distance to exp(A)v against
    Prop. 2.2's bound 2^-n."""
    import torch
    import paper_2306_16778_gb300 as P
    import workloads
    from oracle import coeffs, matrix, scalar
    dev = torch.device("cuda", torch.cuda.current_device())
    n = 12
    w = workloads.dense_small(offset=0)
    th, a = coeffs.theta(n), coeffs.residues(n)
    Yo, _ = matrix.apply_dense(w["A"], w["V"], th, a)
    Yeig = matrix.eig_apply(w["Q"], w["mu"], w["V"], lambda x: scalar.R_n(x, n))
    Yexp = matrix.eig_apply(w["Q"], w["mu"], w["V"], np.exp)
    plan = P.Plan(degree=n)
    A, V = (torch.from_numpy(x).to(dev) for x in (w["A"], w["V"]))
    out = {"workload": "dense real symmetric 64x64, spectrum U[-20,0], 1 Gaussian vector, degree 12",
           "evals_per_path": steps}
    for name, prec in (("fp64", P.EXPM_FP64), ("mixed", P.EXPM_MIXED_FP32)):
        Y = torch.empty_like(V)
        ts = _time_calls(lambda: P.expm_apply_dense(plan, A, V, Y, prec=prec), steps, 20)
        y = Y.cpu().numpy()
        Yg = torch.empty_like(V)
        gr = P.BatchGraph(plan, [A], [V], [Yg], prec=prec, scheme=0)
        tg = _time_calls(lambda: gr.replay(), steps, 20)
        yg = Yg.cpu().numpy()
        gr.close()
        p50, p99 = _pcts(ts)
        g50, g99 = _pcts(tg)
        out[name] = {"us_per_eval": {"p50": round(p50 * 1e6, 2), "p99": round(p99 * 1e6, 2)},
                     "graph_us_per_eval": {"p50": round(g50 * 1e6, 2), "p99": round(g99 * 1e6, 2)},
                     "evals_per_s": round(1.0 / min(p50, g50), 1),
                     "rel_err_vs_oracle": matrix.rel_err(y, Yo), "graph_rel_err_vs_oracle": matrix.rel_err(yg, Yo),
                     "rel_err_vs_eigen_Rn": matrix.rel_err(y, Yeig), "rel_err_vs_exp": matrix.rel_err(y, Yexp)}
        out[name]["queue"] = _queue_small(P, plan, A, V, prec, steps, Yo)
    out["exp_bound"] = {"sup_err_n": 2.0 ** -n, "note": "|R_n(x) - e^x| <= 2^-n on x <= 0 (Prop. 2.2); "
                        "relative to |exp(A)v| this allows ~6e-4 here (reading c6)"}
    out["tolerance"] = {"fp64": 1e-12, "mixed": 1e-8}
    plan.close()
    return out


def cfg_dense(n=4096, steps=2, reduced=False):
    """Dense complex Hermitian n x n, V n x 256 complex, degree 16, spectrum U[-50, 0]:
    binary64 against the mixed modes (binary32 LU, 3xTF32 and bf16x3 tensor-core LU updates,
    all with the binary64-accurate tensor-core residual), tensor-pipe rooflines, parity
    against the binary64 path and the eigen closed form."""
    import torch
    import paper_2306_16778_gb300 as P
    import workloads
    from oracle import matrix, scalar
    dev = torch.device("cuda", torch.cuda.current_device())
    w = workloads.dense_hermitian(n=n, nrhs=256)
    Yeig = matrix.eig_apply(w["Q"], w["mu"], w["V"], lambda x: scalar.R_n(x, 16))
    plan = P.Plan(degree=16)
    A, V = (torch.from_numpy(x).to(dev) for x in (w["A"], w["V"]))
    out = {"workload": f"dense Hermitian n={n}, 256 complex RHS, degree 16, spectrum U[-50,0]",
           "steps": {"fp64": 1, "mixed": steps}}
    Ys = {}
    modes = (("fp64", P.EXPM_FP64), ("mixed", P.EXPM_MIXED_FP32), ("mixed_tc", P.EXPM_MIXED_TF32X3),
             ("mixed_bf16x3", P.EXPM_MIXED_BF16X3))
    for name, prec in modes:
        Y = torch.empty_like(V)
        info = P.expm_apply_dense(plan, A, V, Y, prec=prec)
        k = 1 if prec == P.EXPM_FP64 else max(1, steps)
        ts = _time_calls(lambda: P.expm_apply_dense(plan, A, V, Y, prec=prec), k, 0)
        P.expm_profile_enable(plan, True)
        _time_calls(lambda: P.expm_apply_dense(plan, A, V, Y, prec=prec), 1, 0)
        prof = P.expm_profile_read(plan)
        P.expm_profile_enable(plan, False)
        Ys[name] = Y.clone()
        med = statistics.median(ts)
        out[name] = {"s_per_eval": round(med, 5), "evals_per_s": round(1 / med, 4),
                     "latency_s": {"p50": round(_pcts(ts)[0], 5), "p99": round(_pcts(ts)[1], 5)},
                     "refine_sweeps": info.refine_iters_max, "resid_rel": info.resid_rel_max,
                     "growth": info.growth_max_seen, "rel_err_vs_eigen_Rn": matrix.rel_err(Y.cpu().numpy(), Yeig),
                     "kernels_ms": {k_: round(v[1], 3) for k_, v in prof.items()},
                     "kernel_launches": {k_: v[0] for k_, v in prof.items()}}
    if reduced:
        for name, prec, kw in (("reduced", P.EXPM_FP64, {}),
                               ("reduced_mixed", P.EXPM_MIXED_FP32, dict(tol=1e-12, max_refine=2))):
            Y = torch.empty_like(V)
            P.expm_apply_dense_reduced(plan, A, V, Y, prec=prec, **kw)
            ts = _time_calls(lambda: P.expm_apply_dense_reduced(plan, A, V, Y, prec=prec, want_info=False, **kw),
                             max(1, steps), 0)
            Ys[name] = Y.clone()
            out[name] = {"s_per_eval": round(statistics.median(ts), 5),
                         "rel_err_vs_eigen_Rn": matrix.rel_err(Y.cpu().numpy(), Yeig)}
    # tensor-pipe rooflines of the bf16x3 step's tensor-core kernels (algorithmic bf16 flops of
    # the split products / their CUDA-event time; inside a long step: the sustained peak)
    kc, nsys = 256, 16
    burst, sustained, src = _bf16_peak()
    prof = out["mixed_bf16x3"]["kernels_ms"]
    launches = out["mixed_bf16x3"]["kernel_launches"]
    for key, kname, pairs in (("oz_gemm", "oz_gemm_kernel<OzFull>", 28), ("oz_gemm_light", "oz_gemm_kernel<OzLight>", 10)):
        if key in prof:
            fl = 2.0 * pairs * n * (2 * n) * (2 * nsys * kc) * launches[key]
            tf = fl / (prof[key] * 1e-3) / 1e12
            out["roofline_" + key] = {"kernel": kname, "bound": "tensor", "achieved": round(tf, 1), "peak": sustained,
                                      "unit": "TFLOP/s", "frac": round(tf / sustained, 4),
                                      "peak_source": f"{src} bf16 sustained", "launches": launches[key],
                                      "algorithmic": f"{pairs} slice products x 2 x n x 2n x (2 x 16 systems x 256 columns)"}
    if "tc_gemm_bf16x3" in prof:
        fl = sum(2.0 * 8 * r * (2 * r) * (12 * 256) for r in range(n - 256, 0, -256))
        tf = fl / (prof["tc_gemm_bf16x3"] * 1e-3) / 1e12
        out["roofline_tc_lu"] = {"kernel": "tc_gemm_persistent<bf16>", "bound": "tensor", "achieved": round(tf, 1),
                                 "peak": sustained, "unit": "TFLOP/s", "frac": round(tf / sustained, 4),
                                 "peak_source": f"{src} bf16 sustained",
                                 "algorithmic": "sum over panels of 8 pairs x 2 x right x 2 right x 12 x 256"}
    # algorithmic complex-LU rate of the fastest mixed mode: 8 pair LUs x (8/3) n^3 real flops
    best = min(("mixed", "mixed_tc", "mixed_bf16x3"), key=lambda m: out[m]["s_per_eval"])
    out["best_mixed"] = {"mode": best, "speedup_vs_fp64": round(out["fp64"]["s_per_eval"] / out[best]["s_per_eval"], 2),
                         "lu_algorithmic_tflops": round(8 * (8.0 / 3.0) * n ** 3 / out[best]["s_per_eval"] / 1e12, 2),
                         "note": "whole-step rate of the 8 pair LUs' algorithmic flops (the LU is one part of the step)"}
    for name in [m for m, _ in modes[1:]] + (["reduced", "reduced_mixed"] if reduced else []):
        d = (Ys[name] - Ys["fp64"]).abs().pow(2).sum().sqrt() / Ys["fp64"].abs().pow(2).sum().sqrt()
        out[name]["rel_err_vs_fp64"] = float(d)
    out["tolerance"] = {"mixed_vs_fp64": 1e-10, "fp64_vs_closed_form": 1e-12}
    plan.close()
    return out


def run_dense(args):
    print(json.dumps(cfg_dense(args.dense_n, max(1, args.steps), reduced=True)), flush=True)


def run_laplacian2d(args):
    """2D Laplacian 100 (1,-2,1) along both axes on a 1024 x 1024 grid (N = 2^20), 8 RHS, degree 16."""
    import torch
    import paper_2306_16778_gb300 as P
    dev = torch.device("cuda", 0)
    d = 1024
    g = np.random.default_rng(20230629 + 6)
    V = torch.from_numpy(g.standard_normal((d * d, NRHS))).to(dev)
    plan = P.Plan(degree=DEGREE)
    out = {"workload": f"2D Laplacian 100 (1,-2,1) along x and y, {d} x {d} grid, {NRHS} RHS, degree {DEGREE}"}
    Ys = {}
    for name, prec, kw in (("fp64", P.EXPM_FP64, {}), ("mixed", P.EXPM_MIXED_FP32, MIXED_OPTS),
                           ("mixed_f32x2", P.EXPM_MIXED_F32X2, {})):
        Y = torch.empty_like(V)
        P.expm_apply_laplacian2d(plan, d, d, 100.0, -200.0, 100.0, -200.0, V, Y, prec=prec, **kw)
        P.expm_profile_enable(plan, True)
        ts = _time_calls(lambda: P.expm_apply_laplacian2d(plan, d, d, 100.0, -200.0, 100.0, -200.0, V, Y, prec=prec,
                                                          want_info=False, **kw), max(3, args.steps), 2)
        prof = P.expm_profile_read(plan)
        P.expm_profile_enable(plan, False)
        Ys[name] = Y.clone()
        med = statistics.median(ts)
        out[name] = {"ms_per_eval": round(med * 1e3, 4), "evals_per_s": round(1 / med, 2),
                     "kernels_ms": {k: round(v[1] / v[0], 4) for k, v in prof.items()}}
    out["mixed_vs_fp64_rel"] = float((Ys["mixed"] - Ys["fp64"]).norm() / Ys["fp64"].norm())
    from oracle import matrix, scalar
    ref = matrix.laplacian2d_apply(d, d, 100.0, -200.0, 100.0, -200.0, V.cpu().numpy(),
                                   lambda m: scalar.R_n(m, DEGREE))
    for name in Ys:
        out[name]["rel_err_vs_closed_form"] = matrix.rel_err(Ys[name].cpu().numpy(), ref)
    out["tolerance"] = {"fp64": 1e-12, "mixed": 1e-8, "mixed_f32x2": 1e-8}
    out["transforms"] = ("fp64: binary64 products with S; mixed, mixed_f32x2: binary64-accurate slice products "
                         "on the bf16 tensor cores")
    print(json.dumps(out), flush=True)


def _thread_map(fn, items, workers=None):
    from concurrent.futures import ThreadPoolExecutor
    workers = workers or min(16, os.cpu_count() or 1)
    with ThreadPoolExecutor(workers) as ex:
        return list(ex.map(fn, items))


def cfg_batched(count=4096, steps=3):
    """Uneven batch: `count` complex Hermitian instances, n log-uniform in [32, 768], spectra
    U[-30, 0], one complex RHS each, degree 12 (6 pair LUs per instance).  Binary64 and
    binary32 + refinement through expm_apply_batched, and the mixed batch captured into one
    CUDA graph with the autotuned bucket scheme; worst-instance parity against the eigen
    closed form and against the binary64 path."""
    import torch
    import paper_2306_16778_gb300 as P
    import workloads
    from oracle import matrix, scalar
    dev = torch.device("cuda", torch.cuda.current_device())
    w = workloads.uneven_batch(count=count, workers=min(16, os.cpu_count() or 1))
    inst = w["instances"]
    Yeig = _thread_map(lambda i: matrix.eig_apply(i["Q"], i["mu"], i["V"], lambda x: scalar.R_n(x, 12)), inst)
    plan = P.Plan(degree=12)
    As = [torch.from_numpy(i["A"]).to(dev) for i in inst]
    Vs = [torch.from_numpy(i["V"]).to(dev) for i in inst]
    out = {"workload": f"{count} complex Hermitian instances, n log-uniform [32,768], 1 RHS, degree 12",
           "sum_n3": float(np.sum(w["sizes"].astype(float) ** 3)), "steps": {"fp64": 1, "mixed": steps}}

    def worst(Ys, ref):
        return max(matrix.rel_err(y.cpu().numpy(), r) for y, r in zip(Ys, ref))

    Ys = {}
    for name, prec in (("fp64", P.EXPM_FP64), ("mixed", P.EXPM_MIXED_FP32)):
        Y = [torch.empty_like(v) for v in Vs]
        k = 1 if prec == P.EXPM_FP64 else steps
        ts = _time_calls(lambda: P.expm_apply_batched(plan, As, Vs, Y, prec=prec), k, 1)
        Ys[name] = Y
        med = statistics.median(ts)
        out[name] = {"s_per_batch": round(med, 4), "instances_per_s": round(count / med, 2),
                     "worst_rel_err_vs_eigen_Rn": worst(Y, Yeig)}
        P.expm_profile_enable(plan, True)
        P.expm_apply_batched(plan, As, Vs, Y, prec=prec)
        prof = P.expm_profile_read(plan)
        P.expm_profile_enable(plan, False)
        out[name]["kernels_ms"] = {k_: round(v[1], 3) for k_, v in prof.items()}
    out["mixed"]["worst_rel_err_vs_fp64"] = max(
        float((a - b).abs().pow(2).sum().sqrt() / b.abs().pow(2).sum().sqrt()) for a, b in zip(Ys["mixed"], Ys["fp64"]))
    Yg = [torch.empty_like(v) for v in Vs]
    t0 = time.perf_counter()
    gr = P.BatchGraph(plan, As, Vs, Yg, prec=P.EXPM_MIXED_FP32, scheme=-1)
    cap_s = time.perf_counter() - t0
    infos = gr.replay(want_info=True)
    ts = _time_calls(lambda: gr.replay(), steps, 1)
    med = statistics.median(ts)
    gi = gr.info()
    out["mixed_graph"] = {"s_per_batch": round(med, 4), "instances_per_s": round(count / med, 2),
                          "latency_s": {"p50": round(_pcts(ts)[0], 4), "p99": round(_pcts(ts)[1], 4)},
                          "scheme": gi["scheme"], "ms_per_scheme": [round(x, 2) for x in gi["ms_per_scheme"]],
                          "launch_groups": gi["launch_groups"], "capture_and_tune_s": round(cap_s, 2),
                          "bucket_tiles": [[b_["order"], b_["ninst"], b_["tile"], round(b_["ms_tile"][0], 3),
                                            round(b_["ms_tile"][1], 3)] for b_ in gr.buckets()],
                          "refine_sweeps_max": max(i.refine_iters_max for i in infos),
                          "worst_status": max(i.status_worst for i in infos),
                          "worst_rel_err_vs_eigen_Rn": worst(Yg, Yeig),
                          "worst_rel_err_vs_fp64": max(float((a - b).abs().pow(2).sum().sqrt() /
                                                             b.abs().pow(2).sum().sqrt())
                                                       for a, b in zip(Yg, Ys["fp64"]))}
    out["speedup_mixed_graph_vs_fp64"] = round(out["fp64"]["s_per_batch"] / med, 2)
    gr.close()
    # the same graph with the trailing updates of buckets above order 256 on the tensor cores
    Yt = [torch.empty_like(v) for v in Vs]
    gt = P.BatchGraph(plan, As, Vs, Yt, prec=P.EXPM_MIXED_BF16X3, scheme=gi["scheme"])
    infos = gt.replay(want_info=True, check=False)
    tt = _time_calls(lambda: gt.replay(), steps, 1)
    medt = statistics.median(tt)
    out["mixed_tc_graph"] = {"prec": "EXPM_MIXED_BF16X3 (tensor-core trailing updates for padded orders > 256)",
                             "scheme": gi["scheme"], "s_per_batch": round(medt, 4),
                             "instances_per_s": round(count / medt, 2),
                             "latency_s": {"p50": round(_pcts(tt)[0], 4), "p99": round(_pcts(tt)[1], 4)},
                             "refine_sweeps_max": max(i.refine_iters_max for i in infos),
                             "worst_status": max(i.status_worst for i in infos),
                             "worst_rel_err_vs_eigen_Rn": worst(Yt, Yeig)}
    out["speedup_mixed_tc_graph_vs_fp64"] = round(out["fp64"]["s_per_batch"] / medt, 2)
    gt.close()
    out["tolerance"] = {"mixed_vs_closed_form": 1e-8, "fp64_vs_closed_form": 1e-12}
    plan.close()
    return out


def run_batched(args):
    print(json.dumps(cfg_batched(args.batch_count, max(1, args.steps))), flush=True)


def cfg_served(requests=600, fracs=(0.5, 0.9, 1.2), sample=12, all_new=200, max_inflight=8):
    """Served stream: Poisson arrivals, 70 % tridiagonal Laplacian requests (N log-uniform in
    [2^12, 2^20], 1-4 RHS), 30 % dense Hermitian (n log-uniform in [64, 2048], 1-64 RHS,
    spectra U[-40, 0]), degree 12 or 16, operators from a seeded pool of 64 + 64 (resident
    factorizations reused).  Saturation (everything submitted at once) per precision, then
    both precisions at the SAME offered rates (fractions of the binary64 saturation), p50/p99
    of submit -> done and completed requests/s; a sample of each run's requests checked
    against the closed form (dense) or the oracle (tridiagonal); and a run in which every
    request names an operator never seen before (no factorization reused)."""
    import torch
    import paper_2306_16778_gb300 as P
    import workloads
    from oracle import coeffs, matrix, scalar
    dev = torch.device("cuda", torch.cuda.current_device())
    plans = {12: P.Plan(degree=12), 16: P.Plan(degree=16)}
    reqs = workloads.served_stream(requests, rate=1.0)
    keys = sorted({(r["kind"], r["op"]) for r in reqs})
    opdata = dict(zip(keys, _thread_map(lambda k: workloads.served_operator(*k), keys)))
    bufs = []
    for r in reqs:
        od = opdata[(r["kind"], r["op"])]
        n = od["d"].shape[0] if r["kind"] == "tridiag" else od["A"].shape[0]
        bufs.append(torch.from_numpy(workloads.request_rhs(n, r["nrhs"], r["seed"], r["kind"] == "dense")).to(dev))
    dev_ops = {}
    for k, od in opdata.items():
        dev_ops[k] = tuple(torch.from_numpy(x).to(dev) for x in ((od["d"], od["e"]) if k[0] == "tridiag" else (od["A"],)))
    precs = {"fp64": (P.EXPM_FP64, P.EXPM_FP64), "mixed": (P.EXPM_MIXED_FP32, P.EXPM_MIXED_FP32)}

    def sub_opts(kind, ptri, pden):
        if kind == "tridiag":
            return dict(prec=ptri, **(MIXED_OPTS if ptri == P.EXPM_MIXED_FP32 else {}))
        return dict(prec=pden)

    def make_server(fresh):
        server = P.Server(hbm_budget_bytes=64 << 30, max_inflight=max_inflight)
        ids = {}
        for i, r in enumerate(reqs):
            k = (r["kind"], r["op"])
            key = (k, i) if fresh else k
            if key not in ids:
                t = dev_ops[k]
                ids[key] = server.register_tridiag(*t) if k[0] == "tridiag" else server.register_dense(t[0])
        return server, [ids[((r["kind"], r["op"]), i) if fresh else (r["kind"], r["op"])] for i, r in enumerate(reqs)]

    def run(server, oids, ptri, pden, rate, n_req):
        outs = [torch.empty_like(V) for V in bufs[:n_req]]
        torch.cuda.synchronize()
        gaps = workloads.rng(77).exponential(1.0 / rate, n_req) if rate else np.zeros(n_req)
        t_start = time.perf_counter()
        arrival = t_start + np.cumsum(gaps)
        lat, pending, i = [], {}, 0
        while i < n_req or pending:
            now = time.perf_counter()
            while i < n_req and arrival[i] <= now:
                r = reqs[i]
                t = server.submit(oids[i], plans[r["degree"]], bufs[i], outs[i], **sub_opts(r["kind"], ptri, pden))
                pending[t] = i
                i += 1
            for t in list(pending):
                res = server.poll(t)
                if res is not None:
                    assert res[0] == 0, ("request failed", res[0])
                    del pending[t]
                    lat.append(res[2][3] - res[2][0])
        wall = time.perf_counter() - t_start
        lat.sort()
        return {"offered_rps": round(rate, 2) if rate else None, "requests": n_req,
                "evals_per_s": round(n_req / wall, 2), "p50_ms": round(1e3 * lat[len(lat) // 2], 3),
                "p99_ms": round(1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))], 3)}, outs

    def check(outs, n_req):
        idx = list(range(0, n_req, max(1, n_req // sample)))[:sample]

        def one(i):
            r = reqs[i]
            od = opdata[(r["kind"], r["op"])]
            V = bufs[i].cpu().numpy()
            if r["kind"] == "dense":
                ref = matrix.eig_apply(od["Q"], od["mu"], V, lambda x: scalar.R_n(x, r["degree"]))
            else:
                ref, _ = matrix.apply_tridiag(od["d"], od["e"], V, coeffs.theta(r["degree"]),
                                              coeffs.residues(r["degree"]))
            return matrix.rel_err(outs[i].cpu().numpy(), ref)
        errs = _thread_map(one, idx)
        return {"checked": len(idx), "worst_rel_err": max(errs)}

    out = {"workload": "served stream: 70% Laplacian N log-uniform [2^12,2^20] 1-4 RHS, 30% dense Hermitian "
                       "n log-uniform [64,2048] 1-64 RHS, degree 12/16, operator pool 64+64",
           "requests_per_run": requests, "max_inflight": max_inflight,
           "budget": f"{requests} requests per rate (rates {list(fracs)} x the binary64 saturation), "
                     f"{sample} requests per run checked, {all_new} requests in the all-new-operator runs"}
    sat = {}
    for name, (ptri, pden) in precs.items():
        server, oids = make_server(False)
        run(server, oids, ptri, pden, 0, min(requests, 200))  # warm: factorizations built and cached
        res, outs = run(server, oids, ptri, pden, 0, requests)
        sat[name] = res["evals_per_s"]
        out[name] = {"saturation": dict(res, accuracy=check(outs, requests)), "rates": {}}
        server.close()
    for f in fracs:
        rate = f * sat["fp64"]
        for name, (ptri, pden) in precs.items():
            server, oids = make_server(False)
            run(server, oids, ptri, pden, 0, min(requests, 200))
            res, outs = run(server, oids, ptri, pden, rate, requests)
            out[name]["rates"][f"{f:g}x_fp64_sat"] = dict(res, accuracy=check(outs, requests))
            server.close()
    out["all_new_operators"] = {}
    n_new = min(all_new, requests)
    for name, (ptri, pden) in precs.items():
        server, oids = make_server(True)
        res, outs = run(server, oids, ptri, pden, 0.5 * sat["fp64"], n_new)
        out["all_new_operators"][name] = dict(res, accuracy=check(outs, n_new))
        server.close()
    out["tolerance"] = {"fp64": 1e-12, "mixed": 1e-8}
    for p_ in plans.values():
        p_.close()
    return out


def run_served(args):
    print(json.dumps(cfg_served(args.served_requests, fracs=(0.25, 0.5, 0.75, 0.9, 1.0, 1.2), sample=24,
                                all_new=min(1000, args.served_requests))), flush=True)


def main():
    args = parse()
    if args.peaks:
        run_peaks()
        return
    if args.workload == "laplacian2d":
        return run_laplacian2d(args)
    if args.workload == "dense":
        run_dense(args)
        return
    if args.workload == "batched":
        run_batched(args)
        return
    if args.workload == "served":
        run_served(args)
        return
    if args.workload == "dense_small":
        print(json.dumps({"workload": "dense_small", **cfg_dense_small(args.steps)}), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
