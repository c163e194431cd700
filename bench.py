"""Benchmark of the RPCholesky-preconditioned CG hot path on one GB300.

Workload (the configuration the headline metric is quoted on): full-data KRR
with mixed precision and iterative refinement -- N = 100000 points, d = 16,
x uniform on [0,1]^16 with 5% of the rows duplicated plus 1e-6 jitter,
Gaussian sigma = 0.5, mu = 1e-7 (shift mu N), 4 right-hand sides
y_r = sum_j cos(2 pi r x_j) + noise, RPCholesky rank 1000 (B = 100), inner
float32 PCG with float64 refinement to relative residual 1e-6.  Inputs are
synthetic (seeded), resident in HBM before the timed region.

One step = the whole hot path once: krr_rpcholesky (pivot sampling, column
evaluation, Schur update, block Cholesky, triangular solve, residual
downdate) + krr_pcg_solve (Woodbury core, fused products, preconditioner
applies, PCG updates, float64 refinement residuals).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank runs an independent replica of the step
(the method has no data-parallel exchange at this size); value = entries of
all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PCG time-to-1e-6 residual & kernel evals/s vs plain FP64 path; p50/p99 latency"
UNIT = "kernel_evals/s"
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--n", type=int, default=100_000, help="points (workload size)")
    ap.add_argument("--fp64-path", action="store_true",
                    help="also time the plain float64 path (one step, slow)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--product-path", default="tensor", choices=["tensor", "fma", "mma_sync"],
                    help="float32 product: inner products on the tensor cores, or all FMA")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end step")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the short runs of the other configurations (c1, c3, c4)")
    ap.add_argument("--no-pcg-graphs", action="store_true",
                    help="step the PCG iterations one launch at a time (no CUDA graphs)")
    ap.add_argument("--kmv-prec", default="mixed", choices=["mixed", "ff"],
                    help="kmv workload: the float32 product (mixed) or the float-float one")
    ap.add_argument("--product-variant", type=int, default=0,
                    help="force an epilogue variant of the tcgen05 product (0: autotuned "
                         "or default)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the product's default tile instead of tuning it in the warm-up")
    ap.add_argument("--no-fp64", action="store_true",
                    help="skip the composed plain float64 GPU path (about 45 s)")
    ap.add_argument("--workload", default="c2",
                    choices=["c1", "c2", "c3", "c4", "serving", "kmv"],
                    help="c2: one RPCholesky + refined PCG solve per step (headline); "
                         "c1: the plain float64 solve; c3: the batched 8-setting x 2-shift "
                         "product; c4: KRILL build + solve; "
                         "serving: a Poisson stream of solve requests through the server")
    ap.add_argument("--requests", type=int, default=512, help="serving: stream length")
    ap.add_argument("--n-max", type=int, default=200_000,
                    help="serving: largest N of the log-uniform range [2000, n_max]")
    ap.add_argument("--rates", default="0.8",
                    help="serving: Poisson arrival rates as fractions of the closed-loop "
                         "throughput measured first on the same stream (comma separated)")
    ap.add_argument("--slots", type=int, default=32, help="serving: max concurrent solves")
    ap.add_argument("--iters-per-step", type=int, default=4, help="serving: PCG iterations/step")
    ap.add_argument("--serving-log", default="",
                    help="serving: write one JSON line per request to this file")
    ap.add_argument("--no-serving", action="store_true",
                    help="c2: skip the bounded serving stream reported beside the headline")
    return ap.parse_args()


def dist_setup(n_gpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        return dist, rank, world
    torch.cuda.set_device(0)
    return None, 0, 1


def aggregate_ranks(dist, total_ms: float, work: float, device="cpu"):
    """Whole-job figures of the replicas: the slowest rank's time and the work
    of all ranks (identity without a process group)."""
    if dist is None:
        return total_ms, work
    import torch
    tmax = torch.tensor([total_ms], dtype=torch.float64, device=device)
    tsum = torch.tensor([work], dtype=torch.float64, device=device)
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(tsum[0])


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# float32 product, mean of three launches from one ncu capture of this bench's
# default workload, keyed by (path, kernel, N, d, m, tile): the autotuned
# column splits of the FMA and mma.sync kernels, the epilogue variant of the
# tcgen05 kernel.  Any other shape or tile has no capture and reports None; a
# change to the kernel invalidates the entry until it is captured again.
KMV32_TRAFFIC = {("fma", 0, 100_000, 16, 4, 50): 8_748_117 + 16_672_768,
                 ("tensor", 0, 100_000, 16, 4, 1): 22_511_616 + 0,
                 ("tensor", 0, 100_000, 16, 4, 3): 22_520_320 + 0}

# Register-operand mma.sync (m16n8k16, f16 inputs, f32 accumulator) measured by
# this repository's probe on this machine's GB300 (independent MMAs, 2-8 CTAs of
# 256 threads per SM): the peak of the mma.sync kernel's tensor pipe.
MMA_SYNC_F16_TFLOPS = 606.0


def kmv32_traffic(path, w, tile):
    return KMV32_TRAFFIC.get((path, w.kernel, w.N, w.d, w.m, tile))


def measured_peak(key, fallback):
    """A peak from MEASURED_PEAKS.json beside this file, else the fallback."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)),
                               "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key]), "measured"
    except (OSError, KeyError, ValueError):
        return fallback, "fallback"


def tc5_mmas(d):
    """MMAs (K = 16 each) per entry of the tcgen05 product: (L_i, H_j), (H_i, L_j)
    and (H_i, H_j) per 16-coordinate block, plus one for c_i + c_j when c has a
    block of its own (d mod 16 = 0 or > 10)."""
    nh = (d + 15) // 16
    csep = 1 if (d % 16 == 0 or d % 16 > 10) else 0
    return 3 * nh + csep


def product_roofline(path, w, per_launch_ms, tile, sm_max):
    """Roofline of the float32 product: its roofline time is the largest of the
    ideal times of the pipes it uses (FP32 ops, MUFU ops, tensor ops, each at
    its peak) and frac = that time / the measured launch time.

    tcgen05 path (default): 2 x 16 flop per MMA per entry on the tensor cores
    (tc5_mmas), 2m flop on the FP32 pipe (the m FMAs; c_i + c_j is folded into
    the MMAs) and 1 ex2 (Matern 2) on the MUFU; tensor peak = the measured
    dense 16-bit peak, sustained.  mma.sync path: 96 flop per 16 coordinates
    (three fp16 MMAs), 1 + 2m flop on the FP32 pipe (c_i + c_j, m FMA), tensor
    peak = the measured mma.sync f16 rate.  FMA path: (2d + 1 + 2m) flop per
    entry (d FMA distance, c_i + c_j, m FMA).  FP32 peak: 152 SM x 128 lanes x
    2 flop x the maximum SM clock; MUFU: 32 ex2 per clock per SM (measured)."""
    entries = float(w.N) * w.N
    sec = per_launch_ms / 1e3
    traffic = kmv32_traffic(path, w, tile)
    mufu_per_entry = 2 if w.kernel == 2 else 1
    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12          # TFLOP/s
    mufu_peak = 152 * 32 * sm_max * 1e6 / 1e12                # T ex2/s
    tensor_path = path in ("tensor", "mma_sync") and w.kernel != 1
    if tensor_path and path == "tensor":
        tc_flop = 2 * 16 * tc5_mmas(w.d)
        fp32_flop = 2 * w.m
        tc_peak, basis = measured_peak("bf16_tflops_sustained", 1700.0)
        basis = (f"dense 16-bit tensor peak, {basis} (bf16 cuBLAS, sustained; fp16 has the "
                 "same nominal rate)")
        kernel = "kmvtc5_kernel (tcgen05 tensor-core product, fp16 two-half split, TMEM)"
    elif tensor_path:
        tc_flop = 2 * 16 * 3 * ((w.d + 15) // 16)
        fp32_flop = 1 + 2 * w.m
        tc_peak = MMA_SYNC_F16_TFLOPS
        basis = "register-operand mma.sync f16 m16n8k16, measured by this repository's probe"
        kernel = "kmvtc_kernel (mma.sync tensor-core product, fp16 two-half split)"
    else:
        tc_flop = 0
        fp32_flop = 2 * w.d + 1 + 2 * w.m
        tc_peak, basis = None, None
        kernel = "kmv32_kernel (fused float32 product)"
    pipes = {"fp32": {"ideal_ms": fp32_flop * entries / fp32_peak / 1e9,
                      "achieved": fp32_flop * entries / sec / 1e12, "peak": fp32_peak,
                      "unit": "TFLOP/s", "per_entry": fp32_flop},
             "mufu": {"ideal_ms": mufu_per_entry * entries / mufu_peak / 1e9,
                      "achieved": mufu_per_entry * entries / sec / 1e12, "peak": mufu_peak,
                      "unit": "T ex2/s", "per_entry": mufu_per_entry}}
    if tensor_path:
        pipes["tensor"] = {"ideal_ms": tc_flop * entries / tc_peak / 1e9,
                           "achieved": tc_flop * entries / sec / 1e12, "peak": tc_peak,
                           "unit": "TFLOP/s", "per_entry": tc_flop, "peak_basis": basis}
    for p in pipes.values():
        p["frac"] = p["achieved"] / p["peak"]
    top = max(pipes, key=lambda k: pipes[k]["ideal_ms"])
    t = pipes[top]
    return {"kernel": kernel, "bound": "tensor" if top == "tensor" else "alu", "pipe": top,
            "achieved": t["achieved"], "peak": t["peak"], "unit": t["unit"],
            "frac": t["ideal_ms"] / per_launch_ms, "traffic": traffic,
            "peak_basis": t.get("peak_basis",
                                f"152 SM x {'128 FP32 lanes x 2 flop' if top == 'fp32' else '32 ex2'}"
                                f" x {sm_max:.0f} MHz (max SM clock); derived from unit counts"),
            "roofline_ms": t["ideal_ms"], "measured_ms": per_launch_ms,
            "entries_per_launch": entries, "pipes": pipes}


def entries_rpcholesky(N, k):
    # Alg. 3 evaluates the diagonal and one kernel column per pivot
    return float(N) * (k + 1)


def fp64_path_composed(K, w, X, Y, mixed_step_s):
    """The plain float64 GPU path on the same inputs and seed, composed from
    live measurements (a whole float64 solve at N = 1e5 takes minutes):
    RPCholesky time + a float64 PCG whose products are the float-float product
    (float64-accurate entries: the same iterates as the float64 products up to
    rounding), with the float-float product time replaced by the measured
    float64 product time per launch times the number of products."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    f = K.krr_rpcholesky(X, w.kernel, w.sigma, w.k, w.block, seed=w.seed)
    torch.cuda.synchronize()
    t_rpc = time.perf_counter() - t0
    K.krr_set_profiling(True)
    t1 = time.perf_counter()
    _, info = K.krr_pcg_solve(X, w.kernel, w.sigma, Y, w.mu, f, tol=w.tol, prec="ff")
    torch.cuda.synchronize()
    t_ff = time.perf_counter() - t1
    K.krr_set_profiling(False)
    f.free()
    gen = torch.Generator(device=X.device).manual_seed(11)
    V = torch.randn((w.m, w.N), dtype=torch.float64, device=X.device, generator=gen)
    stream = torch.cuda.current_stream()
    times = []
    for _ in range(2):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        K.krr_kmatvec(X, w.kernel, w.sigma, w.lam, V, prec="fp64")
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    kmv64_s = times[-1]
    n_prod = int(info["kmvff_launches"])
    ff_prod_s = info["kmvff_ms"] / 1e3
    composed = t_rpc + (t_ff - ff_prod_s) + n_prod * kmv64_s
    return {"time_to_tol_s": composed, "kind": "composed",
            "iters": info["iters"], "status": info["status"],
            "rel_residual_fp64": info["rel_residual"], "products": n_prod,
            "kmv64_ms_per_launch": kmv64_s * 1e3,
            "float_float_pcg_s": t_ff, "rpcholesky_s": t_rpc,
            "speedup_mixed_vs_fp64": composed / mixed_step_s,
            "composition": "RPCholesky + float64 PCG with float-float products (same iterates "
                           "to rounding), its product time replaced by products x the measured "
                           "float64 product launch; all measured in this run on the same inputs"}


def run_native(args):
    import torch
    import paper_2304_12465_gb300 as K
    from inputs import make_c2_mixed

    dist, rank, world = dist_setup(args.gpus)
    K.load()
    K.krr_set_product_path(args.product_path)
    K.krr_set_pcg_graphs(not args.no_pcg_graphs)
    w = make_c2_mixed(n=args.n)
    dev = torch.device("cuda", torch.cuda.current_device())
    X = torch.from_numpy(w.X).to(dev)
    Y = torch.from_numpy(w.Y).to(dev)
    alpha = torch.empty_like(Y)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(profile=False):
        f = K.krr_rpcholesky(X, w.kernel, w.sigma, w.k, w.block, seed=w.seed)
        a, info = K.krr_pcg_solve(X, w.kernel, w.sigma, Y, w.mu, f, tol=w.tol, prec="mixed",
                                  out=alpha)
        rank_ = f.rank
        f.free()
        if info["status"] != "KRR_OK":
            raise RuntimeError(f"solve did not converge: {info}")
        info["entries"] = entries_rpcholesky(w.N, rank_) + info["kernel_entries"]
        return info

    # the product's tile (epilogue variant / column splits) is tuned during the
    # first warm-up step
    K.krr_set_autotune(not args.no_autotune)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler(torch.cuda.current_device())
    K.krr_set_profiling(True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = K.krr_launch_count()
    step_ms, infos = [], []
    for _ in range(args.steps):
        flush.zero_()                       # L2 flush between timed steps
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos.append(step())
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    launches = K.krr_launch_count() - launches0
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    K.krr_set_profiling(False)

    total_ms = float(sum(step_ms))
    entries = float(sum(i["entries"] for i in infos))
    total_ms, entries = aggregate_ranks(dist, total_ms, entries, dev)
    value = entries / (total_ms / 1e3)

    # roofline of the dominant kernel: the float32 fused product
    kmv_ms = sum(i["kmv_ms"] for i in infos)
    kmv_n = sum(i["kmv_launches"] for i in infos)
    per_launch_ms = kmv_ms / max(kmv_n, 1)
    sm_max = clk.get("sm_max_mhz") or 2070.0
    variant_ms = None
    if args.product_path == "tensor":
        tile, variant_ms = K.krr_autotune_variant(w.kernel, w.d, w.m, w.N)
    else:
        tile = K.krr_autotune_choice(w.kernel, w.d, w.m, w.N)
    kmv64_ms = sum(i["kmv64_ms"] for i in infos)
    kmv64_n = sum(i["kmv64_launches"] for i in infos)
    kmvff_ms = sum(i["kmvff_ms"] for i in infos)
    kmvff_n = sum(i["kmvff_launches"] for i in infos)

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": f"full-data KRR, N={w.N}, d={w.d}, 5% near-duplicates, "
                               f"Gaussian sigma={w.sigma}, mu={w.mu}, m={w.m} RHS, "
                               f"RPCholesky k={w.k} B={w.block}, mixed precision + float64 "
                               f"refinement, tol={w.tol}",
                   "N": w.N, "d": w.d, "m": w.m, "k": w.k, "block": w.block,
                   "kernel": "gaussian", "sigma": w.sigma, "mu": w.mu, "tol": w.tol,
                   "l2": "flushed between timed steps (512 MiB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "time_to_tol_s": total_ms / args.steps / 1e3,
        "pcg": {"iters": [i["iters"] for i in infos],
                "outer_refinements": [i["outer_refinements"] for i in infos],
                "rel_residual_fp64": [i["rel_residual"] for i in infos],
                "t_build_core_s": [i["t_build_s"] for i in infos],
                "t_solve_s": [i["t_solve_s"] for i in infos],
                "kmv32_ms_per_launch": per_launch_ms, "kmv32_launches": kmv_n,
                "kmv64_ms_per_launch": kmv64_ms / max(kmv64_n, 1),
                "kmv64_launches": kmv64_n,
                "kmvff_ms_per_launch": kmvff_ms / max(kmvff_n, 1),
                "kmvff_launches": kmvff_n,
                "graph_replays": [i["graph_replays"] for i in infos],
                "host_checks": [i["host_checks"] for i in infos],
                "kmv32_tile_autotuned": tile,
                "kmv32_tile_kind": ("epilogue variant" if args.product_path == "tensor"
                                    else "column splits"),
                "kmv32_variant_ms": variant_ms,
                "product_path": args.product_path},
        "roofline": product_roofline(args.product_path, w, per_launch_ms, tile, sm_max),
        "clocks": clk,
        "gpu_launches": int(launches),
    }
    if not args.no_serving and world == 1:
        # a bounded sample of the serving workload: the first 32 requests of the
        # serving stream, closed loop, then Poisson arrivals at 0.8x its throughput
        from inputs import make_serving_stream
        sreqs = make_serving_stream(32, seed=4 + rank)
        closed, runs = serving_protocol(K, sreqs, [0.8], 32, 4)
        result["serving"] = {"requests": 32, "arrival_rate": "0.8 x closed-loop throughput",
                             "solves_per_s": runs["0.8x"]["solves_per_s"],
                             "latency_s": runs["0.8x"]["latency_s"],
                             "closed_loop_solves_per_s": closed["solves_per_s"],
                             "status": runs["0.8x"]["status"],
                             "escalations": runs["0.8x"]["escalations"]}

    if rank == 0 and world == 1 and not args.no_fp64 and not args.fp64_path:
        result["fp64_path"] = fp64_path_composed(K, w, X, Y, total_ms / args.steps / 1e3)

    if rank == 0 and world == 1 and args.fp64_path:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f = K.krr_rpcholesky(X, w.kernel, w.sigma, w.k, w.block, seed=w.seed)
        a64, i64 = K.krr_pcg_solve(X, w.kernel, w.sigma, Y, w.mu, f, tol=w.tol, prec="fp64")
        torch.cuda.synchronize()
        t64 = time.perf_counter() - t0
        f.free()
        result["fp64_path"] = {"time_to_tol_s": t64, "iters": i64["iters"],
                               "status": i64["status"],
                               "speedup_mixed_vs_fp64": t64 / (total_ms / args.steps / 1e3)}

    if rank == 0 and world == 1 and not args.no_configs:
        # the other configurations, short runs (3 warm-up and 2 timed steps each):
        # plain float64 (c1), the batched product (c3), KRILL (c4)
        result["configs"] = {}
        for name in ("c1", "c3", "c4"):
            r = measure_config(K, name, 2, 3)
            r.pop("metric", None)
            result["configs"][name] = r

    # end to end through the C ABI with host buffers (copies inside the region)
    if args.no_e2e:
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            result["cpu_baseline"] = cpu_baseline(w)
        if rank == 0:
            print(json.dumps(result), flush=True)
        if dist:
            dist.destroy_process_group()
        return
    Xh, Yh = w.X, w.Y
    alpha_h = np.empty_like(Yh)
    t0 = time.perf_counter()
    f = K.krr_rpcholesky(Xh, w.kernel, w.sigma, w.k, w.block, seed=w.seed)
    a_h, info_h = K.krr_pcg_solve(Xh, w.kernel, w.sigma, Yh, w.mu, f, tol=w.tol, prec="mixed",
                                  out=alpha_h)
    t_e2e = time.perf_counter() - t0
    e2e_entries = entries_rpcholesky(w.N, f.rank) + info_h["kernel_entries"]
    f.free()
    result["e2e"] = {"value": e2e_entries * world / t_e2e, "unit": UNIT,
                     "h2d_bytes_per_step": int(2 * Xh.nbytes + Yh.nbytes),
                     "d2h_bytes_per_step": int(alpha_h.nbytes),
                     "seconds_per_step": t_e2e}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(w)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist:
        dist.destroy_process_group()


def serve_stream(K, reqs, rate, slots, iters_per_step, seed=5, log=""):
    """Runs a request stream through the server: request i arrives at the i-th
    point of a Poisson process of the given rate (all at once for rate 0) and
    is submitted when the server clock passes its arrival time.  Inputs are
    host arrays (copied to the device by the server), results land in host
    arrays; latency = completion - arrival."""
    from inputs import make_serving_request
    data = [make_serving_request(r) for r in reqs]
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, len(reqs)) if rate > 0 else np.zeros(len(reqs))
    arrive = np.cumsum(gaps) - gaps[0]
    launches0 = K.krr_launch_count()
    with K.KrrServer(max_slots=slots, iters_per_step=iters_per_step) as srv:
        t0 = srv.clock()
        nxt, done = 0, []
        while True:
            now = srv.clock() - t0
            while nxt < len(reqs) and arrive[nxt] <= now:
                r = reqs[nxt]
                X, Y = data[nxt]
                rid = srv.submit(X, r["kernel"], r["sigma"], Y, r["mu"], r["k"], tol=1e-6,
                                 maxit=5000, seed=r["seed"])
                assert rid == nxt
                nxt += 1
            left = srv.step()
            done += srv.poll()
            if nxt == len(reqs) and left == 0:
                break
        t_end = srv.clock() - t0
        stats = srv.stats()
    launches = K.krr_launch_count() - launches0
    if log:
        with open(log, "w") as fh:
            for d in sorted(done, key=lambda d: d["id"]):
                r = reqs[d["id"]]
                fh.write(json.dumps({**{k: r[k] for k in ("N", "d", "kernel", "sigma", "mu", "m",
                                                          "k", "seed")},
                                     **{k: v for k, v in d.items() if k != "alpha"},
                                     "arrive": float(arrive[d["id"]])}) + "\n")
    lat = np.array([d["t_done"] - t0 - arrive[d["id"]] for d in done])
    wait = np.array([d["t_admit"] - t0 - arrive[d["id"]] for d in done])
    build = np.array([d["t_built"] - d["t_admit"] for d in done])
    status = {}
    for d in done:
        status[d["status_name"]] = status.get(d["status_name"], 0) + 1
    entries = float(sum(d["kernel_entries"] for d in done))
    return {
        "requests": len(reqs), "wall_s": t_end,
        "solves_per_s": len(reqs) / t_end,
        "kernel_evals_per_s": entries / t_end,
        "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                      "mean": float(lat.mean()), "max": float(lat.max())},
        "queue_wait_s": {"p50": float(np.percentile(wait, 50)),
                         "p99": float(np.percentile(wait, 99))},
        "build_s": {"p50": float(np.percentile(build, 50)),
                    "p99": float(np.percentile(build, 99))},
        "status": status,
        "iters": {"p50": float(np.median([d["iters"] for d in done])),
                  "max": int(max(d["iters"] for d in done))},
        "rel_residual_max": float(max(d["rel_residual"] for d in done)),
        "max_concurrent": stats["max_concurrent"], "steps": stats["steps"],
        "step_device_s": stats["step_ms"] / 1e3, "build_thread_s": stats["build_s"],
        "escalations": stats["escalations"], "escalate_thread_s": stats["escalate_s"],
        "escalated_ok": sum(1 for d in done if d["escalated"] and d["status"] == 0),
        "peak_reserved_gb": stats["peak_reserved_bytes"] / 1e9,
        "gpu_launches": int(launches),
        "arrival_rate_per_s": rate if rate > 0 else "all at t=0",
        "slots": slots, "iters_per_step": iters_per_step,
        "h2d_bytes": int(sum(a.nbytes + b.nbytes for a, b in data)),
        "d2h_bytes": int(sum(8 * r["m"] * r["N"] for r in reqs)),
    }


def serving_protocol(K, reqs, rates, slots, iters_per_step, log=""):
    """Closed loop (every request at time 0) to measure the stream's
    throughput, then Poisson arrivals at the given fractions of it."""
    closed = serve_stream(K, reqs, 0.0, slots, iters_per_step)
    runs = {}
    for f in rates:
        rho = f * closed["solves_per_s"]
        runs[f"{f:g}x"] = serve_stream(K, reqs, rho, slots, iters_per_step,
                                       log=log if f == rates[0] else "")
    return closed, runs


def run_serving(args):
    """Serving workload: a Poisson stream of KRR solve requests (N log-uniform
    in [2000, 200000], d in {4, 8, 16, 32}, three kernels, sigma log-uniform
    in [0.3, 3], mu log-uniform in [1e-8, 1e-4], 1-16 right-hand sides,
    RPCholesky k = min(1000, N/10), x ~ N(0, I)), tol 1e-6.  The stream runs
    closed loop first; its throughput sets the Poisson rates; value = solves/s
    and p50/p99 latency at the first rate."""
    import torch
    import paper_2304_12465_gb300 as K
    from inputs import make_serving_stream

    dist, rank, world = dist_setup(args.gpus)
    K.load()
    rates = [float(x) for x in args.rates.split(",")]
    reqs = make_serving_stream(args.requests, seed=4 + rank, n_range=(2000, args.n_max))
    warm = make_serving_stream(max(args.warmup, 1), seed=1000 + rank, n_range=(2000, 20000))
    serve_stream(K, warm, 0.0, args.slots, args.iters_per_step)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    if dist:
        dist.barrier()
    clocks.start()
    closed, runs = serving_protocol(K, reqs, rates, args.slots, args.iters_per_step,
                                    log=args.serving_log)
    clk = clocks.stop()
    head = runs[f"{rates[0]:g}x"]
    wall = head["wall_s"]
    wall, _ = aggregate_ranks(dist, wall * 1e3, 0.0, "cuda")
    wall /= 1e3
    value = world * args.requests / wall
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.requests, "warmup": len(warm), "ms_per_step": wall / args.requests * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"serving: Poisson stream of {args.requests} KRR solve "
                                   f"requests, N log-uniform [2000, {args.n_max}], "
                                   "d in {4,8,16,32}, x ~ N(0, I), "
                                   "Gaussian/Laplace/Matern-5/2, sigma log-uniform [0.3, 3], "
                                   "mu log-uniform [1e-8, 1e-4], 1-16 RHS, "
                                   "k = min(1000, N/10), tol 1e-6; arrival rate "
                                   f"{rates[0]:g} x the closed-loop throughput",
                       "l2": "inputs larger than L2 (each request's points, factor and "
                             "state are distinct)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "latency_s": head["latency_s"],
            "serving": {"closed_loop": closed, **runs},
            "e2e": {"value": value, "unit": "solves/s",
                    "h2d_bytes_per_step": head["h2d_bytes"] // args.requests,
                    "d2h_bytes_per_step": head["d2h_bytes"] // args.requests},
            "clocks": clk, "gpu_launches": head["gpu_launches"],
        }), flush=True)
    if dist:
        dist.destroy_process_group()


def run_config(args):
    """The other configurations (--workload c1|c3|c4) as their own bench line."""
    import paper_2304_12465_gb300 as K

    dist, rank, world = dist_setup(args.gpus)
    K.load()
    res = measure_config(K, args.workload, args.steps, args.warmup, dist, rank, world)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if dist:
        dist.destroy_process_group()


def measure_config(K, workload, steps, warmup, dist=None, rank=0, world=1):
    """The other configurations, one step each:
    c1 -- plain float64 path: RPCholesky (k = 200, B = 20) + float64 PCG to 1e-10,
          N = 4096, d = 8;
    c3 -- the batched product of 8 (kernel, sigma) settings x 2 shifts sharing one
          tile generation, N = 500000, d = 8 (the product a batched PCG iteration runs);
    c4 -- KRILL: krill_build (sparse sign sketch, Gram, Cholesky) + krill_solve
          (refined PCG to 1e-6), N = 2e6, d = 20, k = 2000 centers.
    value = kernel entries evaluated per second over the step.  Returns the
    result (rank 0) or None."""
    import torch
    from inputs import make_c1_plain_fp64, make_c3_batched, make_c4_krill

    dev = torch.device("cuda", torch.cuda.current_device())
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    extra = {}
    if workload == "c1":
        w = make_c1_plain_fp64()
        X, Y = torch.from_numpy(w.X).to(dev), torch.from_numpy(w.Y).to(dev)

        def step():
            f = K.krr_rpcholesky(X, w.kernel, w.sigma, w.k, w.block, seed=w.seed)
            a, info = K.krr_pcg_solve(X, w.kernel, w.sigma, Y, w.mu, f, tol=w.tol, prec="fp64")
            rk = f.rank
            f.free()
            if info["status"] != "KRR_OK":
                raise RuntimeError(f"solve did not converge: {info}")
            return entries_rpcholesky(w.N, rk) + info["kernel_entries"], info
        desc = (f"plain float64 KRR, N={w.N}, d={w.d}, Gaussian sigma={w.sigma}, mu={w.mu}, "
                f"RPCholesky k={w.k} B={w.block}, float64 PCG to {w.tol}")
        dtype = "f64"
    elif workload == "c3":
        w = make_c3_batched()
        X = torch.from_numpy(w.X).to(dev)
        kerns = [k for k, _ in w.settings]
        sigmas = [sg for _, sg in w.settings]
        ms = len(w.mus)
        lams = [mu * w.N for _ in w.settings for mu in w.mus]
        V = torch.from_numpy(np.random.default_rng(0).standard_normal(
            (len(w.settings) * ms, w.N))).to(dev)

        def step():
            K.krr_kmatvec_batched(X, kerns, sigmas, lams, V)
            return float(len(w.settings)) * w.N * w.N, {}
        desc = (f"batched product, N={w.N}, d={w.d}, Matern-5/2 and Laplace at sigma in "
                f"{{0.5,1,2,4}} (8 settings) x mu in {w.mus} sharing one tile generation")
        dtype = "f32"
        extra["entries_counted"] = "N^2 kernel evaluations per setting (8 per product)"
        # per pair of points: d differences, d squares-and-adds, d |.|-adds; per
        # Matern setting sqrt, scale, ex2, 2-FMA polynomial, product (6 flop +
        # 2 MUFU); per Laplace setting scale + ex2 (1 flop + 1 MUFU); 2 FMA per
        # shift column (4 flop) for every setting
        nmat = sum(1 for k in kerns if k == 2)
        nlap = len(kerns) - nmat
        flop_pair = 4 * w.d + nmat * 6 + nlap * 1 + len(kerns) * 2 * ms * 2
        mufu_pair = 2 * nmat + nlap
        extra["roofline_model"] = {"flop_per_pair": flop_pair, "mufu_per_pair": mufu_pair}
    else:
        w = make_c4_krill()
        X, Y = torch.from_numpy(w.X).to(dev), torch.from_numpy(w.Y).to(dev)
        centers = torch.from_numpy(w.centers).to(dev)

        def step():
            P = K.krill_build(X, w.kernel, w.sigma, centers, w.mu, seed=w.seed)
            b, info = K.krill_solve(P, Y, w.tol)
            P.free()
            if info["status"] != "KRR_OK":
                raise RuntimeError(f"solve did not converge: {info}")
            zeta = max(1, math.ceil(math.log(w.k + 1)))
            return zeta * float(w.N) * w.k + info["kernel_entries"], info
        desc = (f"restricted KRR (KRILL), N={w.N}, d={w.d}, k={w.k} uniform centers, "
                f"Gaussian sigma={w.sigma}, mu={w.mu}, sparse sign s=2k, tol {w.tol}")
        dtype = "f32+f64"

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = K.krr_launch_count()
    step_ms, entries, infos = [], 0.0, []
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        n, info = step()
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        entries += n
        infos.append(info)
    launches = K.krr_launch_count() - launches0
    clk = clocks.stop()
    total_ms = float(sum(step_ms))
    total_ms, entries = aggregate_ranks(dist, total_ms, entries, dev)
    if rank != 0:
        return None
    res = {"metric": METRIC, "value": entries / (total_ms / 1e3), "unit": UNIT,
           "n_gpus": world, "steps": steps, "warmup": warmup,
           "ms_per_step": total_ms / steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
           "config": {"workload": desc, "N": w.N, "d": w.d,
                      "l2": "flushed between timed steps (512 MiB write)",
                      "parallelism": "replicas" if world > 1 else "single GPU", **extra},
           "clocks": clk, "gpu_launches": int(launches)}
    if workload == "c3":
        pairs = float(w.N) * w.N
        sec = total_ms / steps / 1e3
        sm_max = clk.get("sm_max_mhz") or 2070.0
        peak_flop = 152 * 128 * 2 * sm_max * 1e6
        peak_mufu = 152 * 32 * sm_max * 1e6
        t_flop = pairs * extra["roofline_model"]["flop_per_pair"] / peak_flop
        t_mufu = pairs * extra["roofline_model"]["mufu_per_pair"] / peak_mufu
        res["roofline"] = {
            "kernel": "kmvb_kernel (batched 8-setting product)", "bound": "alu",
            "achieved": pairs * extra["roofline_model"]["flop_per_pair"] / sec / 1e12,
            "peak": peak_flop / 1e12, "unit": "TFLOP/s",
            "frac": max(t_flop, t_mufu) / sec, "traffic": None,
            "peak_basis": f"FP32 152 x 128 x 2 x {sm_max:.0f} MHz and MUFU 152 x 32 "
                          f"x {sm_max:.0f} MHz (derived); frac = the larger of the FP32 "
                          f"and MUFU times over the measured time",
            "fp32_time_s": t_flop, "mufu_time_s": t_mufu}
    if infos and infos[0]:
        res["solve"] = {k: [i.get(k) for i in infos] for k in
                        ("iters", "outer_refinements", "rel_residual", "t_build_s",
                         "t_solve_s")}
    return res


def cpu_baseline(w, target_s: float = 6.0):
    """The oracle's float64 product on a bounded sample of rows of the same
    workload, timed on this host's cores; kernel evaluations per second."""
    import oracle as O
    rng = np.random.default_rng(0)
    V = rng.standard_normal((w.m, w.N))
    rows = np.sort(rng.choice(w.N, 64, replace=False))
    t0 = time.perf_counter()
    O.kmatvec(w.X, w.kernel, w.sigma, w.lam, V, rows)
    dt = time.perf_counter() - t0
    nrows = int(min(w.N, max(64, 64 * target_s / max(dt, 1e-3))))
    rows = np.sort(rng.choice(w.N, nrows, replace=False))
    t0 = time.perf_counter()
    O.kmatvec(w.X, w.kernel, w.sigma, w.lam, V, rows)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": nrows * float(w.N) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"float64 oracle product (A + lam I)V, {nrows} of {w.N} rows x {w.N} "
                      f"columns, m={w.m}, d={w.d}, {dt:.1f} s"}


def run_reference(args):
    """The oracle timed on the host cores, per step a bounded sample of the
    same workload (kernel entries of the product on a row subset)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from inputs import make_c2_mixed
    import oracle as O
    w = make_c2_mixed(n=args.n)
    rng = np.random.default_rng(0)
    V = rng.standard_normal((w.m, w.N))
    nrows = 256
    rows = np.sort(rng.choice(w.N, nrows, replace=False))
    for _ in range(args.warmup):
        O.kmatvec(w.X, w.kernel, w.sigma, w.lam, V, rows[:32])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.kmatvec(w.X, w.kernel, w.sigma, w.lam, V, rows)
    dt = time.perf_counter() - t0
    value = args.steps * nrows * float(w.N) / dt
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    sample = (f"float64 oracle product (A + lam I)V on {nrows} of {w.N} rows x {w.N} columns "
              f"per step, m={w.m}")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"full-data KRR, N={w.N}, d={w.d}, Gaussian sigma={w.sigma}, "
                               f"mu={w.mu}, m={w.m} RHS (oracle row sample)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def run_kmv(args):
    """The float32 fused product alone on the headline inputs (N = 1e5, d = 16,
    the 5 % near-duplicate workload, m = 4, Gaussian sigma = 0.5), each step one
    krr_kmatvec, its product launch timed with the library's CUDA events
    (krr_set_profiling / krr_profile_collect): the kernel the headline step
    spends most of its time in, reported against its roofline.  The command
    the ncu captures of the product use."""
    import torch
    import paper_2304_12465_gb300 as K
    from inputs import make_c2_mixed

    dist, rank, world = dist_setup(args.gpus)
    K.load()
    K.krr_set_product_path(args.product_path)
    K.krr_set_product_variant(args.product_variant)
    w = make_c2_mixed(n=args.n)
    dev = torch.device("cuda", torch.cuda.current_device())
    X = torch.from_numpy(w.X).to(dev)
    gen = torch.Generator(device=dev).manual_seed(5)
    V = torch.randn((w.m, w.N), dtype=torch.float64, device=dev, generator=gen)
    for _ in range(args.warmup):
        K.krr_kmatvec(X, w.kernel, w.sigma, w.lam, V, prec=args.kmv_prec)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    which = 2 if args.kmv_prec == "ff" else 0   # product timer: float-float or float32
    K.krr_set_profiling(True)
    K.krr_profile_collect(which)
    stream = torch.cuda.current_stream()
    ms, launch_ms = [], []
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        K.krr_kmatvec(X, w.kernel, w.sigma, w.lam, V, prec=args.kmv_prec)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        t, n = K.krr_profile_collect(which)
        launch_ms.append(t / max(n, 1))
    K.krr_set_profiling(False)
    clk = clocks.stop()
    call_ms = float(np.median(ms))
    kmv_ms = float(np.median(launch_ms))
    sm_max = clk.get("sm_max_mhz") or 2070.0
    if args.product_path == "tensor":
        tile = args.product_variant or K.krr_autotune_variant(w.kernel, w.d, w.m, w.N)[0] or 3
    else:
        tile = K.krr_autotune_choice(w.kernel, w.d, w.m, w.N)
    result = {"metric": "fused product (A + lambda I) V launch time", "value": kmv_ms,
              "unit": "ms", "higher_is_better": False, "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "dtype": "f32", "data": "synthetic",
              "config": {"workload": f"fused product, N={w.N}, d={w.d}, m={w.m}, Gaussian "
                                     f"sigma={w.sigma}, 5% near-duplicates",
                         "product_path": args.product_path},
              "call_ms": call_ms,
              "note": "value: the product kernel's launch (CUDA events around it on the "
                      "launching stream, median over steps); call_ms adds the point "
                      "preparation, the reduction and the float64 conversions of krr_kmatvec",
              "roofline": (product_roofline(args.product_path, w, kmv_ms, tile, sm_max)
                           if args.kmv_prec == "mixed" else None),
              "clocks": clk}
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "kmv":
        run_kmv(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload in ("c1", "c3", "c4"):
        run_config(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
