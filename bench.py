#!/usr/bin/env python
"""Benchmark of the particle forward map on GB300.

One step = one evaluation of the time-dependent forward map G(u) (Algorithm 1)
on the 440-mode workload: K = 10 stream function, kappa = 0.01, 16-mode theta0,
10x10 observation grid x times {0.25, 0.5, 1}, M = 1e4 particles per
observation, dt = 1e-3, float paths with double reductions -- 1.75e9
particle-steps per evaluation.  Inputs are device-resident; L2 is flushed
(256 MiB write) between timed steps, outside the timed events.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
(the plain FP64 path) on the host cores instead, on a bounded sample of the
same workload.  Under torchrun each rank evaluates its own instance (weak
scaling, no data-path collective); the time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1808_10580_gb300 import inputs  # noqa: E402

METRIC = "particle-steps/s and forward-map evals/s at fixed MC error, vs plain FP64 path"
UNIT = "particle-steps/s"


def particle_steps(w) -> int:
    return int(sum(int(np.ceil(t / w.dt - 1e-9)) for t in w.t) * w.M)


def flops_per_step(K: int) -> int:
    # Velocity contraction: two FMAs per real coefficient (2 N_u) plus four per
    # x1-harmonic to combine the partial sums (4 K); an FMA counts as 2 FLOP.
    n_u = (2 * K + 1) ** 2 - 1
    return 2 * (2 * n_u + 4 * K)


def method_flops_per_step(K: int) -> int:
    """The method's own work per particle-step, independent of how a kernel
    organises it: the velocity of Eq. v_expand summed directly takes 8 FMAs per
    half-mode (the complex product of the x1 and x2 harmonics, then p cos + q
    sin for both velocity components), about 8H instructions, plus about 90
    for the noise, the Euler step and the wrap; an FMA counts as 2 FLOP.
    K = 10: 2 (8 * 220 + 90) = 3700 FLOP."""
    H = ((2 * K + 1) ** 2 - 1) // 2
    return 2 * (8 * H + 90)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except Exception:
            pass
    return {"sm_max_mhz": 2070.0}, "fallback"


def tensor_flops_per_step(K: int) -> int:
    """FLOP per particle-step of the tensor-core path: the per-step contraction
    P = A W with A one row of (2K+1) basis values and W the (2K+1) x (4K+1)
    coefficient matrix, done as three products (hi.hi, lo.hi, hi.lo)."""
    return 3 * 2 * (2 * K + 1) * (4 * K + 1)


def tensor_operands(K: int) -> str:
    """Operand type of the library's tensor-core particle kernels at this K:
    FP16 (kind::f16) from K = 10 on, TF32 below."""
    return "f16" if K >= 10 else "tf32"


def tensor_peak(K: int, peaks: dict, peaks_kind: str):
    """Dense peak for the operand type at K: FP16 runs at the BF16 rate (the
    measured cuBLAS bf16 figure), TF32 at 1.1/2.25 of it (nominal ratio)."""
    bf16 = float(peaks.get("bf16_tflops", 1900.0))
    if tensor_operands(K) == "f16":
        return bf16, f"FP16 dense = bf16_tflops {bf16} ({peaks_kind}, burst; same dense rate)"
    return bf16 * 1.1 / 2.25, f"TF32 dense = bf16_tflops {bf16} ({peaks_kind}, burst) x 1.1/2.25"


def tensor_roofline(K, steps, kernel_ms, peaks, peaks_kind):
    """Roofline of the tensor-core particle kernel: the method's work
    (method_flops_per_step) per second against the dense peak of its operand
    type; beside it the fraction the issued MMAs reach (three hi/lo products of
    the padded contraction)."""
    peak, basis = tensor_peak(K, peaks, peaks_kind)
    sec = kernel_ms / 1e3
    achieved = steps * method_flops_per_step(K) / sec / 1e12
    issued = steps * tensor_flops_per_step(K) / sec / 1e12
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "flop_per_particle_step": method_flops_per_step(K),
            "work_basis": "the method's work: direct-sum velocity, 8 FMAs per half-mode + ~90 per step",
            "peak_basis": basis, "operands": tensor_operands(K), "tensor_issued_frac": issued / peak,
            "tensor_issued_flop_per_particle_step": tensor_flops_per_step(K),
            "tensor_issued_note": "the MMAs the kernel issues: three hi/lo products of the padded "
                                  "(2K+1) x (4K+1) contraction"}


def fp32_peak_tflops(peaks, sm_count):
    """FP32 FMA pipe: SMs x 128 lanes x 2 FLOP x the maximum SM clock."""
    return sm_count * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12


def fp32_roofline(K, steps, kernel_ms, peaks, peaks_kind, sm_count):
    """Roofline of the FP32-pipe particle kernel: the FMAs it executes
    (flops_per_step) per second against the FP32 pipe peak; beside it the
    method's work (method_flops_per_step) on the same peak."""
    peak = fp32_peak_tflops(peaks, sm_count)
    sec = kernel_ms / 1e3
    achieved = steps * flops_per_step(K) / sec / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "flop_per_particle_step": flops_per_step(K),
            "flop_note": "the FMAs it executes: 2 per real coefficient + 4 per x1 harmonic",
            "method_work_frac": steps * method_flops_per_step(K) / sec / 1e12 / peak,
            "peak_basis": f"{sm_count} SMs x 128 FP32 lanes x 2 FLOP x sm_max_mhz "
                          f"{peaks.get('sm_max_mhz', 2070.0)} ({peaks_kind})",
            "particle_steps_per_s": steps / sec}


def profile_value(name, key):
    """The number on the line '<key>: <number>' of a committed ncu summary, or None."""
    p = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(p):
        return None
    for line in open(p):
        if line.startswith(key + ":"):
            v = line.split(":", 1)[1].strip()
            return None if v in ("", "null") else float(v)
    return None


def profile_traffic(name="timedep_k10_kernel.md"):
    """DRAM bytes per launch of the particle kernel from the committed ncu summary
    (line 'traffic_bytes_per_launch: <int>'), or None."""
    v = profile_value(name, "traffic_bytes_per_launch")
    return None if v is None else int(v)


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.idx), "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.f is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [s.strip() for s in line.split(",")]
            if len(parts) >= 9:
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    pass
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for _, _, flags in rows for n, f in zip(names, flags) if f.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if n_gpus > 0 else "gloo")
    return rank, world, local


def oracle_sample(w, budget_s=12.0, max_paths=512, obs_id=None):
    """Times the FP64 oracle on paths [0, P) of every observation, P sized so the
    run takes about budget_s.  Returns (steps/s, threads, P, per-path g, seconds).
    obs_id: the RNG stream of each observation (shared paths), default its index."""
    import oracle
    oracle.lib()
    ids = None if obs_id is None else np.asarray(obs_id, dtype=np.int64)
    t0 = time.perf_counter()
    g1 = oracle.timedep_paths(w.K, w.u, w.kappa, w.theta0, w.x, w.t, w.dt, w.seed, npaths=1, obs_id=ids)
    t1 = time.perf_counter() - t0
    P = int(max(1, min(max_paths, budget_s / max(t1, 1e-3))))
    t0 = time.perf_counter()
    g = oracle.timedep_paths(w.K, w.u, w.kappa, w.theta0, w.x, w.t, w.dt, w.seed, npaths=P, obs_id=ids)
    secs = time.perf_counter() - t0
    steps = particle_steps(w) // w.M * P
    threads = os.cpu_count() or 1
    del g1
    return steps / secs, threads, P, g, secs


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.lib()
    w = inputs.timedep_k10()
    cores = os.cpu_count() or 1
    obs = np.arange(0, len(w.t), 10)          # 30 observations spanning the three times
    P = 32                                    # 960 (observation, path) items: every host core busy
    sub_steps = sum(int(np.ceil(t / w.dt - 1e-9)) for t in w.t[obs]) * P

    def step():
        oracle.timedep_paths(w.K, w.u, w.kappa, w.theta0, w.x[obs], w.t[obs], w.dt, w.seed, npaths=P, obs_id=obs)

    for _ in range(args.warmup):
        step()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = sub_steps * args.steps / total
    sample = f"{len(obs)} of 300 observations (every 10th) x paths 0..{P - 1}, all steps, per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "K": w.K, "n_obs": len(w.t), "M": w.M, "dt": w.dt},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch

    import paper_1808_10580_gb300 as pm

    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = inputs.timedep_k10(M=args.M) if args.M else inputs.timedep_k10()
    n_obs = len(w.t)
    inst = rank                                   # each rank evaluates its own instance (weak scaling)
    steps_per_eval = particle_steps(w)
    stream_of = None
    if args.share_paths:
        # one path per point and path index, stopped at every time of that point
        _, stream_of, _, steps_per_path = pm.pm_path_groups(w.x, w.t, w.dt)
        steps_per_eval = steps_per_path * w.M
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ctx = pm.pm_create(local, stream.cuda_stream)
    fld = pm.Field(w.K, w.u)
    th = pm.Fourier(w.theta0.k, w.theta0.a, w.theta0.b)
    x = torch.from_numpy(w.x).to(dev)
    t = torch.from_numpy(w.t).to(dev)
    mean = torch.empty(n_obs, dtype=torch.float64, device=dev)
    var = torch.empty_like(mean)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    mode = (pm.PM_TENSOR if args.tensor else 0) | (pm.PM_SHARE_PATHS if args.share_paths else 0)
    flags = pm.PM_FP32 | pm.PM_ASYNC | mode

    def step():
        pm.pm_forward_timedep(ctx, fld, w.kappa, th, x, t, n_obs, w.M, w.dt, w.seed, flags, mean, var,
                              instance=inst)

    pm.pm_set_kernel_timing(ctx, 1)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)

    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize(dev)
    step_ms, kern_ms = [], []
    launches0 = pm.pm_launch_count(ctx)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    gpu_index = local
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    if vis and vis.split(",")[local].strip().isdigit():
        gpu_index = int(vis.split(",")[local])
    with ClockSampler(gpu_index) as clocks:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
            kern_ms.append(pm.pm_last_kernel_ms(ctx))
        torch.cuda.synchronize(dev)
    launches = pm.pm_launch_count(ctx) - launches0
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize(dev)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(step_ms) / 1e3
    if world > 1:
        import torch.distributed as dist
        tt = torch.tensor([total_s], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_s = float(tt.item())
    value = steps_per_eval * world * args.steps / total_s
    clock = clocks.summary()

    # End to end through the public API with host arrays: H2D of x, t and D2H of mean, var inside.
    hx, ht = np.ascontiguousarray(w.x), np.ascontiguousarray(w.t)
    hmean, hvar = np.empty(n_obs), np.empty(n_obs)
    e2e_times = []
    for k in range(max(2, min(args.steps, 5))):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        pm.pm_forward_timedep(ctx, fld, w.kappa, th, hx, ht, n_obs, w.M, w.dt, w.seed,
                              pm.PM_FP32 | mode, hmean, hvar, instance=inst)
        e2e_times.append(time.perf_counter() - t0)
    e2e_value = steps_per_eval * world / statistics.median(e2e_times)

    # The same map on the FP32 pipes (timedep_kernel<float, K, 128>: the
    # product-basis sum, no tensor cores), kernel time by events.
    simt = None
    if args.tensor and not args.no_fp32_compare:
        flags32 = pm.PM_FP32 | pm.PM_ASYNC | (pm.PM_SHARE_PATHS if args.share_paths else 0)
        ms32 = []
        for k in range(4):
            flush.zero_()
            pm.pm_forward_timedep(ctx, fld, w.kappa, th, x, t, n_obs, w.M, w.dt, w.seed, flags32, mean, var,
                                  instance=inst)
            if k >= 1:
                ms32.append(pm.pm_last_kernel_ms(ctx))
        simt = {"kernel": f"timedep_kernel<float,{w.K},128>", "kernel_ms": statistics.mean(ms32)}
        step()                                     # leave the tensor-core estimate in mean / var
        torch.cuda.synchronize(dev)

    # Monte Carlo standard error of the timed estimate.
    se = np.sqrt(var.cpu().numpy() / w.M)

    # The plain FP64 path on the same GPU and workload (one evaluation, kernel
    # time by events): the metric's point of comparison.
    fp64 = None
    if not args.no_fp64_compare:
        m64 = torch.empty_like(mean)
        pm.pm_forward_timedep(ctx, fld, w.kappa, th, x, t, n_obs, w.M, w.dt, w.seed, pm.PM_FP64, m64,
                              instance=inst)
        ms64 = pm.pm_last_kernel_ms(ctx)
        fp64 = {"kernel_ms": ms64, "particle_steps_per_s": particle_steps(w) / (ms64 / 1e3),
                "evaluation_speedup": ms64 / statistics.mean(kern_ms),
                "max_abs_mean_diff": float((m64 - mean).abs().max().item()),
                "note": "timedep_kernel<double,10,128> on the same observations, paths and streams"}

    line = None
    if rank == 0:
        peaks, peaks_kind = measured_peaks()
        sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
        fp32_peak = fp32_peak_tflops(peaks, sm_count)
        kern_mean_ms = statistics.mean(kern_ms)
        simt_rate = steps_per_eval * flops_per_step(w.K) / (kern_mean_ms / 1e3) / 1e12
        if args.tensor:
            roof = tensor_roofline(w.K, steps_per_eval, kern_mean_ms, peaks, peaks_kind)
            roof.update({
                    "traffic": profile_traffic("timedep_k10_tc_kernel.md") if w.K == 10 else None,
                    "kernel": f"timedep_tc_kernel<{w.K}>", "kernel_ms": kern_mean_ms,
                    "issue_active_frac_ncu": (profile_value("timedep_k10_tc_kernel.md", "issue_active_frac")
                                              if w.K == 10 else None),
                    "binding_constraint": "SIMT instruction issue (harmonics, operand split, RNG, Euler "
                                          "step), not the tensor pipe: see issue_active_frac_ncu"})
        else:
            peak_tflops = fp32_peak
            achieved = simt_rate
            roof = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                    "frac": achieved / peak_tflops, "traffic": profile_traffic(),
                    "kernel": f"timedep_kernel<float,{w.K},128>", "kernel_ms": kern_mean_ms,
                    "flop_per_particle_step": flops_per_step(w.K),
                    "peak_basis": f"{sm_count} SMs x 128 FP32 lanes x 2 FLOP x sm_max_mhz "
                                  f"{peaks.get('sm_max_mhz', 2070.0)} ({peaks_kind})"}
        if simt is not None:
            simt.update(fp32_roofline(w.K, steps_per_eval, simt["kernel_ms"], peaks, peaks_kind, sm_count))
            simt["tensor_speedup"] = simt["kernel_ms"] / kern_mean_ms
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": ("f32 paths; velocity contraction f16 hi/lo x3 on tensor cores; f64 reductions"
                      if args.tensor and tensor_operands(w.K) == "f16" else
                      "f32 paths; velocity contraction tf32 hi/lo x3 on tensor cores; f64 reductions"
                      if args.tensor else "f32 paths; f64 reductions"),
            "data": "synthetic",
            "config": {"workload": w.name, "K": w.K, "n_u": (2 * w.K + 1) ** 2 - 1, "n_obs": n_obs, "M": w.M,
                       "dt": w.dt, "kappa": w.kappa, "particle_steps_per_eval": steps_per_eval,
                       "shared_paths": bool(args.share_paths),
                       "independent_path_steps_per_eval": particle_steps(w),
                       "forward_map_evals_per_s": value / steps_per_eval,
                       "l2": "flushed between timed steps (256 MiB write, outside the timed events)",
                       "reductions": "f64", "mc_se_median": float(np.median(se)), "mc_se_max": float(se.max())},
            "roofline": roof,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": n_obs * 24,
                    "d2h_bytes_per_step": n_obs * 16},
            "gpu_launches": int(launches),
            "clocks": clock,
            "plain_fp64_gpu": fp64,
            "fp32_pipe_kernel": simt,
        }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, threads, P, g_or, secs = oracle_sample(w, obs_id=stream_of)
        # pathwise check of the same sample against the GPU (same stream)
        gdev = torch.empty(n_obs * w.M, dtype=torch.float64, device=dev)
        pm.pm_forward_timedep(ctx, fld, w.kappa, th, x, t, n_obs, w.M, w.dt, w.seed,
                              pm.PM_FP32 | mode, mean, var, g_out=gdev)
        g_gpu = gdev.cpu().numpy().reshape(n_obs, w.M)[:, :P]
        d = (g_gpu - g_or).reshape(-1)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": f"all {n_obs} observations x paths 0..{P - 1} ({secs:.1f} s, FP64 direct sum)"}
        line["accuracy_vs_oracle"] = {
            "paths_compared": int(d.size), "paired_mean_diff": float(d.mean()),
            "paired_diff_se": float(d.std(ddof=1) / np.sqrt(d.size)) if d.size > 1 else None,
            "frac_paths_within_1e-5": float(np.mean(np.abs(d) <= 1e-5)),
            "note": "float paths decorrelate from FP64 paths by t~0.4 (chaotic flow); agreement is in distribution"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    pm.pm_destroy(ctx)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_aux(args):
    """Auxiliary measurements (not the headline line): the Dirichlet disk workload
    (50 obs x M = 1e5, dt = 1e-4) or the 256-instance batched workload (mixed
    time-dependent / Dirichlet, 100 obs x M = 4096 each).  Throughput counts the
    Euler steps the paths actually took (pm_last_step_count)."""
    import torch

    import paper_1808_10580_gb300 as pm

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ctx = pm.pm_create(0, stream.cuda_stream)
    pm.pm_set_kernel_timing(ctx, 1)
    if args.workload == "dirichlet":
        w = inputs.dirichlet_disk_k10(M=args.M or 100_000)
        if args.K:  # another wave-number bound: a prior draw of that size, the same points and steps
            w = dataclasses.replace(w, name=f"dirichlet_disk_k{args.K}_50obs_M{w.M}_dt1e-4", K=args.K,
                                    u=inputs.prior_field(args.K, 1002))
        fld = pm.Field(w.K, w.u)
        gd = pm.DirichletData(w.g.R, w.g.quad, w.g.f_const, w.g.a, w.g.b)
        x = torch.from_numpy(w.x).to(dev)
        mean = torch.empty(len(w.x), dtype=torch.float64, device=dev)
        var = torch.empty_like(mean)

        def step():
            pm.pm_forward_dirichlet(ctx, fld, w.drift_scale, w.kappa, gd, x, len(w.x), w.M, w.dt, w.max_steps,
                                    w.seed, pm.PM_FP32 | (pm.PM_TENSOR if args.tensor else 0), mean, var)
        name, cfg = w.name, {"n_obs": len(w.x), "M": w.M, "dt": w.dt, "kappa": w.kappa, "drift_scale": w.drift_scale,
                             "K": w.K, "tensor_cores": bool(args.tensor)}
    elif args.workload == "dirichlet_general":
        w, dfw = inputs.dirichlet_general_disk(M=args.M or 100_000)
        fld = pm.Field(w.K, w.u)
        gd = pm.DirichletData(w.g.R, w.g.quad, w.g.f_const, w.g.a, w.g.b)
        dfp = pm.DiffusionForcing(dfw.s0, dfw.s1, dfw.milstein, dfw.c, dfw.F, dfw.w)
        x = torch.from_numpy(w.x).to(dev)
        mean = torch.empty(len(w.x), dtype=torch.float64, device=dev)
        var = torch.empty_like(mean)

        def step():
            pm.pm_forward_dirichlet_general(ctx, fld, w.drift_scale, gd, dfp, x, len(w.x), w.M, w.dt, w.max_steps,
                                            w.seed, pm.PM_FP32 | (pm.PM_TENSOR if args.tensor else 0), mean, var)
        name, cfg = w.name, {"n_obs": len(w.x), "M": w.M, "dt": w.dt, "drift_scale": w.drift_scale,
                             "sigma": "diag(0.3 + 0.15 x1, 0.3 - 0.1 x2), Milstein", "sources": 3,
                             "tensor_cores": bool(args.tensor),
                             "kernel": ("dirichlet_tc_kernel<10, general> (velocity on the tensor cores)" if args.tensor
                                        else "dirichlet_general_kernel<float,10> (FP32 pipes)")}
    else:
        ws = inputs.batched_instances(B=args.B, M=args.M or 4096)
        if args.K:  # another wave-number bound: prior draws of that size
            for b, w in enumerate(ws):
                w.K, w.u = args.K, inputs.prior_field(args.K, 1003, counter=b)
        xs, ts, inst = [], [], []
        row = 0
        for w in ws:
            n = len(w.x)
            xs.append(w.x)
            ts.append(w.t if isinstance(w, inputs.TimedepWorkload) else np.zeros(n))
            d = dict(kind=pm.PM_KIND_TIMEDEP if isinstance(w, inputs.TimedepWorkload) else pm.PM_KIND_DIRICHLET,
                     u=torch.from_numpy(w.u).to(dev), kappa=w.kappa, dt=w.dt, row0=row, n_obs=n, M=w.M, seed=w.seed)
            if d["kind"] == pm.PM_KIND_DIRICHLET:
                d.update(drift_scale=w.drift_scale, max_steps=w.max_steps)
            inst.append(d)
            row += n
        th = next(w.theta0 for w in ws if isinstance(w, inputs.TimedepWorkload))
        g = next(w.g for w in ws if isinstance(w, inputs.DirichletWorkload))
        xt = torch.from_numpy(np.ascontiguousarray(np.concatenate(xs))).to(dev)
        tt = torch.from_numpy(np.ascontiguousarray(np.concatenate(ts))).to(dev)
        batch = pm.Batch(ws[0].K, inst, xt, tt, pm.Fourier(th.k, th.a, th.b), pm.DirichletData(g.R, g.quad, g.f_const, g.a, g.b))
        mean = torch.empty(row, dtype=torch.float64, device=dev)
        var = torch.empty_like(mean)

        def step():
            pm.pm_forward_batched(ctx, batch, pm.PM_FP32 | (pm.PM_TENSOR if args.tensor else 0), mean, var)
        name, cfg = (f"batched_{args.B}x100obs_M{args.M or 4096}" + (f"_k{args.K}" if args.K else ""),
                     {"B": args.B, "rows": row, "K": ws[0].K, "tensor_cores": bool(args.tensor)})
    tuned = None
    if args.autotune and args.workload in ("dirichlet", "batched"):
        flags = pm.PM_FP32 | (pm.PM_TENSOR if args.tensor else 0)
        if args.workload == "dirichlet":
            pm.pm_autotune_dirichlet(ctx, fld, w.drift_scale, w.kappa, gd, x, len(w.x), w.M, w.dt, w.max_steps,
                                     w.seed, flags)
            kind = pm.PM_TUNE_DIRICHLET
        else:
            pm.pm_autotune_batched(ctx, batch, flags)
            kind = pm.PM_TUNE_BATCHED
        ctas, pairs = pm.pm_tuned_shape(ctx, kind, args.K or 10, pm.PM_TENSOR if args.tensor else 0)
        tuned = {"ctas_per_sm": ctas, "refill_step_pairs": pairs if args.tensor else None}
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    times, steps = [], []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        times.append(e0.elapsed_time(e1) / 1e3)
        steps.append(pm.pm_last_step_count(ctx))
    total = sum(times)
    line = {"metric": METRIC, "value": sum(steps) / total, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic", "auxiliary": True,
            "config": dict(workload=name, particle_steps_per_call=steps[-1], **cfg)}
    line["config"]["grid"] = pm.pm_last_grid(ctx)
    line["config"]["autotuned_shape"] = tuned
    if args.workload == "batched":
        # CUDA-graph replay against direct launches of the same call (the
        # difference is the launch overhead the graph removes)
        def timed():
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            return e0.elapsed_time(e1)
        replay = timed()
        pm.pm_set_graph_mode(ctx, 0)
        step()
        direct = timed()
        pm.pm_set_graph_mode(ctx, 1)
        line["graph"] = {"replay_ms": replay, "direct_ms": direct, "launches_per_call": 4}
    if args.workload in ("dirichlet", "dirichlet_general"):
        line["kernel_ms"] = pm.pm_last_kernel_ms(ctx)
    if args.workload == "dirichlet":
        # Exit-step distribution of the same call (outside the timed region): the
        # longest path bounds the call from below at one path's step latency.
        es = torch.empty(len(w.x) * w.M, dtype=torch.int32, device=dev)
        pm.pm_forward_dirichlet(ctx, fld, w.drift_scale, w.kappa, gd, x, len(w.x), w.M, w.dt, w.max_steps,
                                w.seed, pm.PM_FP32 | (pm.PM_TENSOR if args.tensor else 0), mean, var, exit_step=es)
        e = es.cpu().numpy().astype(np.int64)
        ex = e[e >= 0]
        q = np.quantile(ex, [0.5, 0.99, 0.999, 0.99999]) if ex.size else [0, 0, 0, 0]
        line["exit_steps"] = {"mean": float(ex.mean()) if ex.size else 0.0, "p50": float(q[0]), "p99": float(q[1]),
                              "p99.9": float(q[2]), "p99.999": float(q[3]), "max": int(ex.max()) if ex.size else 0,
                              "capped": int((e < 0).sum()),
                              "ms_per_step_of_longest_path": line["kernel_ms"] / max(int(ex.max()), 1)
                              if ex.size else None}
    print(json.dumps(line), flush=True)
    pm.pm_destroy(ctx)
    return 0


def run_sweep(args):
    """Cost against the number of real coefficients N_u (the scaling the paper
    plots for its GPU code, Section 4): the time-dependent workload's 300
    observations x M paths with a prior field of each K, on the FP32 pipes and
    on the tensor cores where the tensor path has the K (auxiliary line).
    K = 24 ... 64 (N_u up to 16640, beyond the 3209 coefficients of the
    paper's second example) run the wide-K kernels, K = 80 (N_u = 25920,
    which holds the 20081 of its third, |k|_2 <= 80) the FP32 pipes only."""
    import torch

    import paper_1808_10580_gb300 as pm

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ctx = pm.pm_create(0, stream.cuda_stream)
    pm.pm_set_kernel_timing(ctx, 1)
    w = inputs.timedep_k10(M=args.M or 10_000)
    th = pm.Fourier(w.theta0.k, w.theta0.a, w.theta0.b)
    x = torch.from_numpy(w.x).to(dev)
    t = torch.from_numpy(w.t).to(dev)
    mean = torch.empty(len(w.t), dtype=torch.float64, device=dev)
    steps = particle_steps(w)
    rows = []
    ks = [int(k) for k in args.sweep_k.split(",")] if args.sweep_k else [2, 3, 4, 5, 6, 8, 10, 12, 16, 24, 32, 40, 48, 56, 64, 80]
    for K in ks:
        fld = pm.Field(K, inputs.prior_field(K, 1001))
        row = {"K": K, "n_u": (2 * K + 1) ** 2 - 1}
        for name, flags in (("fp32_ms", pm.PM_FP32), ("tensor_ms", pm.PM_FP32 | pm.PM_TENSOR)):
            if name == "tensor_ms" and K not in (4, 5, 6, 8, 10, 12, 16, 24, 32, 40, 48, 56, 64):
                continue
            ms = []
            for k in range(args.warmup + args.steps):
                pm.pm_forward_timedep(ctx, fld, w.kappa, th, x, t, len(w.t), w.M, w.dt, w.seed, flags, mean)
                if k >= args.warmup:
                    ms.append(pm.pm_last_kernel_ms(ctx))
            row[name] = statistics.median(ms)
        if "tensor_ms" in row:
            row["tensor_speedup"] = row["fp32_ms"] / row["tensor_ms"]
        rows.append(row)
    fp32 = np.array([[r["n_u"], r["fp32_ms"]] for r in rows if r["K"] >= 4])
    slope, icpt = np.polyfit(fp32[:, 0], fp32[:, 1], 1) if len(fp32) >= 2 else (None, None)
    line = {"metric": "particle-map kernel time vs N_u", "auxiliary": True, "data": "synthetic",
            "unit": "ms per evaluation", "value": None, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "config": {"workload": f"{w.name} with a prior field of each K", "particle_steps_per_eval": steps},
            "rows": rows, "fp32_linear_fit": {"ms_per_coefficient": slope, "ms_at_zero": icpt}}
    print(json.dumps(line), flush=True)
    pm.pm_destroy(ctx)
    return 0


def run_surrogate(args):
    """Training and inference throughput of the surrogate network (auxiliary
    line): 440 -> 512 -> 512 -> 100, BF16 operands with FP32 accumulation on
    the tensor cores, Adam, batch 512, on 2^16 synthetic pairs resident on the
    device; inference at batch 64."""
    import torch

    import paper_1808_10580_gb300 as pm

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ctx = pm.pm_create(0, stream.cuda_stream)
    n_in, h, n_out, N, batch = 440, 512, 100, 1 << 16, 512
    g = torch.Generator(device="cpu").manual_seed(12)
    U = torch.randn(N, n_in, generator=g).to(dev)
    Y = torch.tanh(U[:, :n_out] * 0.5 + 0.1 * U[:, n_out:2 * n_out]).contiguous()
    net = pm.pm_surrogate_create(ctx, n_in, h, n_out, 12)
    epochs = max(1, args.steps)
    pm.pm_surrogate_train(ctx, net, U, Y, epochs=1, batch=batch)          # warm-up epoch
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    hist = pm.pm_surrogate_train(ctx, net, U, Y, epochs=epochs, batch=batch)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    train_s = e0.elapsed_time(e1) / 1e3
    fwd = 2 * (n_in * h + h * h + h * n_out)
    step_flop = fwd + fwd + 2 * (h * h + h * n_out)        # forward, weight gradients, input gradients of layers 2-3
    samples = epochs * (N // batch) * batch
    Ui = U[:64].contiguous()
    Yi = torch.empty(64, n_out, device=dev)
    for _ in range(10):
        pm.pm_surrogate_infer(ctx, net, Ui, Yi)
    torch.cuda.synchronize(dev)
    reps = 200
    e0.record(stream)
    for _ in range(reps):
        pm.pm_surrogate_infer(ctx, net, Ui, Yi)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    infer_ms = e0.elapsed_time(e1) / reps
    # the same GEMM kernel at a large shape (8192^3): what it sustains when the
    # tiles fill the GPU (the training shapes above occupy 32 of the SMs)
    n = 8192
    A = torch.randn(n, n, device=dev).to(torch.bfloat16)
    B = torch.randn(n, n, device=dev).to(torch.bfloat16)
    Cb = torch.empty(n, n, device=dev)
    for _ in range(3):
        pm.pm_gemm_bf16(ctx, A, n, B, n, n, n, n, Cb, n)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(5):
        pm.pm_gemm_bf16(ctx, A, n, B, n, n, n, n, Cb, n)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    big_tflops = 5 * 2.0 * n ** 3 / (e0.elapsed_time(e1) / 1e3) / 1e12
    del A, B, Cb
    peaks, kind = measured_peaks()
    peak = float(peaks.get("bf16_tflops", 1900.0))
    achieved = samples * step_flop / train_s / 1e12
    line = {"metric": "surrogate training samples/s", "auxiliary": True, "data": "synthetic",
            "value": samples / train_s, "unit": "samples/s", "n_gpus": 1, "steps": epochs, "warmup": 1,
            "dtype": "bf16", "config": {"workload": "mlp_440_512_512_100_batch512_2^16pairs", "epochs": epochs,
                                        "final_loss": float(hist[-1])},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "flop_per_sample": step_flop,
                         "peak_basis": f"bf16_tflops ({kind}, burst)"},
            "inference_batch64_ms": infer_ms,
            "gemm_8192_cubed": {"achieved": big_tflops, "peak": peak, "unit": "TFLOP/s", "frac": big_tflops / peak}}
    print(json.dumps(line), flush=True)
    pm.pm_surrogate_destroy(net)
    pm.pm_destroy(ctx)
    return 0


def run_bvp(args):
    """The optimal-forcing example (auxiliary line): the particle functionals of
    the square-domain boundary-value problem (3 observations x M paths, the
    paper's drift, diffusion, sources and boundary data), timed, then the
    Nelder-Mead search for the forcing on those functionals."""
    import torch

    import paper_1808_10580_gb300 as pm
    from paper_1808_10580_gb300 import optimal_forcing as of

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ctx = pm.pm_create(0, stream.cuda_stream)
    pm.pm_set_kernel_timing(ctx, 1)
    w = inputs.optimal_forcing(M=args.M or 1_000_000)
    flags = pm.PM_FP32
    for _ in range(args.warmup):
        E, se = of.functionals(ctx, w, flags)
    times, steps = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        E, se = of.functionals(ctx, w, flags)
        times.append(time.perf_counter() - t0)
        steps.append(pm.pm_last_step_count(ctx))
    kern_ms = pm.pm_last_kernel_ms(ctx)
    t0 = time.perf_counter()
    r = of.solve(E, w.y, xtol=1e-12, ftol=1e-16)
    t_nm = time.perf_counter() - t0
    per_call = statistics.median(times)
    line = {"metric": METRIC, "value": steps[-1] / per_call, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * per_call, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic", "auxiliary": True,
            "config": {"workload": w.name, "n_obs": len(w.x), "M": w.M, "dt": w.dt, "kappa": w.prob.kappa,
                       "b": w.prob.b.tolist(), "sources": w.prob.c.tolist(), "particle_steps_per_call": steps[-1],
                       "grid": pm.pm_last_grid(ctx)},
            "kernel_ms": kern_ms,
            "functionals": {"E": E.tolist(), "se": se.tolist()},
            "nelder_mead": {"F": r.x.tolist(), "cost": r.fun, "evaluations": r.evaluations,
                            "iterations": r.iterations, "seconds": t_nm,
                            "G_evaluations_per_s": r.evaluations / (per_call + t_nm),
                            "note": "G(F) is affine in F (Theorem 3.2), so one set of paths serves every evaluation"}}
    print(json.dumps(line), flush=True)
    pm.pm_destroy(ctx)
    return 0


def run_layout(args):
    """Shared paths on the observation layout of the paper's turbulent-flow
    example (auxiliary line): 2 points x 13 times in [0, 0.5], K = 16 field
    on the tensor cores, M paths per observation; independent paths per
    observation against paths shared by the 13 times of each point."""
    import torch

    import paper_1808_10580_gb300 as pm

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ctx = pm.pm_create(0, stream.cuda_stream)
    pm.pm_set_kernel_timing(ctx, 1)
    w = inputs.two_point_time_series(M=args.M or 100_000)
    n = len(w.t)
    fld = pm.Field(w.K, w.u)
    th = pm.Fourier(w.theta0.k, w.theta0.a, w.theta0.b)
    x = torch.from_numpy(w.x).to(dev)
    t = torch.from_numpy(w.t).to(dev)
    out = {}
    for name, extra in (("independent", 0), ("shared", pm.PM_SHARE_PATHS)):
        mean = torch.empty(n, dtype=torch.float64, device=dev)
        var = torch.empty_like(mean)
        ms, steps = [], 0
        for k in range(args.warmup + args.steps):
            pm.pm_forward_timedep(ctx, fld, w.kappa, th, x, t, n, w.M, w.dt, w.seed,
                                  pm.PM_FP32 | pm.PM_TENSOR | extra, mean, var)
            if k >= args.warmup:
                ms.append(pm.pm_last_kernel_ms(ctx))
                steps = pm.pm_last_step_count(ctx)
        out[name] = {"kernel_ms": statistics.median(ms), "particle_steps": steps,
                     "evals_per_s": 1e3 / statistics.median(ms), "mean": mean.cpu().numpy(),
                     "se": np.sqrt(var.cpu().numpy() / w.M)}
    d = np.abs(out["shared"]["mean"] - out["independent"]["mean"])
    se = np.sqrt(out["shared"]["se"] ** 2 + out["independent"]["se"] ** 2)
    line = {"metric": METRIC, "auxiliary": True, "data": "synthetic", "unit": "forward-map evals/s",
            "value": out["shared"]["evals_per_s"], "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "dtype": "f32", "config": {"workload": w.name, "K": w.K, "n_obs": n, "M": w.M, "dt": w.dt,
                                       "kappa": w.kappa},
            "independent": {k: v for k, v in out["independent"].items() if k in ("kernel_ms", "particle_steps",
                                                                                  "evals_per_s")},
            "shared": {k: v for k, v in out["shared"].items() if k in ("kernel_ms", "particle_steps", "evals_per_s")},
            "speedup": out["independent"]["kernel_ms"] / out["shared"]["kernel_ms"],
            "max_diff_in_se": float((d / np.maximum(se, 1e-300)).max())}
    print(json.dumps(line), flush=True)
    pm.pm_destroy(ctx)
    return 0


def run_mcmc(args):
    """Surrogate-screened pCN against plain pCN on the same GPU (configuration:
    MLP 440 -> 512 -> 512 -> 100 trained on particle-map pairs, data with noise
    sigma = 0.01, 64 chains; one JSON line):
      feasibility  at the configured sigma, the change of the misfit Phi over
                   small pCN proposals (beta = --feas-beta) around the
                   data-generating field, for several particle counts M: with
                   common random numbers the Monte Carlo error of G_M(u) is a
                   rough function of u, and no sampler moves while it exceeds
                   sigma / sqrt(n_obs); the M at which E[dPhi] falls to 1 and
                   its measured cost per evaluation;
      configured   both samplers at the configured sigma and M (accepted/s);
      moving       both samplers at --move-sigma, where the chains move:
                   accepted/s, the relative Monte Carlo error of the pooled
                   posterior mean (between-chain standard errors) and the time
                   each needs for 1e-2 relative error (error ~ 1/sqrt(time)).
    Chains start at the data-generating field."""
    import torch

    import paper_1808_10580_gb300 as pm
    from paper_1808_10580_gb300 import surrogate_mcmc as sm

    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = pm.pm_create(0, stream.cuda_stream)
    M0 = args.M or 4096
    prob = sm.make_data(ctx, sm.make_problem(M=M0, sigma=args.sigma))
    n_obs = len(prob.t)
    u_true = prob.u_true.copy()

    # --- feasibility at the configured sigma: dPhi over small proposals vs M
    props = sm.pcn_proposals(prob, u_true, args.feas_beta, 32, seed=12)
    feas = []
    for M in [int(v) for v in args.feas_M.split(",")]:
        pr = sm.make_problem(M=M, sigma=args.sigma)
        pr.y, pr.u_true = prob.y, u_true
        t0 = time.perf_counter()
        G = sm.forward_many(ctx, pr, np.vstack([u_true[None, :], props]), tensor=args.tensor)
        secs = time.perf_counter() - t0
        phi = sm.misfit(pr, G)
        dphi = phi[1:] - phi[0]
        feas.append({"M": M, "dphi_median": float(np.median(dphi)), "dphi_mean": float(dphi.mean()),
                     "mean_acceptance": float(np.mean(np.minimum(1.0, np.exp(-dphi)))),
                     "seconds_per_eval": secs / G.shape[0]})
    # E[dPhi] = a / M + b: a the Monte Carlo roughness of G_M (n_obs SE^2 / sigma^2
    # times M), b the change of the smooth misfit over proposals of this beta
    # (the posterior's own curvature, ~ beta^2).  Chains move when both are ~ 1:
    # M ~ a and beta ~ feas_beta / sqrt(b).
    need = None
    if len(feas) >= 2:
        Ms = np.array([f["M"] for f in feas], dtype=float)
        dp = np.array([f["dphi_mean"] for f in feas])
        (a_fit, b_fit), *_ = np.linalg.lstsq(np.stack([1.0 / Ms, np.ones_like(Ms)], 1), dp, rcond=None)
        s_per_path_eval = float(np.mean([f["seconds_per_eval"] / f["M"] for f in feas]))
        M_need = max(float(a_fit), 1.0)
        sec = s_per_path_eval * M_need
        need = {"fit": {"a": float(a_fit), "b": float(b_fit), "model": "E[dPhi] = a / M + b"},
                "M_for_noise_term_1": M_need,
                "beta_for_smooth_term_1": args.feas_beta / np.sqrt(b_fit) if b_fit > 0 else None,
                "seconds_per_eval_at_that_M": sec,
                "hours_for_64_chains_x_1e4_steps_plain": sec * 64 * 1e4 / 3600,
                "note": "cost per evaluation from the measured time, proportional to M"}

    # --- surrogate trained on particle-map pairs near the start state
    u0 = sm.start_states(prob, 64, spread=0.0)
    center = u0[0] if args.train_spread > 0 else None
    spread = args.train_spread if args.train_spread > 0 else 1.0
    coords = sm.screen_coords(prob, center, spread) if args.screen_coords == "local" else sm.screen_coords(prob)
    t0 = time.perf_counter()
    Z, G = sm.training_pairs(ctx, prob, args.train_pairs, center=center, spread=spread, tensor=args.tensor,
                             coords=coords)
    t_pairs = time.perf_counter() - t0
    Zv, Gv = sm.training_pairs(ctx, prob, 2048, seed=7005, center=center, spread=spread, tensor=args.tensor,
                               coords=coords)
    t1 = time.perf_counter()
    net, hist = sm.train_surrogate(ctx, prob, Z, G, epochs=args.epochs, weight_decay=args.weight_decay,
                                   lr_decay=args.lr_decay)
    t_train = time.perf_counter() - t1
    rmse = sm.surrogate_rmse(ctx, net, Zv, Gv)

    beta = float(args.betas.split(",")[0])

    def both(pr, steps_plain, steps_da):
        plain, mp = sm.run_chains_tracked(ctx, pr, u0, beta, steps_plain, seed=11, tensor=args.tensor)
        da, md = sm.run_chains_tracked(ctx, pr, u0, beta, steps_da, seed=11, net=net, tensor=args.tensor,
                                       coords=coords)
        out = {"plain": plain, "delayed_acceptance": da,
               "accepted_per_s_ratio": da["accepted_per_s"] / max(plain["accepted_per_s"], 1e-30)}
        if plain["accepts"] and da["accepts"]:
            ep, _ = sm.posterior_mean_error(mp)
            ed, _ = sm.posterior_mean_error(md)
            tp = plain["wall_seconds"] * (ep / 1e-2) ** 2
            td = da["wall_seconds"] * (ed / 1e-2) ** 2
            out["posterior_mean_rel_error"] = {"plain": ep, "delayed_acceptance": ed}
            out["seconds_to_1e-2"] = {"plain": tp, "delayed_acceptance": td, "ratio_plain_over_da": tp / td}
        return out

    configured = both(prob, args.plain_steps, args.da_steps)
    mprob = sm.make_problem(M=M0, sigma=args.move_sigma)
    mprob.u_true = u_true
    mprob.y = sm.forward_many(ctx, mprob, u_true[None, :], tensor=args.tensor)[0] + args.move_sigma * (
        np.random.Generator(np.random.PCG64(6004)).standard_normal(n_obs))
    moving = both(mprob, args.move_plain_steps, args.move_da_steps)
    pm.pm_surrogate_destroy(net)
    value = configured["delayed_acceptance"]["accepted_per_s"]
    line = {"metric": "accepted pCN samples/s (64 chains), surrogate-screened vs plain", "auxiliary": True,
            "data": "synthetic", "value": value, "unit": "accepted samples/s",
            "config": {"sigma": args.sigma, "M": M0, "n_obs": n_obs, "beta": beta, "chains": 64,
                       "train_pairs": args.train_pairs, "epochs": args.epochs, "start": "data-generating field",
                       "tensor_cores": bool(args.tensor),
                       "training_inputs": (f"local: start state + {args.train_spread} x prior std x N(0, I)"
                                           if args.train_spread > 0 else "prior draws"),
                       "screen_coords": args.screen_coords},
            "configured": configured,
            "feasibility": {"beta": args.feas_beta, "proposals": 32, "by_M": feas, "chains_move_at": need},
            "moving": dict(moving, sigma=args.move_sigma,
                           note="a larger noise than configured, where the chains move: not the configured target"),
            "surrogate": {"val_rmse": rmse, "final_train_loss": float(hist[-1]), "train_seconds": t_train,
                          "pair_generation_seconds": t_pairs}}
    print(json.dumps(line), flush=True)
    pm.pm_destroy(ctx)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32-compare", action="store_true",
                    help="skip timing the FP32-pipe kernel beside the tensor-core one")
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="timedep: skip the one FP64-path evaluation reported beside the line")
    ap.add_argument("--M", type=int, default=0, help="particles per observation (default: the workload's own; "
                    "smaller values are for profiling captures only)")
    ap.add_argument("--sweep-k", default="", help="sweep: comma-separated K values (default 2..80)")
    ap.add_argument("--workload", default="timedep", choices=["timedep", "dirichlet", "dirichlet_general", "batched", "mcmc", "sweep", "surrogate",
                             "bvp", "layout"],
                    help="timedep: the headline line; dirichlet / batched / mcmc: auxiliary measurements")
    ap.add_argument("--train-pairs", type=int, default=1 << 16, help="mcmc: surrogate training pairs")
    ap.add_argument("--betas", default="0.03", help="mcmc: comma-separated pCN steps (each the same for both samplers)")
    ap.add_argument("--sigma", type=float, default=0.01,
                    help="mcmc: observation noise standard deviation (the configured 0.01)")
    ap.add_argument("--move-sigma", type=float, default=0.1,
                    help="mcmc: the larger noise at which the samplers are also compared (chains move)")
    ap.add_argument("--feas-M", default="4096,16384,65536", help="mcmc: particle counts of the feasibility sweep")
    ap.add_argument("--feas-beta", type=float, default=0.005, help="mcmc: pCN step of the feasibility proposals")
    ap.add_argument("--move-plain-steps", type=int, default=40, help="mcmc: plain steps at --move-sigma")
    ap.add_argument("--move-da-steps", type=int, default=200, help="mcmc: delayed-acceptance steps at --move-sigma")
    ap.add_argument("--epochs", type=int, default=100, help="mcmc: surrogate training epochs")
    ap.add_argument("--screen-coords", default="prior", choices=["prior", "local"],
                    help="mcmc: surrogate input u / prior std, or (u - start) / (spread x prior std)")
    ap.add_argument("--train-spread", type=float, default=0.1,
                    help="mcmc: training inputs local to the start states with this spread (prior-std units); "
                         "0: prior draws")
    ap.add_argument("--weight-decay", type=float, default=0.0, help="mcmc: AdamW weight decay")
    ap.add_argument("--lr-decay", type=float, default=1.0, help="mcmc: per-epoch step-size factor")
    ap.add_argument("--plain-steps", type=int, default=8, help="mcmc: steps of the plain sampler (configured sigma)")
    ap.add_argument("--da-steps", type=int, default=50, help="mcmc: delayed-acceptance steps (configured sigma)")
    ap.add_argument("--B", type=int, default=256, help="instances of the batched workload")
    ap.add_argument("--K", type=int, default=0, help="dirichlet, batched: wave-number bound (default: the workload's 10)")
    ap.add_argument("--tensor", dest="tensor", action="store_true", default=True,
                    help="timedep: velocity sum on the tensor cores (PM_TENSOR; the default)")
    ap.add_argument("--no-tensor", dest="tensor", action="store_false",
                    help="timedep: velocity sum on the FP32 pipes")
    ap.add_argument("--autotune", action="store_true",
                    help="dirichlet / batched: pick the persistent grid with the autotuner first")
    ap.add_argument("--share-paths", action="store_true",
                    help="timedep: observations at one point share their paths (PM_SHARE_PATHS, tensor path); "
                         "value counts the steps taken, forward_map_evals_per_s the evaluations")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "mcmc":
        return run_mcmc(args)
    if args.workload == "sweep":
        return run_sweep(args)
    if args.workload == "surrogate":
        return run_surrogate(args)
    if args.workload == "bvp":
        return run_bvp(args)
    if args.workload == "layout":
        return run_layout(args)
    if args.workload != "timedep":
        return run_aux(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
