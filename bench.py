#!/usr/bin/env python
"""Benchmark of the SC-4DVAR Gauss-Newton hot path on GB300.

Metric: GN Hessian-vector products per second for a block of k = 128 directions
(the sketch block of the randomized preconditioners), and the GN-step time to a
1e-6 relative residual of the sketched mixed-precision solve against plain FP64
CG (the paper's Prec_Gamma), both on one GB300.

Workload: periodic 1D viscous Burgers, n = 8192, nu = 0.005, output step 5e-5
over 400 output steps (32 RK4 substeps each, 12 800 RK4 steps), observations
every 10 output steps at every 8th grid point (m = 40 960), squared-exponential
prior (sigma_b = 0.1, L = 0.05), synthetic seeded truth / background /
observations. TLM/ADJ sweeps in FP32, reductions and Gram matrices in FP64.

One timed step = one call of sc4dvar_gn_hessian_apply_block with k = 128 FP32
directions (prior square root, TLM sweep, ADJ sweep, prior square root, + X).
The L2 cache (129 MB) is flushed by a 256 MiB write before every timed step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("GN Hessian-vector products/s (block k) and GN-step time to 1e-6 rel. residual "
          "vs plain FP64 PCG")
WORKLOAD = "burgers_n8192"
K_BLOCK = 128
FP32_PEAK_ALU = 152 * 128 * 2 * 2.070e9   # FMA lanes x 2 flops x max SM clock (flop/s)
FP64_PEAK_FMA = 1.20e12   # FP64 FMA throughput measured by a microbenchmark on the same GB300s (flop/s)
# Algorithmic FP32 flops per grid point per RK4 step of one direction, counted
# from the expanded tangent-linear / adjoint stencil formulas (base-state stage
# recomputation not counted): TLM 52, ADJ 55. The kernels evaluate factored
# forms of the same operators with fewer operations, so these counts are the
# method's work, not the instructions executed.
FLOPS_TLM = 52
FLOPS_ADJ = 55
KERNELS = {"tlm": "tlm1_kernel<8>", "adj": "adj1_kernel<16>"}
# DRAM bytes (read + write) per launch of the k=128 FP32 sweeps, from ncu
# (dram__bytes_read.sum + dram__bytes_write.sum) on the 1280-step profile case
# (bench.py --profile), scaled by the step count to the 12 800-step launch.
# Set to None when the kernels change.
TRAFFIC_PER_LAUNCH = {"tlm": (46.178560e6 + 0.083712e6) * 10, "adj": (44.093696e6 + 0.191488e6) * 10}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-gn-step", action="store_true", help="skip the time-to-solution part")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-bve", action="store_true", help="skip the 256^2 vorticity block of the default run")
    ap.add_argument("--workload", default=WORKLOAD, choices=[WORKLOAD, "bve_n256", "bve_n1024", "burgers_batch64", "burgers_paper",
                                                             "bve_gyre"],
                    help="the Burgers block (default) or the barotropic vorticity block")
    ap.add_argument("--gn-iters", type=int, default=25,
                    help="GN iterations of the double-gyre experiment (the paper runs 25) and of the "
                         "1024^2 vorticity comparison (its workload: 5)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the double-gyre and 64-problem batch measurements of the default run")
    ap.add_argument("--profile", action="store_true",
                    help="small case for ncu: first 40 output steps, one TLM and one ADJ block")
    ap.add_argument("--profile-sketch", action="store_true",
                    help="for ncu: two FP32 RandSVD l = 128 sketches of the n = 8192 workload (a warm-up "
                         "and the profiled one), the sketch of the GN-step comparison")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.proc = None
        self.lines = []
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
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
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CPU baseline (oracle)
def oracle_sample(k_sample=8, n_out=40):
    """Oracle block Hessian product on a bounded sample of the workload: the full
    grid and step size, the first n_out output steps (of 400), k_sample directions.
    Returns (seconds, HVP/s scaled to the full 400-step window, description)."""
    import sc4dvar_inputs as si
    from oracle import workload
    wl_full = si.burgers_workload(WORKLOAD)
    wl = si.burgers_workload(WORKLOAD, n_out=n_out)
    draws = si.burgers_draws(wl)
    ref = workload.burgers_problem(wl, draws)
    ref.set_iterate(np.zeros(wl.n))
    X = si.gaussian_matrix(wl.seed, wl.n, k_sample, stream=31)
    t0 = time.perf_counter()
    ref.hvp(X)
    dt = time.perf_counter() - t0
    scale = wl_full.n_steps / wl.n_steps
    desc = (f"oracle (numpy FP64, 1 thread) (I+H)X on n={wl.n}, k={k_sample}, first "
            f"{wl.n_steps} of {wl_full.n_steps} RK4 steps; HVP/s scaled by {scale:g} to the full window")
    return dt, k_sample / (dt * scale), desc


def _oracle_worker(job):
    """One host process of the parallel oracle sample: FWD over the sample window
    (untimed), then the timed block (I + H) X of its columns."""
    n_out, cols = job
    import sc4dvar_inputs as si
    from oracle import workload
    wl = si.burgers_workload(WORKLOAD, n_out=n_out)
    ref = workload.burgers_problem(wl, si.burgers_draws(wl))
    ref.set_iterate(np.zeros(wl.n))
    X = si.gaussian_matrix(wl.seed, wl.n, max(cols) + 1, stream=31)[:, cols]
    t0 = time.perf_counter()
    ref.hvp(X)
    return time.perf_counter() - t0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def oracle_sample_parallel(cols_per_core=2, n_out=40):
    """The oracle block Hessian product on every host core at once (one process
    per core, spawned, numpy FP64 single-threaded in each), cols_per_core
    directions per process over the first n_out output steps. Returns (seconds of
    the slowest process, HVP/s of all processes scaled to the full window, cores,
    description)."""
    import multiprocessing as mp
    import sc4dvar_inputs as si
    cores = host_cores()
    jobs = [(n_out, list(range(c * cols_per_core, (c + 1) * cols_per_core))) for c in range(cores)]
    env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(cores) as pool:
            secs = pool.map(_oracle_worker, jobs)
    finally:
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    wl_full = si.burgers_workload(WORKLOAD)
    wl = si.burgers_workload(WORKLOAD, n_out=n_out)
    scale = wl_full.n_steps / wl.n_steps
    dt = max(secs)
    k = cores * cols_per_core
    desc = (f"oracle (numpy FP64) (I+H)X on n={wl.n}, {cores} processes x {cols_per_core} directions "
            f"(k={k}) in parallel, first {wl.n_steps} of {wl_full.n_steps} RK4 steps; HVP/s = k / slowest "
            f"process, scaled by {scale:g} to the full window")
    return dt, k / (dt * scale), cores, desc


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import sc4dvar_inputs as si
    wl = si.burgers_workload(WORKLOAD)
    times, vals = [], []
    desc, cores = "", 1
    for i in range(args.warmup + args.steps):
        dt, v, cores, desc = oracle_sample_parallel(cols_per_core=1, n_out=20)
        if i >= args.warmup:
            times.append(dt)
            vals.append(v)
    value = statistics.mean(vals)
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "HVP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(wl),
        "cpu_baseline": {"value": value, "unit": "HVP/s", "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "HVP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def config_dict(wl):
    return {"workload": f"{wl.name}: periodic Burgers n={wl.n}, nu={wl.nu}, {wl.n_steps} RK4 steps "
                        f"(dt_out={wl.dt_out}, {wl.substeps} substeps), m={wl.m} observations, "
                        f"block k={K_BLOCK}, FP32 sweeps",
            "n": wl.n, "rk_steps": wl.n_steps, "m": wl.m, "k": K_BLOCK,
            "l2": "256 MiB write before every timed step"}


# ------------------------------------------------------------------ GPU arm
def max_over_ranks(dist, value, device):
    """The largest per-rank value over all ranks (the slowest replica sets the
    job time); `dist` is torch.distributed or None for one process."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, seconds):
    """Whole-job throughput: every replica processes units_per_rank units (weak
    scaling, no data-path exchange), the job takes the slowest rank's time."""
    return units_per_rank * world / seconds


def setup_problem(torch, dev):
    import paper_2401_15758_gb300 as g
    import sc4dvar_inputs as si
    wl = si.burgers_workload(WORKLOAD)
    d = si.burgers_draws(wl)
    prob = g.Problem.from_workload(wl, d["obs_idx"])
    xt = torch.tensor(d["x_true0"], device=dev)
    obs, _ = prob.forecast(xt)
    y = obs + wl.sigma_obs * torch.tensor(d["xi_o"].reshape(-1), device=dev)
    xb = xt + prob.prior_sqrt_apply(torch.tensor(d["xi_b"], device=dev))
    prob.set_background(xb)
    prob.set_observations(y)
    v0 = torch.zeros(wl.n, dtype=torch.float64, device=dev)
    J0 = prob.fwd(v0)
    return g, si, wl, prob, J0


# Barotropic vorticity block (HBM-bound streaming sweeps). Algorithmic bytes
# per Hessian product per grid point per RK4 step (FP32, 4 B values), counted
# from the kernels: per TLM stage a 2D FFT multiplier on one field (6 field
# passes: real in, complex out/in/out/in, real out) plus the stencil stage (6
# field passes); per ADJ stage one Jacobian pass (2), the multiplier (6) and
# the stage kernel (6): 4 x (12 + 14) = 104 field passes per step.
BVE_PASSES_PER_STEP = 104


def gn_run_comparison(torch, g, prob, wl, dev, iters, sketch):
    """Time to solution of `iters` Gauss-Newton iterations from v = 0, each step
    solved to a 1e-6 relative residual: the sketched method (FP32 sketch reused
    while kappa_re < eps_re = 10, Eq. condtext2, FP32-operator PCG with FP64
    defect correction) against plain FP64 CG (Prec_Gamma). FWD and gradients
    are inside both times."""
    res = {}
    for name, opts in (("method", dict(prec=g.FP32, **sketch)), ("plain_fp64_cg", dict(method="none"))):
        prob.counters_reset()
        v = torch.zeros(wl.n, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rec = prob.gauss_newton(v, iters=iters, tol=1e-6, seed=wl.seed, **opts)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        c = prob.counters()
        res[name] = {"seconds": secs, "pcg_its": [r["pcg_its"] for r in rec],
                     "sketched": [bool(r["sketched"]) for r in rec], "rank": [r["rank"] for r in rec],
                     "kappa_re": [r["kappa_re"] for r in rec], "J": [r["J"] for r in rec],
                     "relres": [r["relres"] for r in rec], "counters": c}
        print(f"{name}: {json.dumps(res[name])}", file=sys.stderr, flush=True)
    res["speedup"] = res["plain_fp64_cg"]["seconds"] / res["method"]["seconds"]
    res["iters"] = iters
    res["sketch"] = dict(sketch)
    res["unit"] = "s"
    return res


def bve_block(name, steps, warmup, with_gn=True, gn_iters=0):
    """Block Hessian product of a vorticity workload (FP32 sweeps, k = the
    workload's block) timed with CUDA events (256 MiB L2 flush before every
    step), the autograd gradient, and optionally the GN step to 1e-6 against
    plain FP64 CG. Returns a dict."""
    import torch
    import paper_2401_15758_gb300 as g
    import sc4dvar_inputs as si
    dev = torch.device("cuda", 0)
    wl = si.bve_workload(name)
    d = si.bve_draws(wl)
    prob = g.Problem.from_bve_workload(wl, d)
    xt = torch.tensor(d["x_true0"], device=dev)
    obs, _ = prob.forecast(xt)
    prob.set_observations(obs + d["sigma_obs"] * torch.tensor(d["xi_o"].reshape(-1), device=dev))
    prob.set_background(xt + prob.prior_sqrt_apply(torch.tensor(d["xi_b"], device=dev)))
    prob.fwd(torch.zeros(wl.n, dtype=torch.float64, device=dev))
    k = wl.k
    X = torch.tensor(si.gaussian_matrix(wl.seed, k, wl.n, stream=23), device=dev, dtype=torch.float32)
    Y = torch.empty_like(X)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        flush.zero_()
        prob.gn_hessian_apply_block(X, prec=g.FP32, out=Y)
    torch.cuda.synchronize()
    l0 = g.lib.sc4dvar_launch_count()
    ms = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        prob.gn_hessian_apply_block(X, prec=g.FP32, out=Y)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    launches = g.lib.sc4dvar_launch_count() - l0
    # gradient through the autograd cost: forward = FWD (keeps the checkpoints),
    # backward = adjoint sweep recomputing each segment
    v = torch.zeros(wl.n, dtype=torch.float64, device=dev, requires_grad=True)
    grad_ms = []
    for i in range(4):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        v.grad = None
        a.record(stream)
        g.cost(prob, v).backward()
        b.record(stream)
        torch.cuda.synchronize()
        if i:
            grad_ms.append(a.elapsed_time(b))
    t = statistics.mean(ms) / 1e3
    nbytes = BVE_PASSES_PER_STEP * wl.n * 4 * wl.n_steps * k
    gn = None
    if with_gn and gn_iters <= 1:
        if wl.n_checkpoints:
            # 1024^2 set-up: Nystrom sketch of the block size (k = 512)
            sk = {"method": "nystrom", "l": k}
        else:
            # SketchPrecA set-up: adaptive RandSVD from l0 = k, growing by k/2 to eps_sk = 1.01
            sk = {"method": "randsvd", "l": k, "adaptive": True, "l_hat": k // 2, "eps_sk": 1.01}
        gn = gn_step(torch, g, prob, wl, dev, sketch=sk)
    gn_multi = None
    if with_gn and gn_iters > 1:
        # the sketch of the block size reused across the GN iterations under the
        # reuse rule (adaptive with l_max = l: reuse without growth)
        gn_multi = gn_run_comparison(torch, g, prob, wl, dev, gn_iters,
                                     {"method": "nystrom", "l": k, "adaptive": True, "l_max": k,
                                      "eps_re": 10.0})
    peak = measured_hbm_gbs()
    out = {"value": k / t, "unit": "HVP/s", "ms_per_step": 1e3 * t, "steps": steps, "warmup": warmup,
           "workload": f"{wl.name}: doubly periodic barotropic vorticity {wl.N}x{wl.N}, "
                       f"{wl.n_steps} RK4 steps, m={wl.m}, block k={k}, FP32 sweeps"
                       + (f", {wl.n_checkpoints} FP64 checkpoints" if wl.n_checkpoints else ""),
           "n": wl.n, "rk_steps": wl.n_steps, "m": wl.m, "k": k, "checkpoints": wl.n_checkpoints,
           "gradient_ms": statistics.mean(grad_ms),
           "roofline": {"bound": "hbm", "kernel": "block Hessian product (all sweep kernels)",
                        "achieved": nbytes / t / 1e9, "peak": peak, "unit": "GB/s",
                        "frac": nbytes / t / 1e9 / peak, "traffic": None,
                        "algorithmic_bytes": nbytes, "peak_source": hbm_peak()[1]},
           "gpu_launches": int(launches)}
    if gn is not None:
        out["gn_step"] = gn
    if gn_multi is not None:
        out["gn_iterations"] = gn_multi
    prob.close()
    return out


def bve_arm(args):
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    r = bve_block(args.workload, args.steps, args.warmup, with_gn=not args.no_gn_step,
                  gn_iters=args.gn_iters if args.workload == "bve_n1024" else 0)
    clk = clocks.stop()
    out = {"metric": METRIC, "value": r["value"], "unit": "HVP/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": r["workload"], "n": r["n"], "rk_steps": r["rk_steps"], "m": r["m"],
                      "k": r["k"], "checkpoints": r["checkpoints"],
                      "l2": "256 MiB write before every timed step"},
           "gradient_ms": r["gradient_ms"], "roofline": r["roofline"], "gpu_launches": r["gpu_launches"],
           "clocks": clk}
    if "gn_step" in r:
        out["gn_step"] = r["gn_step"]
    if "gn_iterations" in r:
        out["gn_iterations"] = r["gn_iterations"]
    print(json.dumps(out), flush=True)


def batch_arm(args, emit=True):
    """64 uneven Burgers problems: one graph-replayed batched block Hessian
    product (FP32 sweeps) per step; HVP/s = sum of the block widths / time.
    Prints its JSON line, or returns it with emit=False."""
    import torch
    import paper_2401_15758_gb300 as g
    import sc4dvar_inputs as si
    dev = torch.device("cuda", 0)
    probs, Xs = [], []
    items = si.burgers_batch(64)
    for wl, d in items:
        p = g.Problem.from_workload(wl, d["obs_idx"])
        xt = torch.tensor(d["x_true0"], device=dev)
        obs, _ = p.forecast(xt)
        p.set_observations(obs + wl.sigma_obs * torch.tensor(d["xi_o"].reshape(-1), device=dev))
        p.set_background(xt + p.prior_sqrt_apply(torch.tensor(d["xi_b"], device=dev)))
        p.fwd(torch.zeros(wl.n, dtype=torch.float64, device=dev))
        g.autotune(p, wl.k)
        probs.append(p)
        Xs.append(torch.tensor(si.gaussian_matrix(wl.seed, wl.k, wl.n, stream=25), device=dev,
                               dtype=torch.float32))
    Ys = [torch.empty_like(x) for x in Xs]
    b = g.Batch(probs)
    total_k = sum(x.shape[0] for x in Xs)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(max(1, args.warmup)):
        b.hessian_apply(Xs, Ys, prec=g.FP32)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    l0 = g.lib.sc4dvar_launch_count()
    ms = []
    for _ in range(args.steps):
        flush.zero_()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        b.hessian_apply(Xs, Ys, prec=g.FP32)
        e.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(e))
    launches = g.lib.sc4dvar_launch_count() - l0
    # batched PCG (FP32 operator, no preconditioner): one graph launch advances
    # every problem by one iteration; time per iteration over 20 iterations
    rhs = [-p.gradient() for p in probs]
    b.pcg_start(rhs, None, tol=1e-6, prec=g.FP32)
    b.pcg_step(2)
    torch.cuda.synchronize()
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    b.pcg_step(20)
    e.record(stream)
    torch.cuda.synchronize()
    pcg_ms = a.elapsed_time(e) / 20
    rel, its, _ = b.pcg_status()
    clk = clocks.stop()
    t = statistics.mean(ms) / 1e3
    flops = sum((FLOPS_TLM + FLOPS_ADJ) * wl.n * wl.n_steps * wl.k for wl, _ in items)
    out = {"metric": METRIC, "value": total_k / t, "unit": "HVP/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "burgers_batch64: 64 Burgers problems, n in {512..8192}, "
                                  "N_out in {100,200,400}, k in {16,32,64} per problem",
                      "problems": 64, "total_k": total_k,
                      "l2": "256 MiB write before every timed step"},
           "roofline": {"bound": "alu", "kernel": "batched sweeps (all problems, one graph)",
                        "achieved": flops / t / 1e12, "peak": FP32_PEAK_ALU / 1e12, "unit": "TFLOP/s",
                        "frac": flops / t / FP32_PEAK_ALU, "traffic": None},
           "gpu_launches": int(launches), "graph_launches_per_step": 1, "clocks": clk,
           "batched_pcg": {"ms_per_iteration": pcg_ms, "problems": len(probs),
                           "note": "one graph launch = one FP32-operator PCG iteration of all 64 problems",
                           "iterations_done": int(max(its)), "max_relres": float(max(rel))}}
    b.close()
    for p in probs:
        p.close()
    if not emit:
        return out
    print(json.dumps(out), flush=True)


def paper_counts(table):
    """PDE-solve counts the paper prints for one table (tests/golden/paper_counts.txt)."""
    paper = {}
    with open(os.path.join(ROOT, "tests", "golden", "paper_counts.txt")) as f:
        for line in f:
            if line.startswith(table + " "):
                _, meth, *vals = line.split()
                paper[meth] = [None if v == "-" else int(v) for v in vals]
    return paper


def paper_runs(torch, dev, problem, n, table, runs, iters, tol):
    """Gauss-Newton from v = 0 for each (name, options) run on a fresh problem,
    strong-Wolfe steps; PDE-solve counters and wall time next to the paper's
    counts of the same method."""
    paper = paper_counts(table)
    rows = {}
    for name, opts in runs:
        p = problem()
        p.counters_reset()
        v = torch.zeros(n, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rec = p.gauss_newton(v, iters=iters, tol=tol, gtol=1e-6, line_search=True, **opts)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        c = p.counters()
        ours = {"pcg_its": sum(r["pcg_its"] for r in rec), "tlm_off": c["tlm_offline"],
                "adj_off": c["adj_offline"], "fwd": c["fwd"], "tlm_on": c["tlm_online"],
                "adj_on": c["adj_online"], "gn_iters": len(rec), "J_final": rec[-1]["J"],
                "sketched_at": [i + 1 for i, r in enumerate(rec) if r["sketched"]],
                "ranks": sorted({r["rank"] for r in rec}),
                "alphas": [r["alpha"] for r in rec], "seconds": secs}
        pr = paper.get(name)
        rows[name] = {"ours": ours, "paper": None if pr is None else dict(
            zip(("pcg_its", "tlm_off", "adj_off", "fwd", "tlm_on", "adj_on"), pr))}
        print(f"{name}: {json.dumps(ours)}", file=sys.stderr, flush=True)
        p.close()
    return rows


def paper_arm(args):
    """The Burgers experiment of Sec. 5.1 (Dirichlet, RK3-TVD, n = 399, 8000 steps,
    15 sites, 20 times): 3 GN iterations with l = l1 = 15, l2 = 31, PCG to 1e-9,
    strong-Wolfe steps, FP64, for Prec_Gamma and the three sketches as PCG
    preconditioners (SketchPrec) and as direct steps (SketchSolv);
    PDE-solve counts and times next to the counts the paper prints (Table 3).
    The block product of the sketch size (k = 15, FP64) is the timed step."""
    import torch
    import paper_2401_15758_gb300 as g
    import sc4dvar_inputs as si
    dev = torch.device("cuda", 0)
    wl = si.paper_burgers_workload()
    d = si.paper_burgers_draws(wl)

    def problem():
        p = g.Problem.from_paper_burgers_workload(wl, d)
        xt = torch.tensor(d["x_true0"], device=dev)
        obs, _ = p.forecast(xt)
        p.set_observations(obs + wl.sigma_obs * torch.tensor(d["xi_o"].reshape(-1), device=dev))
        p.set_background(xt + p.prior_sqrt_apply(torch.tensor(d["xi_b"], device=dev)))
        return p

    runs = [(name, dict(method=method, solve=solve, l=wl.k, l2=2 * wl.k + 1))
            for method, solve, name in
            [("none", "pcg", "Prec_Gamma"), ("randsvd", "pcg", "SketchPrec_RandSVD"),
             ("nystrom", "pcg", "SketchPrec_Nystrom"), ("singleview", "pcg", "SketchPrec_SingleView"),
             ("randsvd", "sketchsolv", "SketchSolv_RandSVD"), ("nystrom", "sketchsolv", "SketchSolv_Nystrom"),
             ("singleview", "sketchsolv", "SketchSolv_SingleView")]]
    rows = paper_runs(torch, dev, problem, wl.n, "T3", runs, iters=3, tol=1e-9)
    # timed step: FP64 block product of the sketch size
    p = problem()
    p.fwd(torch.zeros(wl.n, dtype=torch.float64, device=dev))
    X = torch.tensor(si.gaussian_matrix(wl.seed, wl.k, wl.n, stream=29), device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        p.gn_hessian_apply_block(X)
    torch.cuda.synchronize()
    ms = []
    for _ in range(args.steps):
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        p.gn_hessian_apply_block(X)
        e.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(e))
    t = statistics.mean(ms) / 1e3
    out = {"metric": METRIC, "value": wl.k / t, "unit": "HVP/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"{wl.name}: Dirichlet Burgers n={wl.n}, nu={wl.nu}, RK3-TVD, "
                                  f"{wl.n_steps} steps, m={wl.m}, block k={wl.k}, FP64",
                      "n": wl.n, "rk_steps": wl.n_steps, "m": wl.m, "k": wl.k},
           "paper_table3_comparison": rows}
    print(json.dumps(out), flush=True)


def gyre_arm(args, emit=True):
    """The barotropic vorticity experiment of Sec. 5.2 (double gyre in a closed
    basin, 128 x 257 interior points, RK3-TVD, 40 steps, 8 observation times of
    a 16 x 16 sensor grid): 25 GN iterations, PCG to 1e-9, strong-Wolfe steps,
    FP64, for Prec_Gamma, the three sketches with l = l1 = 384 (l2 = 769)
    recomputed every iteration (SketchPrec), and the adaptive sketches with the
    reuse rule (SketchPrecA: l0 = l_hat = 128, eps_sk = 1.01, eps_re = 10);
    PDE-solve counts and times next to the counts the paper prints (Table 4).
    The timed step is the FP64 block product of the sketch size (k = 384)."""
    import torch
    import paper_2401_15758_gb300 as g
    import sc4dvar_inputs as si
    dev = torch.device("cuda", 0)
    wl = si.gyre_workload()
    d = si.gyre_draws(wl)
    # spun-up truth: init_scale Gamma^{1/2} xi_init advanced spin_steps steps by
    # the library's own forecast over a window of that length
    spin = si.gyre_workload(obs_every=wl.spin_steps // 8, n_obs_times=8)
    ps = g.Problem.from_gyre_workload(spin, si.gyre_draws(spin))
    x_init = wl.init_scale * ps.prior_sqrt_apply(torch.tensor(d["xi_init"], device=dev))
    _, xt = ps.forecast(x_init)
    ps.close()

    def problem():
        p = g.Problem.from_gyre_workload(wl, d)
        obs, _ = p.forecast(xt)
        p.set_observations(obs + wl.sigma_obs * torch.tensor(d["xi_o"].reshape(-1), device=dev))
        p.set_background(xt + p.prior_sqrt_apply(torch.tensor(d["xi_b"], device=dev)))
        return p

    fixed = dict(l=wl.k, l2=2 * wl.k + 1)
    adapt = dict(adaptive=True, l=128, l_hat=128, l2=257, l_max=2048, eps_sk=1.01, eps_re=10.0)
    runs = [("Prec_Gamma", dict(method="none")),
            ("SketchPrec_RandSVD", dict(method="randsvd", **fixed)),
            ("SketchPrec_Nystrom", dict(method="nystrom", **fixed)),
            ("SketchPrec_SingleView", dict(method="singleview", **fixed)),
            ("SketchPrecA_RandSVD", dict(method="randsvd", **adapt)),
            ("SketchPrecA_Nystrom", dict(method="nystrom", **adapt)),
            ("SketchPrecA_SingleView", dict(method="singleview", **adapt))]
    if args.gn_iters < 25:
        runs = [r for r in runs if r[0] != "Prec_Gamma"] + [("Prec_Gamma", dict(method="none"))]
    p = problem()
    p.fwd(torch.zeros(wl.n, dtype=torch.float64, device=dev))
    X = torch.tensor(si.gaussian_matrix(wl.seed, wl.k, wl.n, stream=29), device=dev)
    X32 = X.float()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.steps):
            flush.zero_()
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            e.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(e))
        return statistics.mean(ms) / 1e3

    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    l0 = g.lib.sc4dvar_launch_count()
    t = timed(lambda: p.gn_hessian_apply_block(X))
    launches = (g.lib.sc4dvar_launch_count() - l0) // (args.warmup + args.steps)
    t32 = timed(lambda: p.gn_hessian_apply_block(X32, prec=g.FP32))
    clk = clocks.stop()
    x1 = X[:1].contiguous()
    t1 = timed(lambda: p.gn_hessian_apply_block(x1))
    # GN-step time to a 1e-6 residual at the background: FP32 RandSVD sketch of
    # the paper's size + mixed-precision PCG against plain FP64 CG
    gn = None if args.no_gn_step else gn_step(torch, g, p, wl, dev, sketch={"method": "randsvd", "l": wl.k})
    p.close()
    print(f"block k={wl.k}: FP64 {1e3 * t:.2f} ms, FP32 {1e3 * t32:.2f} ms; one FP64 product {1e3 * t1:.3f} ms",
          file=sys.stderr, flush=True)
    rows = (paper_runs(torch, dev, problem, wl.n, "T4", runs, iters=args.gn_iters, tol=wl.pcg_tol)
            if args.gn_iters > 0 else None)
    # flops of the sine transforms (the dense nx x nx products of every row): 12
    # per RK3 step (a Poisson solve per stage in each sweep, two transforms
    # each) and 4 for the two prior applies, 2 ny nx^2 flops per field each
    dst_flops = (12 * wl.n_steps + 4) * 2.0 * wl.ny * wl.nx * wl.nx * wl.k
    out = {"metric": METRIC, "value": wl.k / t, "unit": "HVP/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "roofline": {"bound": "alu", "kernel": "block Hessian product (all kernels; sine-transform flops)",
                        "achieved": dst_flops / t / 1e12, "peak": FP64_PEAK_FMA / 1e12, "unit": "TFLOP/s",
                        "frac": dst_flops / t / FP64_PEAK_FMA, "traffic": None,
                        "peak_source": "FP64 FMA microbenchmark on the pool's GB300 (1.20 TFLOP/s)"},
           "config": {"workload": f"{wl.name}: double-gyre vorticity {wl.nx}x{wl.ny} (Dirichlet), "
                                  f"Re={wl.re}, Ro={wl.ro}, RK3-TVD, {wl.n_steps} steps, m={wl.m}, "
                                  f"block k={wl.k}, FP64",
                      "n": wl.n, "rk_steps": wl.n_steps, "m": wl.m, "k": wl.k, "gn_iters": args.gn_iters,
                      "l2": "256 MiB write before every timed step"},
           "fp32_block": {"value": wl.k / t32, "unit": "HVP/s", "ms_per_step": 1e3 * t32,
                          "roofline": {"bound": "alu", "achieved": dst_flops / t32 / 1e12,
                                       "peak": FP32_PEAK_ALU / 1e12, "unit": "TFLOP/s",
                                       "frac": dst_flops / t32 / FP32_PEAK_ALU}},
           "single_fp64_product_ms": 1e3 * t1,
           "gpu_launches_per_step": int(launches), "clocks": clk,
           "gn_step": gn, "paper_table4_comparison": rows}
    if not emit:
        return out
    print(json.dumps(out), flush=True)


def measured_hbm_gbs():
    return hbm_peak()[0]


def hbm_peak():
    """(GB/s, source): the measured copy bandwidth of MEASURED_PEAKS.json, else
    the 6.8 TB/s fallback of an earlier measurement on a GB300."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (of measured)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6800 GB/s (MEASURED_PEAKS.json absent; of fallback)"


def gpu_arm(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    g, si, wl, prob, J0 = setup_problem(torch, dev)
    stream = torch.cuda.current_stream()
    k = K_BLOCK
    X = torch.tensor(si.gaussian_matrix(wl.seed, k, wl.n, stream=21), device=dev, dtype=torch.float32)
    Y = torch.empty_like(X)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        prob.gn_hessian_apply_block(X, prec=g.FP32, out=Y)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = g.lib.sc4dvar_launch_count()
    for i in range(args.steps):
        flush.zero_()
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    launches = g.lib.sc4dvar_launch_count() - l0
    if dist:
        dist.barrier()
    ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = max_over_ranks(dist, sum(ms), dev)
    value = job_throughput(k * args.steps, world, total_ms / 1e3)

    # dominant kernels: ADJ and TLM sweeps timed alone (each call = sweep + one prior FFT pass)
    W = torch.empty((k, wl.m), dtype=torch.float32, device=dev)
    Z = torch.empty_like(X)
    kern = {}
    for name, fn in (("tlm", lambda: prob.tlm_block(X, prec=g.FP32, out=W)),
                     ("adj", lambda: prob.adj_block(W, prec=g.FP32, out=Z))):
        fn()
        reps = []
        for _ in range(3):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            reps.append(a.elapsed_time(b))
        kern[name] = statistics.mean(reps)
    clk = clocks.stop()
    dom = max(kern, key=kern.get)
    flops = (FLOPS_ADJ if dom == "adj" else FLOPS_TLM) * wl.n * wl.n_steps * k
    achieved = flops / (kern[dom] / 1e3) / 1e12
    peak = FP32_PEAK_ALU / 1e12
    roofline = {"bound": "alu", "kernel": KERNELS[dom], "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": TRAFFIC_PER_LAUNCH.get(dom),
                "algorithmic_bytes": wl.n_steps * wl.n * 4,
                "peak_source": "152 SMs x 128 FP32 lanes x 2 flop/FMA x 2070 MHz (unit counts)",
                "kernel_ms": kern}

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    Xh = X.cpu().pin_memory()
    Yh = torch.empty_like(Xh).pin_memory()
    Xd = torch.empty_like(X)
    Yd = torch.empty_like(X)
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        Xd.copy_(Xh, non_blocking=True)
        prob.gn_hessian_apply_block(Xd, prec=g.FP32, out=Yd)
        Yh.copy_(Yd, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_ms.append(a.elapsed_time(b))
    e2e_val = k * world / (statistics.mean(e2e_ms) / 1e3)
    e2e = {"value": e2e_val, "unit": "HVP/s", "h2d_bytes_per_step": Xh.numel() * 4,
           "d2h_bytes_per_step": Yh.numel() * 4}

    # the same block through the FP64 and the double-float (DF64) sweeps, and the
    # error of every FP32 column against the FP64 product (the FP64 path matches
    # the oracle to 1e-10 in the parity tests)
    X64 = X.double()
    prec_var = {}
    Y64 = None
    for name, pr in (("fp64", g.FP64), ("df64", g.DF64)):
        Yv = torch.empty_like(X64)
        for _ in range(3):
            prob.gn_hessian_apply_block(X64, prec=pr, out=Yv)
        reps = []
        for _ in range(2):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            prob.gn_hessian_apply_block(X64, prec=pr, out=Yv)
            b.record(stream)
            torch.cuda.synchronize()
            reps.append(a.elapsed_time(b))
        t_v = statistics.mean(reps) / 1e3
        prec_var[name] = {"value": k / t_v, "unit": "HVP/s", "ms_per_step": 1e3 * t_v, "steps": 2, "warmup": 3}
        if name == "fp64":
            Y64 = Yv
        else:
            prec_var[name]["max_column_rel_err_vs_fp64"] = float(
                (torch.linalg.norm(Yv - Y64, dim=1) / torch.linalg.norm(Y64, dim=1)).max())
    prec_var["fp32"] = {"value": value, "unit": "HVP/s", "max_column_rel_err_vs_fp64": float(
        (torch.linalg.norm(Y.double() - Y64, dim=1) / torch.linalg.norm(Y64, dim=1)).max())}
    del Y64

    gn = None
    if not args.no_gn_step:
        gn = gn_step(torch, g, prob, wl, dev)

    # the 256^2 barotropic vorticity block (HBM-bound streaming sweeps) and its
    # GN step with the adaptive sketch, as an extra measurement on the same GPU
    bve = None
    if not args.no_bve and world == 1:
        prob.close()
        bve = bve_block("bve_n256", steps=3, warmup=3, with_gn=not args.no_gn_step)
    # the double-gyre experiment's block products (Sec. 5.2, FP64 and FP32, k =
    # 384) and the 64-problem batch, as further measurements on the same GPU
    extras = {}
    if not args.no_extras and world == 1:
        prob.close()
        ns = argparse.Namespace(steps=3, warmup=3, gn_iters=0, no_gn_step=True)
        gy = gyre_arm(ns, emit=False)
        extras["bve_gyre"] = {k: gy[k] for k in ("value", "unit", "ms_per_step", "dtype", "roofline", "config",
                                                 "fp32_block", "gpu_launches_per_step", "clocks")}
        bt = batch_arm(ns, emit=False)
        extras["burgers_batch64"] = {k: bt[k] for k in ("value", "unit", "ms_per_step", "dtype", "roofline",
                                                        "config", "gpu_launches", "batched_pcg", "clocks")}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "HVP/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic", "config": config_dict(wl), "roofline": roofline,
               "e2e": e2e, "gpu_launches": int(launches), "clocks": clk}
        out["precision_variants"] = prec_var
        if gn is not None:
            out["gn_step"] = gn
        if bve is not None:
            out["bve_n256"] = bve
        out.update(extras)
        if not args.no_cpu_baseline:
            dt, v, cores, desc = oracle_sample_parallel()
            dt1, v1, desc1 = oracle_sample()
            out["cpu_baseline"] = {"value": v, "unit": "HVP/s", "cores": cores, "kind": "oracle",
                                   "sample": desc, "seconds": dt,
                                   "one_thread": {"value": v1, "unit": "HVP/s", "cores": 1,
                                                  "sample": desc1, "seconds": dt1}}
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def gn_step(torch, g, prob, wl, dev, sketch=None):
    """GN-step time to a 1e-6 relative residual at the background iterate:
    sketched PCG (default RandSVD, k=128, FP32 sweeps) with FP64 defect
    correction vs plain FP64 CG (Prec_Gamma). FWD and gradient are shared by
    both and timed apart."""
    sketch = sketch or {"method": "randsvd", "l": K_BLOCK}
    v0 = torch.zeros(wl.n, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    prob.fwd(v0)
    gv = prob.gradient()
    torch.cuda.synchronize()
    t_fg = time.perf_counter() - t0
    b = -gv
    res = {}
    # method
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pc = prob.build_precond(prec=g.FP32, seed=wl.seed, **sketch)
    torch.cuda.synchronize()
    t_sk = time.perf_counter() - t0
    x, info = prob.pcg(b, pc, tol=1e-6, prec=g.FP32, refine=3)
    torch.cuda.synchronize()
    t_m = time.perf_counter() - t0
    res["method"] = {"seconds": t_m, "sketch_seconds": t_sk, "pcg_its": info["iterations"],
                     "restarts": info["restarts"], "relres_fp64": info["relres"],
                     "status": info["status"], "rank": pc.rank, "sketch": dict(sketch)}
    # plain FP64 CG
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    xp, infop = prob.pcg(b, None, tol=1e-6, prec=g.FP64)
    torch.cuda.synchronize()
    t_p = time.perf_counter() - t0
    # true FP64 residuals of both solutions (outside the timed regions)
    def true_rel(xx):
        r = b - prob.gn_hessian_apply_block(xx.reshape(1, -1)).reshape(-1)
        return float(torch.linalg.norm(r) / torch.linalg.norm(b))
    res["plain_fp64_cg"] = {"seconds": t_p, "pcg_its": infop["iterations"],
                            "relres_fp64": true_rel(xp), "status": infop["status"]}
    res["method"]["relres_fp64_check"] = true_rel(x)
    res["step_diff"] = float(torch.linalg.norm(x - xp) / torch.linalg.norm(xp))
    res["speedup"] = t_p / t_m
    res["fwd_gradient_seconds"] = t_fg
    res["unit"] = "s"
    pc.close()
    return res


def profile_case():
    """One FP32 TLM block and one FP32 ADJ block (k = 128) on the first 40 output
    steps of the workload (1280 RK4 steps): the kernels of the timed step on a
    window short enough for an ncu capture."""
    import torch
    import paper_2401_15758_gb300 as g
    import sc4dvar_inputs as si
    wl = si.burgers_workload(WORKLOAD, n_out=40)
    d = si.burgers_draws(wl)
    prob = g.Problem.from_workload(wl, d["obs_idx"])
    prob.set_background(torch.tensor(d["x_true0"], device="cuda"))
    prob.fwd(torch.zeros(wl.n, dtype=torch.float64, device="cuda"))
    X = torch.tensor(si.gaussian_matrix(wl.seed, K_BLOCK, wl.n, stream=21), device="cuda",
                     dtype=torch.float32)
    W = prob.tlm_block(X, prec=g.FP32)
    prob.adj_block(W, prec=g.FP32)
    torch.cuda.synchronize()
    print("profile case done")


def profile_case_sketch():
    """Two FP32 RandSVD sketches (l = 128) at the background of the n = 8192
    workload: the sketch phase of the GN step, for a launch list."""
    import torch
    dev = torch.device("cuda", 0)
    g, si, wl, prob, J0 = setup_problem(torch, dev)
    for _ in range(2):
        pc = prob.build_precond(method="randsvd", l=K_BLOCK, prec=g.FP32, seed=wl.seed)
        torch.cuda.synchronize()
        pc.close()
    print("sketch profile case done")


def profile_case_bve(name="bve_n256"):
    """One FP32 TLM block and one FP32 ADJ block of a vorticity workload on its
    first RK4 steps: 256^2 (k = 256) 20 steps; 1024^2 (k = 512) 16 steps with 4
    checkpoints (segments of 4 steps)."""
    import torch
    import paper_2401_15758_gb300 as g
    import sc4dvar_inputs as si
    if name == "bve_n1024":
        wl = si.bve_workload(name, n_steps=16, n_checkpoints=4)
    else:
        wl = si.bve_workload(name, n_steps=20)
    d = si.bve_draws(wl)
    prob = g.Problem.from_bve_workload(wl, d)
    prob.set_background(torch.tensor(d["x_true0"], device="cuda"))
    prob.fwd(torch.zeros(wl.n, dtype=torch.float64, device="cuda"))
    X = torch.tensor(si.gaussian_matrix(wl.seed, wl.k, wl.n, stream=23), device="cuda",
                     dtype=torch.float32)
    W = prob.tlm_block(X, prec=g.FP32)
    prob.adj_block(W, prec=g.FP32)
    torch.cuda.synchronize()
    print("bve profile case done")


def profile_case_gyre():
    """One FP32 TLM block and one FP32 ADJ block (k = 384) of the double-gyre
    workload over its 40-step window."""
    import torch
    import paper_2401_15758_gb300 as g
    import sc4dvar_inputs as si
    wl = si.gyre_workload()
    d = si.gyre_draws(wl)
    prob = g.Problem.from_gyre_workload(wl, d)
    prob.set_background(torch.zeros(wl.n, dtype=torch.float64, device="cuda"))
    prob.fwd(torch.zeros(wl.n, dtype=torch.float64, device="cuda"))
    X = torch.tensor(si.gaussian_matrix(wl.seed, wl.k, wl.n, stream=29), device="cuda", dtype=torch.float32)
    W = prob.tlm_block(X, prec=g.FP32)
    prob.adj_block(W, prec=g.FP32)
    torch.cuda.synchronize()
    print("gyre profile case done")


def main():
    args = parse()
    if args.profile_sketch:
        profile_case_sketch()
        return
    if args.profile:
        if args.workload == "bve_gyre":
            profile_case_gyre()
        elif args.workload in ("bve_n256", "bve_n1024"):
            profile_case_bve(args.workload)
        else:
            profile_case()
        return
    if args.impl == "reference":
        reference_arm(args)
    elif args.workload in ("bve_n256", "bve_n1024"):
        bve_arm(args)
    elif args.workload == "burgers_batch64":
        batch_arm(args)
    elif args.workload == "burgers_paper":
        paper_arm(args)
    elif args.workload == "bve_gyre":
        gyre_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
