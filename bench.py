#!/usr/bin/env python
"""Throughput benchmark of the GB300 dG-VFP library.

Headline (one step = one Crank--Nicolson step of the parallel shock): reduced phase space (x, ln p),
x in [-200, 200] with 256 cells, ln p in [0, 10] with 64 cells, dG degree 1, l_max = 3 (n = 16), tanh
shock U1 = 0.1, r = 4, nu = p, B = e_x, Gaussian source, FP64, dt = 1, restarted GMRES(30) to a true
relative residual of 1e-10.  N = 1,048,576 DoFs.  `value` = whole-job DoF-updates/s per CN step.

The same JSON line carries, under "workloads", the other configurations timed in the same run, each
with its own value, roofline of its dominant kernel, clocks and end-to-end leg:
  shock_fp32     the same CN steps in the precision form (FP32 apply, FP64 residual/refinement);
  box3d_fp64/32  the 48^3 periodic box (k = 2, l_max = 5, N = 107,495,424), DoF-updates/s per RK4
                 stage (FP64 plain; FP32 stage derivatives with FP64 state);
  batched_fp32   512 seeded shock instances (l_max in {1,3,5,7}, 64..512 x-cells), one CN step of
                 the whole batch per step (FP32 apply + FP64 GMRES), beside the same instances run one
                 at a time on the FP64 plain path;
  adjoint_fp64   forward + reverse (discrete adjoint with field gradients) of CN steps of the shock
                 with a per-cell log-normal nu, checkpoints every 50 steps; seconds per step.
Timing: W untimed warm-up steps, then K steps bracketed by CUDA events on the library's stream; the
shock state (8 MB) is L2-resident, so a 256 MiB buffer is written between timed steps (outside the
events); the box and batch states are larger than L2.  `--impl reference` times the FP64 CPU oracle
(its multi-threaded C driver of the assembled CN step, all host cores) on the headline workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "phase-space DoF-updates/s per CN step"
UNIT = "DoF-updates/s"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e-3  # SMs x DFMA/clk/SM x 2 flop x max GHz = 1.2586 TFLOP/s (FP64)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e-3  # SMs x FFMA/clk/SM x 2 flop x max GHz = 80.5 TFLOP/s (FP32)
HBM_FALLBACK_GBS = 6800.0
# DRAM bytes (read + write) per launch of the dominant kernel from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum of one apply launch), valid only for the sources it was
# taken on: keyed by (workload, precision, apply_sha of the kernel source and the epilogue header at
# capture); see profiles/.  The shock at full size; the 48^3 box from a 32^3
# capture scaled by the cell ratio 3.375 (traffic grows with the cells; the rule on capture sizes keeps
# the 48^3 case out of ncu)
APPLY_TRAFFIC = {("shock", "fp64", "7fc8fc6b12e2d515"): 26139392.0,
                 ("shock", "fp32", "7fc8fc6b12e2d515"): 13666560.0,
                 ("box3d", "fp32", "780e84dad4872f24"): 225314560.0 * 3.375,
                 ("box3d", "fp64", "780e84dad4872f24"): 492046848.0 * 3.375}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--workload", default="all", choices=["all", "shock", "box3d", "batched", "adjoint", "dsa"])
    ap.add_argument("--dsa-steps", type=int, default=500000, help="dsa: CN steps (dt = 1) of the run")
    ap.add_argument("--dsa-budget-s", type=float, default=900.0,
                    help="dsa: stop after the first 1000-step chunk that ends past this wall time")
    ap.add_argument("--cells", type=int, default=48, help="box3d: cells per axis")
    ap.add_argument("--instances", type=int, default=512, help="batched: number of shock instances")
    ap.add_argument("--batched-steps", type=int, default=3, help="batched: timed CN steps (each ~seconds)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--compare-single", type=int, default=16,
                    help="batched: also run this many of the instances one at a time on the FP64 path")
    ap.add_argument("--apply-reps", type=int, default=50)
    return ap.parse_args()


# ------------------------------------------------------------------------------------------------
# peaks
# ------------------------------------------------------------------------------------------------
def hbm_peak():
    """(GB/s, provenance) from MEASURED_PEAKS.json, else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "of measured"
    except Exception:
        return HBM_FALLBACK_GBS, "of fallback"


ALU_PROBE = {}  # measured FMA roofs of this run (sap_probe_fma), TFLOP/s per precision


def roofline_entry(kernel, flops, abytes, t_apply, precision, traffic=None, units=None):
    """ALU roofline of an operator apply (the operator is above the ridge point in both
    precisions), with the HBM view of its algorithmic bytes beside it.  `peak` is the nominal one
    from unit counts and the maximum clock; the FMA roof measured in this run is given beside it."""
    peak = FP64_PEAK_TFLOPS if precision == "fp64" else FP32_PEAK_TFLOPS
    achieved = flops / t_apply / 1e12
    hbm, how = hbm_peak()
    out = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
           "traffic": traffic, "kernel": kernel, "apply_us": t_apply * 1e6, "flops_per_apply": flops,
           "algorithmic_bytes_per_apply": abytes,
           "hbm_view": {"achieved_gbs": abytes / t_apply / 1e9, "peak_gbs": hbm, "frac": abytes / t_apply / 1e9 / hbm,
                        "peak_note": how},
           "peak_note": "nominal from unit counts x max clock (FP64: 2 DFMA/clk/SM; FP32: 128 FFMA/clk/SM); "
                        "flops from the kernel's cost model (sap_apply_cost)"}
    if units:
        out["units_per_launch"] = units
    if precision in ALU_PROBE:
        out["measured_fma_roof_tflops"] = ALU_PROBE[precision]
        out["frac_of_measured_fma_roof"] = achieved / ALU_PROBE[precision]
    return out


def probe_alu(local):
    """FMA roofs of the device in both precisions (library probe), with the clocks seen."""
    from paper_2501_05110_gb300 import sapgpu
    clocks = ClockSampler(local, "_alu_probe")
    clocks.start()
    res = {}
    for prec in ("fp64", "fp32"):
        best = 0.0
        for _ in range(3):
            best = max(best, sapgpu.probe_fma(prec) / 1e12)
        res[prec] = best
        ALU_PROBE[prec] = best
    res["clocks"] = clocks.stop()
    res["unit"] = "TFLOP/s"
    res["how"] = "sap_probe_fma: 8 independent FMA chains per thread, 16 blocks of 256 threads per SM, best of 3"
    return res


def apply_sha(source="apply_rows.cu"):
    """First 16 hex digits of the sha256 of the kernel source an ncu traffic figure was taken from,
    followed by the shared epilogue header it includes."""
    import hashlib
    h = hashlib.sha256()
    for name in (source, "kernels_common.cuh"):
        with open(os.path.join(ROOT, "paper_2501_05110_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# ------------------------------------------------------------------------------------------------
# clocks
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, tag: str = ""):
        self.gpu = gpu_index
        self.proc = None
        logdir = os.environ.get("SAP_BENCH_LOGDIR", os.path.join(ROOT, "bench_logs"))
        self.path = os.path.join(logdir, f"clocks{tag}_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # the timed region starts only once the sampler is writing (bounded wait)
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 5.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
# rank aggregation (replicas / instance shards: no collective on the data path, only the timing)
# ------------------------------------------------------------------------------------------------
def max_over_ranks(t: float, world: int, device: str = "cuda") -> float:
    """The job's time: the largest of the ranks' timed regions (all_reduce MAX when world > 1)."""
    if world <= 1:
        return t
    import torch
    import torch.distributed as dist
    tt = torch.tensor([t], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def sum_over_ranks(v: float, world: int, device: str = "cuda") -> float:
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist
    tt = torch.tensor([v], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.SUM)
    return float(tt.item())


def job_value(n_per_rank: int, steps: int, world: int, t_max: float) -> float:
    """Whole-job throughput: the DoF-updates of all ranks divided by the slowest rank's time."""
    return n_per_rank * steps * world / t_max


# ------------------------------------------------------------------------------------------------
# CPU oracle (multi-threaded C driver of the assembled CN step; assembly untimed)
# ------------------------------------------------------------------------------------------------
def shock_config(prob):
    """The headline workload's config (identical in both arms)."""
    return {"workload": "shock_x256_lnp64_k1_l3_cn_dt1_tol1e-10", "dofs": prob.ndofs, "cells": prob.ncells,
            "degree": prob.k, "lmax": prob.lmax, "gmres_restart": prob.gmres_restart, "gmres_tol": prob.gmres_tol,
            "dt": prob.dt, "l2": "flushed between timed steps (256 MiB write)", "parallelism": "replicas"}


def run_cpu_oracle(nsteps: int, warmup: int = 1) -> dict:
    import numpy as np
    from oracle import dg, native
    from paper_2501_05110_gb300 import workloads as W
    prob = W.shock()
    d = dg.Discretisation(prob)
    drv = native.CNDriver(d, prob.dt)
    z = np.zeros(d.N)
    if warmup:
        drv.steps(z, warmup, tol=prob.gmres_tol, restart=prob.gmres_restart)
    t0 = time.perf_counter()
    threads, its = drv.steps(z, nsteps, tol=prob.gmres_tol, restart=prob.gmres_restart)
    t = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0))
    return {"value": d.N * nsteps / t, "unit": UNIT, "cores": threads, "host_cores": cores, "kind": "oracle",
            "ms_per_step": 1e3 * t / nsteps, "seconds": t,
            "sample": f"{nsteps} timed CN steps (after {warmup} warm-up) of the full workload (N={d.N}) by the "
                      f"oracle's C driver: assembled CSR A = M + dt/2 D, GMRES(30) with right point-Jacobi, "
                      f"tol 1e-10, OpenMP on {threads} threads; assembly untimed; "
                      f"{its / nsteps:.1f} GMRES iterations/step"}


def run_cpu_oracle_rk4(nsteps: int = 40, warmup: int = 1, cells: int = 4) -> dict:
    """The oracle's RK4 step on a small box with the 3-D workload's k, l_max and fields (the full
    48^3 box cannot be assembled by the oracle): C driver, all host cores; DoF-updates/s per stage."""
    import numpy as np
    from oracle import dg, native
    from paper_2501_05110_gb300 import workloads as W
    prob = W.box3d(ncells=cells)
    d = dg.Discretisation(prob)
    drv = native.RK4Driver(d)
    z = np.random.default_rng(0).standard_normal(d.N)
    if warmup:
        drv.steps(z, prob.dt, warmup)
    t0 = time.perf_counter()
    threads = drv.steps(z, prob.dt, nsteps)
    t = time.perf_counter() - t0
    return {"value": d.N * 4 * nsteps / t, "unit": UNIT, "cores": threads,
            "host_cores": len(os.sched_getaffinity(0)), "kind": "oracle", "ms_per_step": 1e3 * t / nsteps,
            "seconds": t,
            "sample": f"{nsteps} timed RK4 steps (after {warmup} warm-up) of a {cells}^3 box with the workload's "
                      f"k = 2, l_max = 5 and fields (N = {d.N}) by the oracle's C driver: assembled CSR D "
                      f"({d.D.nnz} nonzeros) and inverted mass blocks, OpenMP on {threads} threads; assembly "
                      f"untimed; DoF-updates per RK4 stage"}


# ------------------------------------------------------------------------------------------------
# GPU measurements
# ------------------------------------------------------------------------------------------------
def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def time_apply(torch, sol, x, reps):
    """Average duration (s) of one operator apply launched alone on the current stream."""
    y = torch.empty_like(x)
    for _ in range(3):
        sol.apply(x, y)
    e0, e1 = _events(torch)
    e0.record()
    for _ in range(reps):
        sol.apply(x, y)
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) * 1e-3 / reps


def measure_shock(args, precision, world, rank, local, with_e2e=True):
    import torch
    from paper_2501_05110_gb300 import sapgpu
    from paper_2501_05110_gb300 import workloads as W
    prob = W.shock()
    sol = sapgpu.Solver(prob, precision)
    N = sol.N
    state = sol.initial_state()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    tol, restart, maxit = prob.gmres_tol, prob.gmres_restart, 5000
    for _ in range(args.warmup):
        sol.step_cn(state, prob.dt, 1, tol, restart, maxit)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    start = state.clone()  # the end-to-end leg replays the same steps from this state
    clocks = ClockSampler(local, f"_shock_{precision}")
    clocks.start()
    barrier()
    t_steps, its, launches = [], [], 0
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = _events(torch)
        e0.record()
        st = sol.step_cn(state, prob.dt, 1, tol, restart, maxit)
        e1.record()
        e1.synchronize()
        t_steps.append(e0.elapsed_time(e1) * 1e-3)
        its.append(st.iterations)
        launches += st.kernel_launches
    barrier()
    clk = clocks.stop()
    t_total = max_over_ranks(sum(t_steps), world)
    out = {"value": job_value(N, args.steps, world, t_total), "unit": UNIT,
           "ms_per_step": 1e3 * t_total / args.steps, "steps": args.steps, "warmup": args.warmup,
           "gmres_iterations_per_step": statistics.mean(its), "gpu_launches": int(launches), "clocks": clk,
           "dofs": N}
    if with_e2e:
        host = torch.empty(N, dtype=torch.float64, pin_memory=True)
        host.copy_(start.cpu())
        dev = torch.empty_like(state)
        barrier()
        t_e2e, its_e2e = 0.0, []
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = _events(torch)
            e0.record()
            dev.copy_(host, non_blocking=True)
            its_e2e.append(sol.step_cn(dev, prob.dt, 1, tol, restart, maxit).iterations)
            host.copy_(dev, non_blocking=True)
            e1.record()
            e1.synchronize()
            t_e2e += e0.elapsed_time(e1) * 1e-3
        barrier()
        t_e2e = max_over_ranks(t_e2e, world)
        out["e2e"] = {"value": job_value(N, args.steps, world, t_e2e), "unit": UNIT, "h2d_bytes_per_step": N * 8,
                      "d2h_bytes_per_step": N * 8, "gmres_iterations_per_step": statistics.mean(its_e2e),
                      "trajectory": "the device-timed steps replayed from the same starting state"}
    flops, abytes = sol.apply_cost()
    x = state.clone() if precision == "fp64" else state.float()
    t_apply = time_apply(torch, sol, x, args.apply_reps * 4)
    traffic = APPLY_TRAFFIC.get(("shock", precision, apply_sha("apply_rows.cu")))
    out["roofline"] = roofline_entry(f"rows_kernel<{'double' if precision == 'fp64' else 'float'},2,2>", flops,
                                     abytes, t_apply, precision, traffic, units=f"{N} DoFs (one apply)")
    sol.close()
    return out


def measure_box3d(args, precision):
    """RK4 on the 48^3 periodic box: DoF-updates/s per RK4 stage (4 per step); the state (0.86 GB
    FP64) is larger than L2."""
    import torch
    from paper_2501_05110_gb300 import sapgpu
    from paper_2501_05110_gb300 import workloads as W
    prob = W.box3d(ncells=args.cells)
    sol = sapgpu.Solver(prob, precision)
    N = sol.N
    y = sol.initial_state()
    start = y.clone()
    for _ in range(args.warmup):
        sol.step_erk(y, prob.dt, 1)
    clocks = ClockSampler(0, f"_box3d_{precision}")
    clocks.start()
    torch.cuda.synchronize()
    e0, e1 = _events(torch)
    e0.record()
    sol.step_erk(y, prob.dt, args.steps)
    e1.record()
    e1.synchronize()
    clk = clocks.stop()
    t = e0.elapsed_time(e1) * 1e-3
    # end to end: the state comes from and returns to pinned host memory every step
    host = torch.empty(N, dtype=torch.float64, pin_memory=True)
    host.copy_(start.cpu())
    dev = torch.empty_like(y)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        dev.copy_(host, non_blocking=True)
        sol.step_erk(dev, prob.dt, 1)
        host.copy_(dev, non_blocking=True)
    e1.record()
    e1.synchronize()
    t_e2e = e0.elapsed_time(e1) * 1e-3
    flops, abytes = sol.apply_cost()
    x = (y if precision == "fp64" else y.float()).clone()
    del host, dev
    t_apply = time_apply(torch, sol, x, max(5, args.apply_reps // 5))
    tname = "double" if precision == "fp64" else "float"
    node = sol.apply_kernel_in_use() == "node"
    kernel = f"uniform_kernel<{tname},5>" if node else f"rows_kernel<{tname},3,3>"
    # the row kernel on the same state, for comparison
    sol.set_apply_kernel("rows")
    t_rows = time_apply(torch, sol, x, max(5, args.apply_reps // 5))
    sol.set_apply_kernel("auto")
    stage_bytes = N * 5 * 8 if precision == "fp64" else N * (2 * 4 + 3 * 8)
    traffic = APPLY_TRAFFIC.get(("box3d", precision, apply_sha("uniform.cu" if node else "apply_rows.cu")))
    out = {"metric": "phase-space DoF-updates/s per ERK stage", "value": N * 4 * args.steps / t, "unit": UNIT,
           "ms_per_step": 1e3 * t / args.steps, "steps": args.steps, "warmup": args.warmup,
           "dtype": "f64" if precision == "fp64" else "f32 stage derivatives, f64 state",
           "config": {"workload": f"box3d_{args.cells}c_k2_l5_erk4_dt0.01", "dofs": N, "l2": "state larger than L2"},
           "stage_algorithmic_bytes_per_dof": stage_bytes / N,
           "stage_gbs": stage_bytes * 4 * args.steps / t / 1e9,
           "e2e": {"value": N * 4 * args.steps / t_e2e, "unit": UNIT, "h2d_bytes_per_step": N * 8,
                   "d2h_bytes_per_step": N * 8},
           "roofline": roofline_entry(kernel, flops, abytes, t_apply, precision, traffic,
                                      units=f"{N} DoFs (one apply)"),
           "row_kernel_apply_us": 1e6 * t_rows,
           "clocks": clk, "gpu_launches": 4 * args.steps + (args.steps if precision == "fp32" else 0)}
    sol.close()
    if precision == "fp64" and not args.no_cpu_baseline:
        try:
            out["cpu_baseline"] = run_cpu_oracle_rk4()
        except Exception as exc:  # reported, never fatal for the GPU measurement
            out["cpu_baseline"] = {"value": None, "error": f"{type(exc).__name__}: {str(exc)[:200]}"}
    return out


def measure_batched(args, world=1, rank=0, local=0):
    """CN steps on a batch of independent seeded shock instances (r, nu0, l_max, x-cell count drawn
    per instance), FP32 apply + FP64 GMRES.  With several ranks the instances are sharded across them
    (instance i on rank i mod world): no exchange, only the timing reduction."""
    import torch
    from paper_2501_05110_gb300 import sapgpu, sharding
    from paper_2501_05110_gb300 import workloads as W
    probs_all = W.batched_shocks(count=args.instances)
    mine = sharding.shard_instances(len(probs_all), rank, world)
    probs = [probs_all[i] for i in mine]
    t0 = time.perf_counter()
    batch = sapgpu.Batch(probs, "fp32")
    t_setup = time.perf_counter() - t0
    N = batch.N
    y = batch.initial_state()
    start = y.clone()
    for _ in range(1):
        batch.step_cn(y, 1.0, 1, 1e-10, 30, 20000)
    clocks = ClockSampler(local, "_batched")
    clocks.start()
    torch.cuda.synchronize()
    times, its, launches = [], [], 0
    for _ in range(args.batched_steps):
        e0, e1 = _events(torch)
        e0.record()
        st = batch.step_cn(y, 1.0, 1, 1e-10, 30, 20000)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1) * 1e-3)
        its.append(st.max_iterations)
        launches += st.kernel_launches
    clk = clocks.stop()
    t = max_over_ranks(sum(times), world)
    n_all = int(sum_over_ranks(N, world))
    # end to end: the whole batch state from / to pinned host memory each step
    host = torch.empty(N, dtype=torch.float64, pin_memory=True)
    host.copy_(start.cpu())
    dev = torch.empty_like(y)
    torch.cuda.synchronize()
    e0, e1 = _events(torch)
    e0.record()
    for _ in range(args.batched_steps):
        dev.copy_(host, non_blocking=True)
        batch.step_cn(dev, 1.0, 1, 1e-10, 30, 20000)
        host.copy_(dev, non_blocking=True)
    e1.record()
    e1.synchronize()
    t_e2e = max_over_ranks(e0.elapsed_time(e1) * 1e-3, world)
    del host, dev
    x = y.float()
    t_apply = time_apply(torch, batch, x, 3)
    flops, abytes = batch.apply_cost()
    batch.close()
    single = None
    if args.compare_single > 0 and rank == 0:
        # the same kind of instances one at a time on the plain FP64 path (equal tolerance)
        idx = list(range(0, len(probs), max(1, len(probs) // args.compare_single)))[:args.compare_single]
        dofs, t_single, its_single = 0, 0.0, []
        for i in idx:
            sol = sapgpu.Solver(probs[i], "fp64")
            ys = sol.initial_state()
            sol.step_cn(ys, 1.0, 1, 1e-10, 30, 20000)
            torch.cuda.synchronize()
            for _ in range(args.batched_steps):
                e0, e1 = _events(torch)
                e0.record()
                st = sol.step_cn(ys, 1.0, 1, 1e-10, 30, 20000)
                e1.record()
                e1.synchronize()
                t_single += e0.elapsed_time(e1) * 1e-3
                its_single.append(st.iterations)
            dofs += sol.N
            sol.close()
        single = {"path": "one instance at a time, FP64 plain, tol 1e-10", "instances": len(idx), "dofs": dofs,
                  "value": dofs * args.batched_steps / t_single, "unit": UNIT,
                  "gmres_iterations_per_step": statistics.mean(its_single)}
    return {"metric": "phase-space DoF-updates/s per CN step (batched)", "value": n_all * args.batched_steps / t,
            "unit": UNIT, "ms_per_step": 1e3 * t / args.batched_steps, "steps": args.batched_steps, "warmup": 1,
            "dtype": "f32 apply + f64 residual/refinement",
            "config": {"workload": f"batched_shocks_{args.instances}_seed4", "dofs": n_all,
                       "instances": args.instances, "instances_per_rank": len(probs), "setup_s": t_setup,
                       "l2": "state larger than L2",
                       "lmax_counts": {str(l): sum(p.lmax == l for p in probs_all) for l in (1, 3, 5, 7)}},
            "max_gmres_iterations_per_step": statistics.mean(its),
            "e2e": {"value": n_all * args.batched_steps / t_e2e, "unit": UNIT, "h2d_bytes_per_step": N * 8,
                    "d2h_bytes_per_step": N * 8},
            "roofline": roofline_entry("rows_kernel_batched<float,2,2>", flops, abytes, t_apply, "fp32",
                                       APPLY_TRAFFIC.get(("batched", "fp32", apply_sha())),
                                       units=f"{N} DoFs (one batched apply)"),
            "clocks": clk, "gpu_launches": int(launches), "single_instances": single}


def measure_adjoint(args):
    """Forward + reverse (discrete adjoint with field gradients) of CN steps on the full shock with a
    per-cell log-normal nu field, checkpoints every 50 steps; wall time per forward+reverse step."""
    import numpy as np
    import torch
    from paper_2501_05110_gb300 import adjoint, sapgpu
    from paper_2501_05110_gb300 import workloads as W
    base = W.shock()
    xe, pe = base.edges
    nu_fun, _ = W.lognormal_cell_nu(xe, pe, seed=6)
    probe = sapgpu.Solver(W.shock(nu_field=nu_fun))
    pts = probe.points(sapgpu.PTS_PHASE)
    nu_nodes = nu_fun(pts[:, :1], np.exp(pts[:, 1]))
    probe.close()

    def make(nu_np, U1):
        vals = np.ascontiguousarray(nu_np if nu_np is not None else nu_nodes, dtype=np.float64)
        return W.shock(U1=U1, nu_field=lambda xs, p, _v=vals: _v)

    xc = 0.5 * (xe[1:] + xe[:-1])
    sel = torch.from_numpy(np.abs(xc) < 20.0).cuda()
    target = torch.from_numpy(np.random.default_rng(5).normal(0.0, 1e-3, 64)).cuda()

    def run(nsteps):
        fam = adjoint.CNProblemFamily(make_problem=make, nsteps=nsteps, dt=1.0, tol=1e-10, checkpoint=50)
        nu_t = torch.tensor(nu_nodes, dtype=torch.float64, device="cuda", requires_grad=True)
        u1_t = torch.tensor(0.1, dtype=torch.float64, requires_grad=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        zN = adjoint.CNTrajectory.apply(nu_t, u1_t, fam)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        S = zN.view(64, 256, 16, 4)[:, :, 0, :].mean(dim=2)[:, sel].mean(dim=1)
        L = ((S - target) ** 2).sum()
        L.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        return t0, t1, t2, fam, nu_t, u1_t

    run(2)  # first use of the torch kernels of the loss and its backward
    t0, t1, t2, fam, nu_t, u1_t = run(args.steps)
    return {"metric": "forward + reverse wall time per CN step (adjoint, FP64)", "value": (t2 - t0) / args.steps,
            "unit": "s/step", "higher_is_better": False, "steps": args.steps, "warmup": 1,
            "forward_s": t1 - t0, "reverse_s": t2 - t1, "dtype": "f64",
            "config": {"workload": "adjoint_shock_x256_lnp64_k1_l3_cn_lognormal_nu", "checkpoint": 50,
                       "dofs": base.ndofs, "gmres_tol": 1e-10},
            "grad_norm_nu": float(nu_t.grad.norm()), "grad_U1": float(u1_t.grad),
            "reverse_parts": dict(fam.last_backward)}


def measure_dsa(args):
    """The paper's diffusive-shock-acceleration run (Sec. 4.4): l_max = 1 parallel shock on the graded
    mesh, CN with dt = 1 from an empty domain; reports the spectrum at the shock (slope, normalisation
    N_num) at the end and the time dependence phi(t) at p = 59.9 against the paper's formula."""
    import numpy as np
    import torch
    from paper_2501_05110_gb300 import sapgpu
    from paper_2501_05110_gb300 import workloads as W
    prob = W.dsa_shock(nsteps=args.dsa_steps)
    sol = sapgpu.Solver(prob, args.precision)
    xe, pe = prob.edges
    nx, npc = len(xe) - 1, len(pe) - 1
    i0 = int(np.searchsorted(xe, 0.0)) - 1  # the x-cells on both sides of x = 0
    lpc = 0.5 * (pe[1:] + pe[:-1])
    j1 = int(np.searchsorted(pe, math.log(59.9)) - 1)
    y = sol.initial_state()
    p0, U1, r = 2.0, 1.0 / 60.0, 4.0
    N = 0.1 / (p0 * U1) * 3 * r / (r - 1)  # 12

    def spectrum(v):
        f = v.view(npc, nx, prob.n, 4)[:, i0:i0 + 2, 0, :].mean(dim=(1, 2)) / math.sqrt(4 * math.pi)
        return f.cpu().numpy()

    chunk = 1000
    done, series, its = 0, [], 0
    clocks = ClockSampler(0, "_dsa")
    clocks.start()
    t0 = time.perf_counter()
    while done < args.dsa_steps and time.perf_counter() - t0 < args.dsa_budget_s:
        nst = min(chunk, args.dsa_steps - done)
        st = sol.step_cn(y, prob.dt, nst, 1e-10, 30, 5000)
        its += st.iterations
        done += nst
        F = spectrum(y)
        series.append((done, float(F[j1] / (N * (math.exp(lpc[j1]) / p0) ** -4))))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    F = spectrum(y)
    sel = (lpc > math.log(4.0)) & (lpc < math.log(40.0))
    slope, icpt = np.polyfit(lpc[sel], np.log(F[sel]), 1)
    Nnum = float(np.mean(F[sel] * (np.exp(lpc[sel]) / p0) ** 4))
    phi = [{"t": t, "numerical": v, "paper_formula": W.dsa_phi(t)} for (t, v) in series
           if t in (10000, 20000, 50000, 80000, 100000, 150000, 200000, 300000, 400000, 500000) or t == done]
    spec = [{"p": float(math.exp(lpc[j])), "F": float(F[j])} for j in range(0, npc, 8)]
    return {"metric": "diffusive shock acceleration run (Sec. 4.4)", "steps": done, "dt": prob.dt,
            "dofs": prob.ndofs, "cells": prob.ncells, "precision": args.precision,
            "wall_s": wall, "ms_per_step": 1e3 * wall / done, "gmres_iterations_per_step": its / done,
            "slope": float(slope), "slope_error": float(abs(slope + 4.0)), "paper_slope_error": 1.5e-3,
            "fit": "ln p in (ln 4, ln 40), f_000 / sqrt(4 pi) averaged over the two x-cells at the shock",
            "N_num": Nnum, "paper_N_num": 12.14, "N_analytic": N,
            "N_analytic_gaussian_source": N * math.exp(8 * (0.125 / p0) ** 2),
            "phi_p59.9": phi, "spectrum_at_shock": spec, "clocks": clk}


def run_mine(args):
    import torch
    import torch.distributed as dist
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2501_05110_gb300 import build as sap_build
    sap_build.build()
    alu = probe_alu(local)
    head = measure_shock(args, args.precision, world, rank, local)
    from paper_2501_05110_gb300 import workloads as W
    prob = W.shock()
    out = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if args.precision == "fp64" else "f32 apply + f64 residual/refinement",
           "data": "synthetic", "config": shock_config(prob), "precision": args.precision,
           "gmres_iterations_per_step": head["gmres_iterations_per_step"],
           "roofline": head["roofline"], "e2e": head["e2e"], "clocks": head["clocks"],
           "gpu_launches": head["gpu_launches"], "alu_probe": alu}
    workloads = {}
    if args.workload == "all":
        plan = [("shock_fp32", lambda: measure_shock(args, "fp32", world, rank, local)),
                ("batched_fp32", lambda: measure_batched(args, world, rank, local))]
        if world == 1:
            plan[1:1] = [("box3d_fp64", lambda: measure_box3d(args, "fp64")),
                         ("box3d_fp32", lambda: measure_box3d(args, "fp32"))]
            plan.append(("adjoint_fp64", lambda: measure_adjoint(args)))
        for name, fn in plan:
            try:
                workloads[name] = fn()
            except Exception as exc:  # reported in the line, not hidden
                workloads[name] = {"error": f"{type(exc).__name__}: {str(exc)[:300]}"}
            torch.cuda.empty_cache()
        out["workloads"] = workloads
        out["gpu_launches"] += sum(int(w.get("gpu_launches", 0)) for w in workloads.values())
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            out["cpu_baseline"] = run_cpu_oracle(min(args.steps, 10))
        except Exception as exc:  # reported, not hidden
            out["cpu_baseline"] = {"value": None, "error": str(exc)[:300]}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def run_single_workload(args):
    """--workload box3d | batched | adjoint | shock: one configuration on its own line."""
    import torch
    torch.cuda.set_device(0)
    from paper_2501_05110_gb300 import build as sap_build
    sap_build.build()
    probe_alu(0)
    if args.workload == "box3d":
        res = measure_box3d(args, args.precision)
    elif args.workload == "batched":
        res = measure_batched(args)
    elif args.workload == "adjoint":
        res = measure_adjoint(args)
    elif args.workload == "dsa":
        res = measure_dsa(args)
    else:
        res = measure_shock(args, args.precision, 1, 0, 0)
    res.setdefault("n_gpus", 1)
    print(json.dumps(res))


def run_reference(args):
    """The reference arm: the FP64 CPU oracle (its multi-threaded C driver, all host cores) on the
    headline workload; each timed step is one full CN step of the 1,048,576-DoF shock."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2501_05110_gb300 import workloads as W
    timed = min(args.steps, 30)
    res = run_cpu_oracle(timed, warmup=min(args.warmup, 1))
    if timed < args.steps:
        res["sample"] += f" (first {timed} of the {args.steps} requested steps)"
    prob = W.shock()
    line = {"impl": "reference", "metric": METRIC, "value": res["value"], "unit": UNIT,
            "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": shock_config(prob),
            "cpu_baseline": {"value": res["value"], "unit": UNIT, "kind": "oracle", "cores": res["cores"],
                             "sample": res["sample"]},
            "e2e": {"value": res["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "all":
        run_mine(args)
    else:
        run_single_workload(args)


if __name__ == "__main__":
    main()
