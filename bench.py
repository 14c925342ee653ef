#!/usr/bin/env python
"""Throughput benchmark of the GB300 dG-VFP library on the parallel-shock Crank--Nicolson workload.

Workload (default, "shock"): reduced phase space (x, ln p), x in [-200, 200] with 256 cells,
ln p in [0, 10] with 64 cells, dG degree 1, lmax = 3 (n = 16), tanh shock U1 = 0.1, r = 4,
nu = p, B = e_x, Gaussian source, FP64; one step = one Crank--Nicolson step (dt = 1) solved by
restarted GMRES(30) to a true relative residual of 1e-10.  N = 1,048,576 DoFs.

Prints ONE JSON line.  `value` is whole-job DoF-updates/s per CN step (N * steps / time, summed
over ranks; each rank runs an independent replica: the single-shock solve does not shard).
Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events on the stream the
library runs on, with a 256 MiB L2 flush between timed steps (outside the events).
`--impl reference` times the FP64 CPU oracle (the only baseline that exists: the paper publishes
no performance numbers) on the same workload and prints the same line with "impl": "reference".
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
# DRAM bytes (read + write) per apply launch from the ncu capture in profiles/rows_kernel_fp64_shock.md,
# valid only for the kernel source it was taken on (first 16 hex of sha256 of csrc/apply_rows.cu)
APPLY_TRAFFIC = {"29ab0aa921f8c3aa": 11002112.0}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--workload", default="shock", choices=["shock", "box3d", "batched", "adjoint"])
    ap.add_argument("--cells", type=int, default=48, help="box3d: cells per axis")
    ap.add_argument("--instances", type=int, default=512, help="batched: number of shock instances")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--compare-single", type=int, default=16,
                    help="batched: also run this many of the instances one at a time on the FP64 path")
    ap.add_argument("--cpu-worker", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--apply-reps", type=int, default=200)
    return ap.parse_args()


def workload_problem():
    from paper_2501_05110_gb300 import workloads as W
    return W.shock()


def workload_config(prob, extra=None):
    cfg = {"workload": "shock_x256_lnp64_k1_l3_cn_dt1_tol1e-10", "dofs": prob.ndofs,
           "cells": prob.ncells, "degree": prob.k, "lmax": prob.lmax, "gmres_restart": prob.gmres_restart,
           "gmres_tol": prob.gmres_tol, "dt": prob.dt, "l2": "flushed between timed steps (256 MiB write)",
           "parallelism": "replicas"}
    if extra:
        cfg.update(extra)
    return cfg


# ------------------------------------------------------------------------------------------------
# CPU oracle timing (runs in a fresh single-threaded interpreter)
# ------------------------------------------------------------------------------------------------
def cpu_worker(nsteps: int):
    """Time the oracle's CN step (assembled CSR, GMRES(30) with Jacobi, tol 1e-10) on the full
    workload; assembly is set-up and untimed."""
    import numpy as np
    from oracle import dg, steppers
    prob = workload_problem()
    d = dg.Discretisation(prob)
    A = (d.M + 0.5 * prob.dt * d.D).tocsr()
    B = (d.M - 0.5 * prob.dt * d.D).tocsr()
    z = np.zeros(d.N)
    times, its = [], []
    for _ in range(nsteps):
        t0 = time.perf_counter()
        b = B @ z + prob.dt * d.h
        z, it = steppers.gmres(A, b, z, tol=prob.gmres_tol, restart=prob.gmres_restart)
        times.append(time.perf_counter() - t0)
        its.append(it)
    print(json.dumps({"times": times, "its": its, "N": d.N}))


def run_cpu_oracle(nsteps: int, skip: int = 0) -> dict:
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    env.pop("CUDA_VISIBLE_DEVICES", None)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-worker", str(nsteps)],
                       capture_output=True, text=True, env=env, cwd=ROOT, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError("cpu worker failed: " + r.stderr[-2000:])
    out = json.loads(r.stdout.strip().splitlines()[-1])
    times = out["times"][skip:]
    t = sum(times)
    return {"value": out["N"] * len(times) / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "ms_per_step": 1e3 * t / len(times),
            "sample": f"{len(times)} timed CN steps of the full workload (N={out['N']}) with the oracle's "
                      f"assembled CSR + GMRES(30)/Jacobi, tol 1e-10, single thread; assembly untimed; "
                      f"{statistics.mean(out['its']):.1f} GMRES iterations/step",
            "seconds": t}


# ------------------------------------------------------------------------------------------------
# clocks
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        logdir = os.environ.get("SAP_BENCH_LOGDIR", os.path.join(ROOT, "bench_logs"))
        self.path = os.path.join(logdir, f"clocks_rank{gpu_index}.csv")

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
# rank aggregation (replicas: no collective on the data path, only the timing reduction)
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


def job_value(n_per_rank: int, steps: int, world: int, t_max: float) -> float:
    """Whole-job throughput: the DoF-updates of all ranks divided by the slowest rank's time."""
    return n_per_rank * steps * world / t_max


# ------------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------------
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
    from paper_2501_05110_gb300 import sapgpu
    sap_build.build()
    prob = workload_problem()
    sol = sapgpu.Solver(prob, args.precision)
    N = sol.N
    stream = torch.cuda.current_stream()
    state = sol.initial_state()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    tol, restart, maxit = prob.gmres_tol, prob.gmres_restart, 5000
    for _ in range(args.warmup):
        sol.step_cn(state, prob.dt, 1, tol, restart, maxit)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-timed steps --------------------------------------------------------------------
    start = state.clone()  # the end-to-end leg below replays the same steps from this state
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    t_steps, its, launches = [], [], 0
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = sol.step_cn(state, prob.dt, 1, tol, restart, maxit)
        e1.record(stream)
        e1.synchronize()
        t_steps.append(e0.elapsed_time(e1) * 1e-3)
        its.append(st.iterations)
        launches += st.kernel_launches
    barrier()
    clk = clocks.stop()
    t_total = max_over_ranks(sum(t_steps), world)
    value = job_value(N, args.steps, world, t_total)

    # ---- end to end through the public API with host buffers -------------------------------------
    host = torch.empty(N, dtype=torch.float64, pin_memory=True)
    host.copy_(start.cpu())
    dev = torch.empty_like(state)
    barrier()
    t_e2e, its_e2e = 0.0, []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dev.copy_(host, non_blocking=True)
        its_e2e.append(sol.step_cn(dev, prob.dt, 1, tol, restart, maxit).iterations)
        host.copy_(dev, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        t_e2e += e0.elapsed_time(e1) * 1e-3
    barrier()
    t_e2e = max_over_ranks(t_e2e, world)
    e2e = {"value": job_value(N, args.steps, world, t_e2e), "unit": UNIT, "h2d_bytes_per_step": N * 8,
           "d2h_bytes_per_step": N * 8, "gmres_iterations_per_step": statistics.mean(its_e2e),
           "trajectory": "the device-timed steps replayed from the same starting state"}

    # ---- dominant kernel: the operator apply, timed alone on the same stream ----------------------
    flops, abytes = sol.apply_cost()
    x = state.clone() if args.precision == "fp64" else state.float()
    y = torch.empty_like(x)
    for _ in range(10):
        sol.apply(x, y)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.apply_reps):
        sol.apply(x, y)
    e1.record(stream)
    e1.synchronize()
    t_apply = e0.elapsed_time(e1) * 1e-3 / args.apply_reps
    achieved = flops / t_apply / 1e12
    peak_alu = FP64_PEAK_TFLOPS if args.precision == "fp64" else FP32_PEAK_TFLOPS
    import hashlib
    src_sha = hashlib.sha256(open(os.path.join(ROOT, "paper_2501_05110_gb300", "csrc", "apply_rows.cu"), "rb").read()).hexdigest()[:16]
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_alu, "unit": "TFLOP/s",
                "frac": achieved / peak_alu,
                "traffic": APPLY_TRAFFIC.get(src_sha) if args.precision == "fp64" else None,
                "kernel": "rows_kernel<double,2,2>" if args.precision == "fp64" else "rows_kernel<float,2,2>",
                "apply_us": t_apply * 1e6, "flops_per_apply": flops, "algorithmic_bytes_per_apply": abytes,
                "hbm_view": {"achieved_gbs": abytes / t_apply / 1e9, "peak_gbs": 6746.3,
                             "frac": abytes / t_apply / 1e9 / 6746.3},
                "peak_note": "nominal from unit counts x max clock (FP64: 2 DFMA/clk/SM; FP32: 128 FFMA/clk/SM)"}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f64" if args.precision == "fp64" else "f32 apply + f64 residual/refinement",
           "data": "synthetic",
           "config": workload_config(prob, {"gmres_iterations_per_step": statistics.mean(its),
                                            "precision": args.precision}),
           "roofline": roofline, "e2e": e2e, "clocks": clk, "gpu_launches": int(launches)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            out["cpu_baseline"] = run_cpu_oracle(2)
        except Exception as exc:  # reported, not hidden
            out["cpu_baseline"] = {"value": None, "error": str(exc)[:300]}
    if rank == 0:
        print(json.dumps(out))
    sol.close()
    if world > 1:
        dist.destroy_process_group()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    res = run_cpu_oracle_steps(args.warmup, args.steps)
    prob = workload_problem()
    line = {"impl": "reference", "metric": METRIC, "value": res["value"], "unit": UNIT,
            "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": workload_config(prob),
            "cpu_baseline": {"value": res["value"], "unit": UNIT, "kind": "oracle", "cores": 1,
                             "sample": res["sample"]},
            "e2e": {"value": res["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


ORACLE_MAX_STEPS = 30  # about 40 s of single-thread oracle time: the reference arm stays within minutes


def run_cpu_oracle_steps(warmup: int, steps: int) -> dict:
    timed = min(steps, ORACLE_MAX_STEPS)
    res = run_cpu_oracle(min(warmup, 1) + timed, skip=min(warmup, 1))
    if timed < steps:
        res["sample"] += f" (first {timed} of the {steps} requested steps)"
    return res


def run_box3d(args):
    """RK4 on the 48^3 periodic box (k = 2, lmax = 5, N = 107,495,424): DoF-updates/s per RK4
    stage; the state (0.86 GB FP64) is larger than L2, so no flush is needed between steps."""
    import torch
    from paper_2501_05110_gb300 import build as sap_build
    from paper_2501_05110_gb300 import sapgpu
    from paper_2501_05110_gb300 import workloads as W
    sap_build.build()
    prob = W.box3d(ncells=args.cells)
    sol = sapgpu.Solver(prob, args.precision)
    N = sol.N
    stream = torch.cuda.current_stream()
    y = sol.initial_state()
    for _ in range(args.warmup):
        sol.step_erk(y, prob.dt, 1)
    clocks = ClockSampler(0)
    clocks.start()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sol.step_erk(y, prob.dt, args.steps)
    e1.record(stream)
    e1.synchronize()
    clk = clocks.stop()
    t = e0.elapsed_time(e1) * 1e-3
    flops, abytes = sol.apply_cost()
    x = (y if args.precision == "fp64" else y.float()).clone()
    out = torch.empty_like(x)
    for _ in range(3):
        sol.apply(x, out)
    e0.record(stream)
    for _ in range(args.apply_reps):
        sol.apply(x, out)
    e1.record(stream)
    e1.synchronize()
    t_apply = e0.elapsed_time(e1) * 1e-3 / args.apply_reps
    w = 8 if args.precision == "fp64" else 4
    stage_bytes = N * 5 * 8 if args.precision == "fp64" else N * (2 * 4 + 3 * 8)
    print(json.dumps({"metric": "phase-space DoF-updates/s per ERK stage", "value": N * 4 * args.steps / t,
                      "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
                      "dtype": "f64" if args.precision == "fp64" else "f32 apply, f64 state",
                      "data": "synthetic", "config": {"workload": f"box3d_{args.cells}c_k2_l5_erk4_dt0.01", "dofs": N,
                                                      "l2": "state larger than L2"},
                      "apply": {"us": t_apply * 1e6, "flops": flops, "tflops": flops / t_apply / 1e12,
                                "algorithmic_bytes": abytes, "gbs": abytes / t_apply / 1e9,
                                "hbm_frac": abytes / t_apply / 1e9 / 6746.3},
                      "stage_algorithmic_bytes_per_dof": stage_bytes / N,
                      "stage_gbs": stage_bytes * 4 * args.steps / t / 1e9, "clocks": clk}))


def run_batched(args):
    """CN steps on a batch of independent seeded shock instances (r, nu0, lmax, x-cell count drawn
    per instance), one batched apply launch per operator application, per-instance GMRES."""
    import torch
    from paper_2501_05110_gb300 import build as sap_build
    from paper_2501_05110_gb300 import sapgpu
    from paper_2501_05110_gb300 import workloads as W
    sap_build.build()
    probs = W.batched_shocks(count=args.instances)
    t0 = time.perf_counter()
    batch = sapgpu.Batch(probs, args.precision)
    t_setup = time.perf_counter() - t0
    N = batch.N
    y = batch.initial_state()
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        batch.step_cn(y, 1.0, 1, 1e-10, 30, 20000)
    clocks = ClockSampler(0)
    clocks.start()
    torch.cuda.synchronize()
    times, its, launches = [], [], 0
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = batch.step_cn(y, 1.0, 1, 1e-10, 30, 20000)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) * 1e-3)
        its.append(st.max_iterations)
        launches += st.kernel_launches
    clk = clocks.stop()
    x = (y if args.precision == "fp64" else y.float()).clone()
    out = torch.empty_like(x)
    for _ in range(2):
        batch.apply(x, out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(5):
        batch.apply(x, out)
    e1.record(stream)
    e1.synchronize()
    t_apply = e0.elapsed_time(e1) * 1e-3 / 5
    flops, abytes = batch.apply_cost()
    t = sum(times)
    batch.close()
    # the same instances run one at a time on the plain FP64 path (equal tolerance, same steps): every
    # (count/K)-th instance, each from its own initial state with the same warm-up
    single = None
    if args.compare_single > 0:
        idx = list(range(0, len(probs), max(1, len(probs) // args.compare_single)))[:args.compare_single]
        dofs, t_single, its_single = 0, 0.0, []
        for i in idx:
            sol = sapgpu.Solver(probs[i], "fp64")
            ys = sol.initial_state()
            for _ in range(args.warmup):
                sol.step_cn(ys, 1.0, 1, 1e-10, 30, 20000)
            torch.cuda.synchronize()
            for _ in range(args.steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                st = sol.step_cn(ys, 1.0, 1, 1e-10, 30, 20000)
                e1.record(stream)
                e1.synchronize()
                t_single += e0.elapsed_time(e1) * 1e-3
                its_single.append(st.iterations)
            dofs += sol.N
            sol.close()
        single = {"path": "one instance at a time, FP64 plain, tol 1e-10", "instances": len(idx),
                  "instance_index_step": max(1, len(probs) // args.compare_single), "dofs": dofs,
                  "value": dofs * args.steps / t_single, "unit": UNIT,
                  "gmres_iterations_per_step": statistics.mean(its_single)}
    print(json.dumps({"metric": "phase-space DoF-updates/s per CN step (batched)", "value": N * args.steps / t,
                      "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
                      "dtype": "f64" if args.precision == "fp64" else "f32 apply + f64 residual/refinement",
                      "data": "synthetic",
                      "config": {"workload": f"batched_shocks_{args.instances}_seed4", "dofs": N,
                                 "instances": args.instances, "setup_s": t_setup,
                                 "max_gmres_iterations_per_step": statistics.mean(its),
                                 "lmax_counts": {str(l): sum(p.lmax == l for p in probs) for l in (1, 3, 5, 7)}},
                      "apply": {"us": t_apply * 1e6, "gbs": abytes / t_apply / 1e9,
                                "hbm_frac": abytes / t_apply / 1e9 / 6746.3, "tflops": flops / t_apply / 1e12},
                      "gpu_launches": int(launches), "clocks": clk, "single_instances": single}))


def run_adjoint(args):
    """Forward + reverse (discrete adjoint) of CN steps on the full shock workload with a per-cell
    log-normal nu field, checkpoints every 50 steps; reports wall time per forward+reverse step."""
    import numpy as np
    import torch
    from paper_2501_05110_gb300 import adjoint, sapgpu
    from paper_2501_05110_gb300 import build as sap_build
    from paper_2501_05110_gb300 import workloads as W
    sap_build.build()
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
        """One forward + reverse pass over nsteps CN steps; returns timings (s) and the gradients."""
        fam = adjoint.CNProblemFamily(make_problem=make, nsteps=nsteps, dt=1.0, tol=1e-10, checkpoint=50)
        nu_t = torch.tensor(nu_nodes, dtype=torch.float64, device="cuda", requires_grad=True)
        u1_t = torch.tensor(0.1, dtype=torch.float64, requires_grad=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        zN = adjoint.CNTrajectory.apply(nu_t, u1_t, fam)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        # spectrum misfit near the shock: S_j = mean over the x-cells within 20 of the shock of the
        # cell-averaged f_000 at momentum cell j; L = sum_j (S_j - T_j)^2 with a seeded target
        S = zN.view(64, 256, 16, 4)[:, :, 0, :].mean(dim=2)[:, sel].mean(dim=1)
        L = ((S - target) ** 2).sum()
        L.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        return t0, t1, t2, fam, nu_t, u1_t

    # warm-up passes: the first use of each torch kernel of the loss (and of its backward) can cost
    # seconds on a fresh machine (module loading); they are not part of the method
    for _ in range(max(1, args.warmup)):
        run(2)
    nsteps = args.steps
    t0, t1, t2, fam, nu_t, u1_t = run(nsteps)
    print(json.dumps({"metric": "forward + reverse wall time per CN step (adjoint, FP64)",
                      "value": (t2 - t0) / nsteps, "unit": "s/step", "steps": nsteps, "warmup": max(1, args.warmup),
                      "forward_s": t1 - t0, "reverse_s": t2 - t1, "higher_is_better": False,
                      "dtype": "f64", "data": "synthetic",
                      "config": {"workload": "adjoint_shock_x256_lnp64_k1_l3_cn_lognormal_nu",
                                 "checkpoint": 50, "dofs": base.ndofs, "gmres_tol": 1e-10},
                      "grad_norm_nu": float(nu_t.grad.norm()), "grad_U1": float(u1_t.grad),
                      "reverse_parts": {k: v for k, v in fam.last_backward.items() if k != "entered_at"}}))


def main():
    args = parse()
    if args.workload == "box3d" and not args.cpu_worker:
        run_box3d(args)
        return
    if args.workload == "batched" and not args.cpu_worker:
        run_batched(args)
        return
    if args.workload == "adjoint" and not args.cpu_worker:
        run_adjoint(args)
        return
    if args.cpu_worker:
        cpu_worker(args.cpu_worker)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_mine(args)


if __name__ == "__main__":
    main()
