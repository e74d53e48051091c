#!/usr/bin/env python3
"""Benchmark: time to a relative true residual of 1e-10 for the staggered
variable-coefficient Stokes system on one GB300, through libstokes_gb300.

One step = set the coefficients (face densities, node/edge viscosities, the
FP64 and FP32 multigrid hierarchy) and solve M x = b from x = 0 to
||b - M x|| <= 1e-10 ||b|| with GMRES(10) and the workload's preconditioner.

Default workload: 3D unsteady Stokes on 128^3 periodic cells, rho contrast
1e2 and mu contrast 1e3 from seeded smooth log-normal fields, theta = 1
(viscous CFL number 1), forcing f ~ N(0,1) and mean-free g ~ N(0,1), P1.
Inputs are larger than L2 (8.4M unknowns: b and x alone are 134 MB, the FP64
Krylov basis 740 MB) and L2 is flushed by writing 256 MB between steps.

Forms: "fp64" (left-preconditioned GMRES, all FP64; the line's value) and
"mixed" (flexible GMRES in FP64 around an FP32 preconditioner; reported
beside it).  `--impl reference` times the FP64 CPU oracle instead.

Multi-GPU: replicas only (each rank solves its own copy; value = max over
ranks of the per-solve time).
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

METRIC = "Stokes time-to-1e-10 residual & GMRES iters; V-cycle/matvec HBM GB/s vs peak"
UNIT = "ms"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3",
                    choices=["c3", "c2", "c1", "c5", "bubble2d", "bubble3d", "c4", "c5adj", "study", "timeloop"])
    ap.add_argument("--n", type=int, default=0, help="override the grid size")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-others", action="store_true",
                    help="skip the other configurations measured after the headline")
    ap.add_argument("--quick", action="store_true",
                    help="profiling runs: only the timed solves of --form, no baseline/e2e/profile passes")
    ap.add_argument("--form", default="both", choices=["both", "fp64", "mixed"])
    ap.add_argument("--batched-forms", default="",
                    help="--workload c4: comma-separated forms to time (e.g. stacked_mixed; for "
                         "profilers), else every form")
    ap.add_argument("--no-graphs", action="store_true",
                    help="quick mode and the stacked forms of --workload c4: launch every kernel "
                         "from the host (for profilers)")
    ap.add_argument("--schedule", default="",
                    help="quick mode: coarse_level,threads,pair_level instead of the tuned schedule")
    ap.add_argument("--big", action="store_true",
                    help="study: add the 512^3 steady bubble to the size series (about 140 GB)")
    return ap.parse_args()


class Replicas:
    """`--gpus N` under torchrun: one process per GPU, each solving its own
    copy of the workload.  There is no collective on the data path; the
    process group only brackets the timed region with barriers and takes the
    maximum per-solve time over ranks."""

    def __init__(self, backend):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend, init_method="env://")

    def barrier(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()

    def max(self, values, device):
        """Element-wise maximum of a list of floats over all ranks."""
        if self.world == 1:
            return list(values)
        import torch
        import torch.distributed as dist
        t = torch.tensor(values, dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return t.tolist()

    def close(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


def make_problem(name, n):
    from paper_1308_4605_gb300 import workloads as wl
    if name == "c3":
        return wl.config_c3(n or 128), {"workload": f"3d_unsteady_periodic_{n or 128}^3",
                                         "rho_contrast": 1e2, "mu_contrast": 1e3, "precond": "P1"}
    if name == "c2":
        return wl.config_c2(n or 512), {"workload": f"2d_steady_noslip_20_inclusions_mu1e4_{n or 512}^2",
                                         "precond": "P2"}
    if name == "c1":
        return wl.config_c1(n or 32), {"workload": f"2d_unsteady_periodic_{n or 32}^2", "precond": "P1"}
    if name == "c5":
        return wl.config_c5(n or 64), {"workload": f"3d_steady_noslip_{n or 64}^3", "precond": "P2"}
    if name == "bubble2d":
        return wl.bubble(2, n or 512), {"workload": f"bubble_2d_r100_steady_{n or 512}^2", "precond": "P1"}
    return wl.bubble(3, n or 128), {"workload": f"bubble_3d_r100_steady_{n or 128}^3", "precond": "P1"}


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ roofline
FP64_PEAK_TFLOPS = 1.25   # nominal GB300 FP64 rate (an FMA probe measured 1.20 on this machine)
# FP64 instructions per FLOP of the level-0 velocity Gauss-Seidel point
# (16 instructions, 22 FLOP, from ncu's SASS op counters): the FP64 pipe
# issues one instruction (an FMA = 2 FLOP) per slot, so the kernel's share of
# the pipe's issue rate is achieved FLOP/s x 16/22 / (peak FLOP/s / 2).
FP64_INSTR_PER_FLOP = 16.0 / 22.0


TRAFFIC_WORKLOAD = "3d_unsteady_periodic_128^3"   # the workload the ncu summary covers


def traffic_per_launch(family, form, workload):
    """DRAM bytes per launch of `family` from the committed ncu summary, or
    None when the kernel sources changed since the counters were taken or
    the workload is not the one the counters were taken on."""
    import hashlib
    if workload != TRAFFIC_WORKLOAD:
        return None
    h = hashlib.sha256()
    for f in ("stencil.cuh", "kernels.cu", "pair.cu"):
        with open(os.path.join(ROOT, "paper_1308_4605_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    src = h.hexdigest()[:16]
    try:
        text = open(os.path.join(ROOT, "profiles", "kernels_3d_unsteady_periodic_128.md")).read()
    except OSError:
        return None
    for line in text.splitlines():
        parts = line.split()
        if len(parts) == 6 and parts[0] == "traffic:" and parts[1] == family and parts[2] == form:
            return float(parts[3]) if parts[5] == src else None
    return None


# kernel families that pool launches on grids of every size (the per-level
# smoothers below the finest level, the first sweeps from zero on every
# level, the coarse-level kernels): not one kernel configuration, so never
# "the dominant kernel" of a roofline
MULTI_LEVEL_FAMILIES = {"vel_smooth_colour", "cell_smooth_colour", "vel_smooth_pair",
                        "cell_smooth_pair", "vel_smooth_first", "cell_smooth_first", "coarse_levels"}


def roofline_of(fams, form, peaks, family=None, workload=TRAFFIC_WORKLOAD):
    """Roofline of the dominant kernel of a solve -- the family with the
    largest device time among those that are one kernel configuration
    (MULTI_LEVEL_FAMILIES pool many grid sizes and are left out) -- or of
    `family`.  FP64 Gauss-Seidel kernels are bound by the FP64 pipe (about 0.19
    FLOP per byte, at the GB300 balance of 1.25 TFLOP/s over 6.8 TB/s, with
    the pipe 80-89 % busy under ncu): reported as "alu" in TFLOP/s.  The rest
    is reported against HBM bandwidth."""
    if family is None:
        single = [f for f in fams if f["name"] not in MULTI_LEVEL_FAMILIES]
        dom = max(single or fams, key=lambda f: f["ms"])
    else:
        dom = next(f for f in fams if f["name"] == family)
    secs = dom["ms"] * 1e-3
    per_launch_us = dom["ms"] * 1e3 / dom["launches"]
    traffic = traffic_per_launch(dom["name"], form, workload) if dom["name"].endswith("_l0") else None
    hbm = peaks.get("hbm_gbs")
    if form == "fp64" and dom["flops"] > 0:
        achieved = dom["flops"] / secs / 1e12
        return {"bound": "alu", "kernel": dom["name"], "achieved": achieved,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "traffic": traffic, "peak_source": "nominal FP64 (recipe table); FMA probe 1.20",
                "fp64_issue_frac": achieved * FP64_INSTR_PER_FLOP / (FP64_PEAK_TFLOPS / 2.0),
                "avg_launch_us": per_launch_us, "flops_per_launch": dom["flops"] / dom["launches"],
                "bytes_per_launch": dom["bytes"] / dom["launches"],
                "hbm_gbps_alongside": dom["bytes"] / secs / 1e9}
    peak = hbm or 6800.0
    achieved = dom["bytes"] / secs / 1e9
    return {"bound": "hbm", "kernel": dom["name"], "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic,
            "peak_source": "measured" if hbm else "fallback",
            "avg_launch_us": per_launch_us, "bytes_per_launch": dom["bytes"] / dom["launches"]}


# --------------------------------------------------------------- oracle arm
def oracle_solve_time(pr):
    """Time the FP64 CPU oracle solving the workload `pr` as it stands:
    sparse assembly of M, the preconditioner's multigrid hierarchy (setup),
    then GMRES(10) from x = 0 to ||b - M x|| <= 1e-10 ||b|| with its own
    iteration count.  Nothing is extrapolated: the value is the wall time of
    that one solve.  scipy.sparse and numpy run single-threaded here.
    Returns (ms, description, threads used)."""
    from oracle import assemble as asm
    from oracle import krylov
    from oracle.grid import Grid
    from oracle.precond import Preconditioner
    g = Grid(pr.dim, pr.n, pr.h, pr.bc)
    t0 = time.perf_counter()
    M = asm.stokes_from_fields(g, pr.rho, pr.mu, pr.theta)
    P = Preconditioner(g, pr.rho, pr.mu, pr.theta, pr.precond)
    t_setup = time.perf_counter() - t0
    b = g.pack(pr.b_u, pr.b_p)
    b[~g.active] = 0.0
    t1 = time.perf_counter()
    _, info = krylov.gmres(lambda v: M @ v, P, b, rtol=1e-10, maxit=600)
    t_solve = time.perf_counter() - t1
    ms = (t_setup + t_solve) * 1e3
    desc = (f"oracle (scipy.sparse, FP64, one thread) on the full "
            f"{'x'.join(map(str, pr.n[:pr.dim]))} workload: setup {t_setup:.1f} s + "
            f"{info['iterations']} GMRES(10) iterations {t_solve:.1f} s to a true residual of "
            f"{info['true_residual'][-1]:.1e} (its own count, measured, not scaled); "
            f"host has {os.cpu_count()} cores")
    return ms, desc, 1


def reference_sample(pr):
    """The bounded sample a reference-arm step solves: the same generator at
    half the grid size per axis in 3D (64^3 for the 128^3 workload), the
    workload itself in 2D."""
    from paper_1308_4605_gb300 import workloads as wl
    if pr.dim == 2:
        return pr
    n = max(pr.n[0] // 2, 8)
    if pr.name.startswith("3d_unsteady_periodic"):
        return wl.config_c3(n)
    if pr.name.startswith("3d_steady_noslip"):
        return wl.config_c5(n)
    return wl.bubble(3, n)


def run_reference(args):
    """The FP64 CPU oracle as the reference arm: each step is one complete
    oracle solve (setup and GMRES to 1e-10 with its own iteration count) of a
    bounded sample of the workload, timed as it runs; the value is that
    measured time, so steps x value is the timed region."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    pr, cfg = make_problem(args.workload, args.n)
    spr = reference_sample(pr)
    times = []
    desc = ""
    t_all = time.perf_counter()
    for i in range(args.warmup + args.steps):
        if i == args.warmup:
            t_all = time.perf_counter()
        ms, desc, cores = oracle_solve_time(spr)
        if i >= args.warmup:
            times.append(ms)
    wall = time.perf_counter() - t_all
    v = statistics.mean(times)
    size = "x".join(map(str, spr.n[:spr.dim]))
    cfg = dict(cfg, l2="oracle on host cores")
    if spr is not pr:
        cfg = dict(cfg, workload=spr.name, sample_of=cfg["workload"])
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "impl": "reference",
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each step: {desc}" + ("" if spr is pr else
                                       f" (a bounded sample of the {cfg['sample_of']} workload: the "
                                       f"same generator at {size})")},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s_timed_steps": wall}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------- our arm
def run_ours(args):
    import numpy as np
    import torch
    from paper_1308_4605_gb300 import stokes as S

    reps = Replicas("nccl")
    world, rank, local = reps.world, reps.rank, reps.local
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    barrier = reps.barrier

    pr, cfg = make_problem(args.workload, args.n)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    rho, mu = t(pr.rho), t(pr.mu)
    b_u = [t(x) for x in pr.b_u]
    b_p = t(pr.b_p)
    solver = S.StokesSolver(pr.dim, pr.n[:pr.dim], pr.bc[:2 * pr.dim], pr.h)
    x_u, x_p = solver.zeros(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def params(precision):
        p = S.stk_default_params()
        p.precond = pr.precond
        p.rtol = 1e-10
        p.maxit = 3000
        p.precision = precision
        return p

    def step(precision):
        solver.set_coefficients(rho, mu, pr.theta)
        for v in x_u:
            v.zero_()
        x_p.zero_()
        return S.stk_solve(solver.handle, params(precision), b_u, b_p, x_u, x_p)

    def timed(precision, k):
        times, infos = [], []
        for _ in range(k):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = step(precision)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            infos.append(info)
        return times, infos

    if args.quick:
        form = S.STK_MIXED if args.form == "mixed" else S.STK_FP64
        from paper_1308_4605_gb300 import tuning
        solver.set_coefficients(rho, mu, pr.theta)
        tuning.tune(solver, form)   # cached: a repeated command launches no tuning kernels
        if args.schedule:
            S.stk_set_schedule(solver.handle, form, *[int(v) for v in args.schedule.split(",")])
        if args.no_graphs:
            S.stk_set_graphs(solver.handle, 0)
        for _ in range(args.warmup):
            step(form)
        times, infos = timed(form, args.steps)
        if rank == 0:
            print(json.dumps({"quick": True, "form": args.form, "graphs": not args.no_graphs,
                              "schedule": S.stk_get_schedule(solver.handle, form),
                              "ms": times, "iterations": infos[0]["iterations"],
                              "true_residual": infos[0]["true_residual"], "config": cfg}))
        solver.close()
        return 0

    from paper_1308_4605_gb300 import tuning
    solver.set_coefficients(rho, mu, pr.theta)
    schedules = {"fp64": tuning.tune(solver, S.STK_FP64), "mixed": tuning.tune(solver, S.STK_MIXED)}
    for _ in range(args.warmup):
        step(S.STK_FP64)
        step(S.STK_MIXED)
    torch.cuda.synchronize()

    clk = ClockSampler(local)
    clk.start()
    barrier()
    torch.cuda.synchronize()
    k0 = S.stk_kernel_launches(solver.handle)
    t_wall = time.perf_counter()
    times64, infos64 = timed(S.STK_FP64, args.steps)
    barrier()
    torch.cuda.synchronize()
    wall64 = time.perf_counter() - t_wall
    launches = S.stk_kernel_launches(solver.handle) - k0
    times_mx, infos_mx = timed(S.STK_MIXED, args.steps)
    torch.cuda.synchronize()
    clocks = clk.stop()

    ms64 = statistics.mean(times64)
    ms_mx = statistics.mean(times_mx)
    ms64, ms_mx = reps.max([ms64, ms_mx], dev)

    # ---- end to end through the C ABI from pinned host buffers
    e2e = None
    if not args.no_e2e:
        h_in = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in
                [pr.rho, pr.mu] + list(pr.b_u) + [pr.b_p]]
        h_out = [torch.empty(v.shape, dtype=torch.float64).pin_memory() for v in x_u + [x_p]]
        d_in = [rho, mu] + b_u + [b_p]
        h2d = sum(v.numel() * 8 for v in h_in)
        d2h = sum(v.numel() * 8 for v in h_out)
        et = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for d, hh in zip(d_in, h_in):
                d.copy_(hh, non_blocking=True)
            step(S.STK_FP64)
            for hh, d in zip(h_out, x_u + [x_p]):
                hh.copy_(d, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            et.append(e0.elapsed_time(e1))
        e2e = {"value": statistics.mean(et), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    # ---- per-kernel device time (CUDA events on the solve's stream), one
    # extra FP64 step and one extra mixed step after the timed ones
    def profile(precision):
        S.stk_profile(solver.handle, 1)
        flush.fill_(1.0)
        step(precision)
        fam = [S.stk_profile_read(solver.handle, k) for k in range(S.STK_NPROF)]
        S.stk_profile(solver.handle, 0)
        return [f for f in fam if f["launches"] > 0]

    fam64 = profile(S.STK_FP64)
    fam_mx = profile(S.STK_MIXED)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    wl_name = cfg["workload"]
    roofline = roofline_of(fam64, "fp64", peaks, workload=wl_name)
    roofline_mixed = roofline_of(fam_mx, "mixed", peaks, workload=wl_name)
    # the level-0 FP32 smoother: the mixed form's bandwidth-bound kernel (the
    # dominant family above is latency-bound work on the small levels)
    roofline_mixed_l0 = roofline_of(fam_mx, "mixed", peaks, "vel_smooth_colour_l0", wl_name) \
        if any(f["name"] == "vel_smooth_colour_l0" for f in fam_mx) else None

    def fam_table(fams, total):
        return {f["name"]: {"launches": f["launches"], "ms": round(f["ms"], 4),
                            "share": round(f["ms"] / total, 4),
                            "GBps": round(f["bytes"] / max(f["ms"], 1e-9) / 1e6, 1),
                            "TFLOPs": round(f["flops"] / max(f["ms"], 1e-9) / 1e9, 3)} for f in fams}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cms, desc, cores = oracle_solve_time(pr)
            cpu = {"value": cms, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}
        except Exception as e:  # the baseline is informative only
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {e}"}

    others = None
    if rank == 0 and world == 1 and args.workload == "c3" and not args.no_others:
        others = other_configs(min(args.steps, 5), min(args.warmup, 2), peaks)

    line = {
        "metric": METRIC, "value": ms64, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms64, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(cfg, l2="flushed between steps (256 MB write); inputs > L2",
                       parallelism="replicas" if world > 1 else "single GPU"),
        "gmres_iterations": infos64[0]["iterations"],
        "multigrid_schedules": schedules,
        "true_residual": max(i["true_residual"] for i in infos64),
        "scalar_vcycles": infos64[0]["scalar_vcycles"],
        "forms": {
            "fp64": {"ms": ms64, "iterations": infos64[0]["iterations"],
                     "true_residual": max(i["true_residual"] for i in infos64)},
            "mixed_fp32_precond": {"ms": ms_mx, "iterations": infos_mx[0]["iterations"],
                                   "true_residual": max(i["true_residual"] for i in infos_mx),
                                   "speedup_vs_fp64": ms64 / ms_mx},
        },
        "roofline": roofline,
        "roofline_mixed": roofline_mixed,
        "roofline_mixed_l0": roofline_mixed_l0,
        "kernels_fp64": fam_table(fam64, sum(f["ms"] for f in fam64)),
        "kernels_mixed": fam_table(fam_mx, sum(f["ms"] for f in fam_mx)),
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
        "wall_s_fp64_steps": wall64,
        "other_configs": others,
    }
    if rank == 0:
        print(json.dumps(line))
    solver.close()
    reps.close()
    return 0


def measure_batched(steps, warmup, e2e=True, only=None, graphs=True):
    """64 independent 2D periodic unsteady instances of {64..512}^2 (sizes
    drawn by seed), mu contrast 1e3, P1: one after another with the FP64
    solver; all together with stk_solve_batched over one handle per instance
    (FP64 and mixed); and as stacked batches, one handle per grid size
    holding all instances of that size (stk_create_stacked), solved one
    group after another (each GMRES cycle one graph launch for the group) or
    all groups together with stk_solve_batched.  With e2e, the fastest
    batched form again from pinned host buffers (inputs copied in, solutions
    copied out, inside the timed region)."""
    import numpy as np
    import torch
    from paper_1308_4605_gb300 import stokes as S
    from paper_1308_4605_gb300 import tuning
    from paper_1308_4605_gb300 import workloads as wl
    dev = torch.device("cuda", 0)
    sizes = wl.config_c4_sizes()
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    solvers, bus, bps, xus, xps, prs = [], [], [], [], [], []
    for i, n in enumerate(sizes):
        pr = wl.config_c4_instance(i, n)
        sv = S.StokesSolver(2, pr.n[:2], pr.bc[:4], pr.h)
        sv.set_coefficients(t(pr.rho), t(pr.mu), pr.theta)
        tuning.tune(sv, S.STK_FP64)
        tuning.tune(sv, S.STK_MIXED)
        solvers.append(sv)
        prs.append(pr)
        bus.append([t(x) for x in pr.b_u])
        bps.append(t(pr.b_p))
        xu, xp = sv.zeros(dev)
        xus.append(xu)
        xps.append(xp)
    # stacked batches: one handle per grid size, the instances of that size
    # along the leading axis of every array
    groups = []
    for n in sorted(set(sizes)):
        idx = [i for i, s in enumerate(sizes) if s == n]
        p0 = prs[idx[0]]
        sv = S.StokesSolver(2, p0.n[:2], p0.bc[:4], p0.h, count=len(idx))
        stk = lambda arrs, shape: t(np.stack(arrs)).reshape(shape)
        sv.set_coefficients(stk([prs[i].rho for i in idx], sv.cell_shape()),
                            stk([prs[i].mu for i in idx], sv.cell_shape()), p0.theta)
        tuning.tune(sv, S.STK_FP64)
        tuning.tune(sv, S.STK_MIXED)
        bu = [stk([prs[i].b_u[a] for i in idx], sv.face_shape(a)) for a in range(2)]
        bp = stk([prs[i].b_p for i in idx], sv.cell_shape())
        xu, xp = sv.zeros(dev)
        if not graphs:   # every kernel launched from the host (for profilers)
            S.stk_set_graphs(sv.handle, 0)
        groups.append({"n": n, "idx": idx, "sv": sv, "bu": bu, "bp": bp, "xu": xu, "xp": xp})
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def params(precision):
        p = S.stk_default_params()
        p.precision = precision
        p.precond = 1
        p.maxit = 3000
        return p

    def zero_stacked():
        for gr in groups:
            for v in gr["xu"]:
                v.zero_()
            gr["xp"].zero_()

    def instance_infos():
        return [gr["sv"].instance_info(k) for gr in groups for k in range(len(gr["idx"]))]

    def stacked(precision):
        """one stacked handle after another (each solve: one graph launch per
        GMRES cycle for all instances of the group)"""
        zero_stacked()
        for gr in groups:
            S.stk_solve(gr["sv"].handle, params(precision), gr["bu"], gr["bp"], gr["xu"], gr["xp"])
        return instance_infos()

    def stacked_batched(precision):
        """the groups together: stk_solve_batched over the stacked handles"""
        zero_stacked()
        S.stk_solve_batched([gr["sv"].handle for gr in groups], params(precision),
                            [gr["bu"] for gr in groups], [gr["bp"] for gr in groups],
                            [gr["xu"] for gr in groups], [gr["xp"] for gr in groups])
        return instance_infos()

    def zero():
        for xu, xp in zip(xus, xps):
            for v in xu:
                v.zero_()
            xp.zero_()

    def sequential(precision):
        zero()
        its = []
        for k, sv in enumerate(solvers):
            its.append(S.stk_solve(sv.handle, params(precision), bus[k], bps[k], xus[k], xps[k]))
        return its

    def batched(precision):
        zero()
        return S.stk_solve_batched([sv.handle for sv in solvers], params(precision), bus, bps, xus, xps)

    def timed(fn, precision, k):
        times, infos = [], None
        for _ in range(k):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            infos = fn(precision)
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        return statistics.mean(times), infos

    res = {}
    forms = (("sequential_fp64", sequential, S.STK_FP64),
             ("batched_fp64", batched, S.STK_FP64),
             ("batched_mixed", batched, S.STK_MIXED),
             ("sequential_mixed", sequential, S.STK_MIXED),
             ("stacked_fp64", stacked, S.STK_FP64),
             ("stacked_mixed", stacked, S.STK_MIXED),
             ("stacked_batched_fp64", stacked_batched, S.STK_FP64),
             ("stacked_batched_mixed", stacked_batched, S.STK_MIXED))
    if only:   # a subset (profiling runs): no comparison solves, no e2e
        forms = tuple(f for f in forms if f[0] in only)
        e2e = False
    for _ in range(warmup):
        for name, fn, prec in forms:
            fn(prec)
    for name, fn, prec in forms:
        ms, infos = timed(fn, prec, steps)
        res[name] = {"ms": ms, "iterations_total": int(sum(i["iterations"] for i in infos)),
                     "max_true_residual": max(i["true_residual"] for i in infos),
                     "all_converged": all(i["converged"] for i in infos)}
        if name.startswith("stacked") and not only:
            # every instance against its own-handle solution of the same form
            ref = batched(prec)
            diff = 0.0
            for gr in groups:
                for k, i in enumerate(gr["idx"]):
                    a = torch.cat([v[k].reshape(-1) for v in gr["xu"]] + [gr["xp"][k].reshape(-1)])
                    b = torch.cat([v.reshape(-1) for v in xus[i]] + [xps[i].reshape(-1)])
                    diff = max(diff, float(torch.linalg.norm(a - b) / torch.linalg.norm(b)))
            res[name]["max_rel_diff_vs_per_handle_solution"] = diff
    best = min((n for n in res if n.startswith(("batched", "stacked"))), key=lambda n: res[n]["ms"],
               default=min(res, key=lambda n: res[n]["ms"]))
    seq = res.get("sequential_fp64")
    out = {"forms": res, "sizes_histogram": {str(n): sizes.count(n) for n in sorted(set(sizes))},
           "cells": int(sum(n * n for n in sizes)), "fastest_batched_form": best,
           "stacked_groups": {str(gr["n"]): len(gr["idx"]) for gr in groups},
           "speedup_batched_mixed_vs_sequential_fp64":
               seq["ms"] / res["batched_mixed"]["ms"] if seq and "batched_mixed" in res else None,
           "speedup_fastest_vs_sequential_fp64": seq["ms"] / res[best]["ms"] if seq else None}
    fns = {name: (fn, prec) for name, fn, prec in forms}
    if e2e:
        # the fastest form from pinned host buffers: the per-handle forms copy
        # each instance's arrays, the stacked forms each group's stacked arrays
        if best.startswith("stacked"):
            dins = [gr["bu"] + [gr["bp"]] for gr in groups]
            douts = [gr["xu"] + [gr["xp"]] for gr in groups]
        else:
            dins = [bus[k] + [bps[k]] for k in range(len(solvers))]
            douts = [xus[k] + [xps[k]] for k in range(len(solvers))]
        h_in = [[torch.empty(d.shape, dtype=torch.float64).pin_memory() for d in ds] for ds in dins]
        for hs, ds in zip(h_in, dins):
            for hh, d in zip(hs, ds):
                hh.copy_(d)
        h_out = [[torch.empty(d.shape, dtype=torch.float64).pin_memory() for d in ds] for ds in douts]
        h2d = sum(v.numel() * 8 for hs in h_in for v in hs)
        d2h = sum(v.numel() * 8 for hs in h_out for v in hs)
        fn, prec = fns[best]
        et = []
        for _ in range(steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for hs, ds in zip(h_in, dins):
                for hh, d in zip(hs, ds):
                    d.copy_(hh, non_blocking=True)
            fn(prec)
            for hs, ds in zip(h_out, douts):
                for hh, d in zip(hs, ds):
                    hh.copy_(d, non_blocking=True)
            e1.record()
            e1.synchronize()
            et.append(e0.elapsed_time(e1))
        out["e2e"] = {"value": statistics.mean(et), "unit": UNIT, "form": best,
                      "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
    for sv in solvers:
        sv.close()
    for gr in groups:
        gr["sv"].close()
    return out


def measure_config(pr, steps, warmup, peaks, maxit=3000, e2e=True, cpu=False, precond=None,
                   history=False):
    """Time-to-1e-10 of one workload on cuda:0 in both forms (set the
    coefficients, solve from x = 0), with the dominant kernel family's
    roofline from one profiled FP64 solve, the FP64 solve from pinned host
    buffers (e2e) and, with cpu, the oracle's full solve of the same
    workload.  A solve that stops at maxit is reported with its residual."""
    import numpy as np
    import torch
    from paper_1308_4605_gb300 import stokes as S
    from paper_1308_4605_gb300 import tuning
    dev = torch.device("cuda", 0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    rho, mu = t(pr.rho), t(pr.mu)
    b_u = [t(x) for x in pr.b_u]
    b_p = t(pr.b_p)
    sv = S.StokesSolver(pr.dim, pr.n[:pr.dim], pr.bc[:2 * pr.dim], pr.h)
    x_u, x_p = sv.zeros(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    pc = precond or pr.precond

    def step(precision):
        sv.set_coefficients(rho, mu, pr.theta)
        for v in x_u:
            v.zero_()
        x_p.zero_()
        p = S.stk_default_params()
        p.precond, p.rtol, p.maxit, p.precision = pc, 1e-10, maxit, precision
        return S.stk_solve(sv.handle, p, b_u, b_p, x_u, x_p)

    sv.set_coefficients(rho, mu, pr.theta)
    out = {"precond": f"P{pc}"}
    for name, prec in (("fp64", S.STK_FP64), ("mixed", S.STK_MIXED)):
        tuning.tune(sv, prec)
        for _ in range(warmup):
            step(prec)
        times = []
        for _ in range(steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            info = step(prec)
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        rec = {"ms": statistics.mean(times), "iterations": info["iterations"],
               "converged": bool(info["converged"]), "true_residual": info["true_residual"]}
        if history:
            h = S.stk_solve_history(sv.handle, 0)
            stride = max(1, len(h) // 20)
            rec["true_residual_at_restarts"] = {str(i): h[i] for i in range(0, len(h), stride)}
            rec["true_residual_at_restarts"][str(len(h) - 1)] = h[-1]
        out[name] = rec
    S.stk_profile(sv.handle, 1)
    flush.fill_(1.0)
    step(S.STK_FP64)
    fams = [f for f in (S.stk_profile_read(sv.handle, k) for k in range(S.STK_NPROF)) if f["launches"] > 0]
    S.stk_profile(sv.handle, 0)
    out["roofline"] = roofline_of(fams, "fp64", peaks, workload=pr.name)
    if e2e:
        h_in = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in
                [pr.rho, pr.mu] + list(pr.b_u) + [pr.b_p]]
        h_out = [torch.empty(v.shape, dtype=torch.float64).pin_memory() for v in x_u + [x_p]]
        et = []
        for _ in range(steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for d, hh in zip([rho, mu] + b_u + [b_p], h_in):
                d.copy_(hh, non_blocking=True)
            step(S.STK_FP64)
            for hh, d in zip(h_out, x_u + [x_p]):
                hh.copy_(d, non_blocking=True)
            e1.record()
            e1.synchronize()
            et.append(e0.elapsed_time(e1))
        out["e2e"] = {"value": statistics.mean(et), "unit": UNIT,
                      "h2d_bytes_per_step": sum(v.numel() * 8 for v in h_in),
                      "d2h_bytes_per_step": sum(v.numel() * 8 for v in h_out)}
    sv.close()
    if cpu:
        cms, desc, cores = oracle_solve_time(pr)
        out["cpu_baseline"] = {"value": cms, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}
    return out


def other_configs(steps, warmup, peaks):
    """The remaining benchmark configurations, measured after the headline:
    2D 32^2 periodic unsteady (P1), the 2D 512^2 sharp-inclusion workload
    (P2 and P1, and the tanh-smoothed variant; these stall, so they run to a
    bounded iteration count and report their residual histories), the
    64-instance batched workload and the 256^3 steady forward + adjoint."""
    from paper_1308_4605_gb300 import workloads as wl
    out = {}
    out["2d_unsteady_periodic_32^2"] = measure_config(wl.config_c1(32), steps, warmup, peaks, cpu=True)
    c2 = wl.config_c2(512)
    out["2d_steady_noslip_20_inclusions_mu1e4_512^2"] = {
        "P2": measure_config(c2, 1, 0, peaks, maxit=500, e2e=False, history=True),
        "P1": measure_config(c2, 1, 0, peaks, maxit=500, e2e=False, precond=1, history=True),
        "P2_tanh_smoothed_eps_h": measure_config(wl.config_c2(512, smooth=True), 1, 0, peaks, maxit=500,
                                                 e2e=False, history=True),
        "note": "the App. C velocity V-cycle diverges on the sharp mu = 1e4 disks and GMRES(10) stalls; "
                "bounded at 500 iterations"}
    out["batched_64_periodic_2d_instances"] = measure_batched(steps, warmup)
    out["adjoint_3d_steady_noslip_256^3"] = measure_adjoint(256, max(1, steps // 4), 1)
    return out


def run_batched(args):
    only = set(f for f in args.batched_forms.split(",") if f) or None
    r = measure_batched(args.steps, args.warmup, only=only, graphs=not args.no_graphs)
    res = r["forms"]
    best = r["fastest_batched_form"]
    line = {"metric": METRIC, "value": res[best]["ms"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res[best]["ms"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
            "data": "synthetic",
            "config": {"workload": f"batched_64_periodic_2d_instances_{r['cells']}_cells",
                       "sizes_histogram": r["sizes_histogram"],
                       "mu_contrast": 1e3, "precond": "P1", "l2": "flushed between steps", "form": best},
            "forms": res, "e2e": r.get("e2e"), "stacked_groups": r["stacked_groups"],
            "speedup_fastest_vs_sequential_fp64": r["speedup_fastest_vs_sequential_fp64"]}
    print(json.dumps(line))
    return 0


def measure_adjoint(n, steps, warmup):
    """Forward + adjoint (gradient w.r.t. log mu) of the 3D steady no-slip
    workload at n^3, loss 1/2||u - u_t||^2, FP64 and mixed."""
    import numpy as np
    import torch
    from paper_1308_4605_gb300 import adjoint
    from paper_1308_4605_gb300 import stokes as S
    from paper_1308_4605_gb300 import tuning
    from paper_1308_4605_gb300 import workloads as wl
    dev = torch.device("cuda", 0)
    pr = wl.config_c5(n)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    solver = S.StokesSolver(3, pr.n, pr.bc, pr.h)
    b_u = [t(x) for x in pr.b_u]
    b_p = t(pr.b_p)
    rng = np.random.default_rng(77)
    ut = [t(rng.standard_normal(x.shape)) for x in pr.b_u]
    rho = t(pr.rho)
    lm0 = t(np.log(pr.mu))
    solver.set_coefficients(rho, t(pr.mu), 0.0)
    for prec in (S.STK_FP64, S.STK_MIXED):
        tuning.tune(solver, prec)
    res = {}
    for name, precision in (("fp64", S.STK_FP64), ("mixed", S.STK_MIXED)):
        def step():
            lm = lm0.clone().requires_grad_(True)
            out = adjoint.stokes_solve(solver, lm, rho, 0.0, b_u, b_p, precond=2, rtol=1e-10,
                                       precision=precision, maxit=4000)
            L = 0.5 * sum(((o - q) ** 2).sum() for o, q in zip(out[:3], ut))
            L.backward()
            return lm.grad
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        times = []
        for _ in range(steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            gr = step()
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        res[name] = {"ms_forward_plus_adjoint": statistics.mean(times),
                     "grad_norm": float(torch.linalg.norm(gr))}
    solver.close()
    return res


def run_adjoint(args):
    n = args.n or 256
    res = measure_adjoint(n, args.steps, args.warmup)
    line = {"metric": METRIC, "value": res["mixed"]["ms_forward_plus_adjoint"], "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res["mixed"]["ms_forward_plus_adjoint"], "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": f"adjoint_3d_steady_noslip_{n}^3", "mu_contrast": 1e2, "precond": "P2"},
            "forms": res}
    print(json.dumps(line))
    return 0


def run_study(args):
    """The paper's bubble experiments (Sec. 4.1.2, 4.2, 4.3) with this solver:
    GMRES iterations and scalar V-cycles to a relative residual of 1e-10
    (FP64, left preconditioning), for the number of V-cycles per subsolve,
    the restart length, the five preconditioners, the viscous CFL number and
    the grid size.  The bubble (Eq. varcoeff_def) has mu = rho = 1 inside and
    r outside, so nu_0 = 1 and the viscous CFL number is beta = 1/theta
    (h = 1); beta = 0 is inviscid flow (mu = 0), beta = inf steady flow."""
    import numpy as np
    import torch
    from paper_1308_4605_gb300 import stokes as S
    from paper_1308_4605_gb300 import tuning
    from paper_1308_4605_gb300 import workloads as wl
    dev = torch.device("cuda", 0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    n2, n3 = 512, 128
    solvers = {}
    recs = []

    def run(exp, dim, n, r=100.0, beta=math.inf, precond=1, restart=10, cu=1, cp=1, note=None):
        pr = wl.bubble(dim, n, r, r)
        theta = 0.0 if math.isinf(beta) else (1.0 if beta == 0.0 else 1.0 / beta)
        mu = np.zeros_like(pr.mu) if beta == 0.0 else pr.mu
        key = (dim, n)
        if key not in solvers:
            for k in list(solvers):
                solvers.pop(k).close()
            torch.cuda.empty_cache()
            solvers[key] = S.StokesSolver(dim, pr.n[:dim], pr.bc[:2 * dim], pr.h)
        sv = solvers[key]
        sv.set_coefficients(t(pr.rho), t(mu), theta)
        tuning.tune(sv, S.STK_FP64)
        bu = [t(x) for x in pr.b_u]
        bp = t(pr.b_p)
        kw = dict(precond=precond, restart=restart, vcycles_u=cu, vcycles_p=cp, maxit=2000)
        sv.solve(bu, bp, **kw)                       # warm-up (graph capture)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        _, _, info = sv.solve(bu, bp, **kw)
        e1.record()
        e1.synchronize()
        rec = {"exp": exp, "dim": dim, "n": n, "r": r, "beta": None if math.isinf(beta) else beta,
               "precond": precond, "restart": restart, "vcycles_u": cu, "vcycles_p": cp,
               "iterations": info["iterations"], "scalar_vcycles": info["scalar_vcycles"],
               "converged": bool(info["converged"]), "true_residual": info["true_residual"],
               "ms": e0.elapsed_time(e1)}
        if note:
            rec["note"] = note
        recs.append(rec)
        print(json.dumps(rec), file=sys.stderr, flush=True)

    # Sec. 4.1.2: V-cycles per subsolve, P1, steady bubble, no restarts
    # (restart 32, the library's largest)
    for dim, n in ((2, n2), (3, n3)):
        for cu, cp in ((1, 1), (2, 2), (3, 3), (1, 2), (2, 1)):
            run("vcycles", dim, n, precond=1, restart=32, cu=cu, cp=cp)
    # Sec. 4.2.2: restart 5 vs 10, P1-P3, 2D: inviscid unsteady and steady viscous
    for beta in (0.0, math.inf):
        for pc in (1, 2, 3):
            for m in (5, 10):
                run("restart", 2, n2, beta=beta, precond=pc, restart=m)
    # Sec. 4.2.3: the five preconditioners, steady bubble, restart 10
    for dim, n in ((2, n2), (3, n3)):
        for pc in (1, 2, 3, 4, 5):
            run("preconditioners", dim, n, precond=pc)
    # Sec. 4.3.1: viscous CFL number, P1 and P2
    for dim, n in ((2, n2), (3, n3)):
        for beta in (0.0, 0.1, 1.0, 10.0, 100.0, 1e3, 1e4, math.inf):
            for pc in (1, 2):
                run("cfl", dim, n, beta=beta, precond=pc)
    # Sec. 4.3.2: grid size, steady, P1 and P2, r = 100 (and r = 2 in 3D)
    for pc in (1, 2):
        for n in (64, 128, 256, 512, 1024, 2048):
            run("size", 2, n, precond=pc)
        for n in (32, 64, 128, 256) + ((512,) if args.big else ()):
            run("size", 3, n, precond=pc)
        for n in (32, 64, 128, 256):
            run("size_r2", 3, n, r=2.0, precond=pc)
    for sv in solvers.values():
        sv.close()
    print(json.dumps({"metric": METRIC, "workload": "study: bubble experiments of Sec. 4",
                      "unit": UNIT, "data": "synthetic", "dtype": "f64", "results": recs}))
    return 0


def run_timeloop(args):
    """Backward-Euler time stepping (Sec. 2, Eq. Stokes_eqn) of the 128^3
    periodic workload (rho contrast 1e2, mu contrast 1e3, dt = 1, i.e.
    viscous CFL 1), constant forcing, from rest: ms and GMRES iterations per
    step, warm-started from the previous step and from zero, FP64 and mixed."""
    import numpy as np
    import torch
    from paper_1308_4605_gb300 import stokes as S
    from paper_1308_4605_gb300 import timeloop, tuning
    pr, cfg = make_problem("c3", args.n)
    dev = torch.device("cuda", 0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    sv = S.StokesSolver(pr.dim, pr.n[:pr.dim], pr.bc[:2 * pr.dim], pr.h)
    rho, mu = t(pr.rho), t(pr.mu)
    sv.set_coefficients(rho, mu, pr.theta)
    for prec in (S.STK_FP64, S.STK_MIXED):
        tuning.tune(sv, prec)
    f = [t(x) for x in pr.b_u]
    bp = t(pr.b_p)
    u0 = [torch.zeros_like(x) for x in f]
    nsteps = max(args.steps, 2)
    res = {}
    for name, prec in (("fp64", S.STK_FP64), ("mixed", S.STK_MIXED)):
        for warm in (True, False):
            timeloop.backward_euler(sv, rho, mu, 1.0, u0, 1, f=f, b_p=bp, warm=warm, precision=prec)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            _, _, infos = timeloop.backward_euler(sv, rho, mu, 1.0, u0, nsteps, f=f, b_p=bp,
                                                  warm=warm, precision=prec)
            e1.record()
            e1.synchronize()
            res[f"{name}_{'warm' if warm else 'cold'}"] = {
                "ms_per_step": e0.elapsed_time(e1) / nsteps,
                "iterations": [i["iterations"] for i in infos],
                "true_residual": max(i["true_residual"] for i in infos)}
    sv.close()
    print(json.dumps({"metric": METRIC, "workload": "backward-Euler steps of " + cfg["workload"],
                      "unit": UNIT, "steps": nsteps, "data": "synthetic", "dtype": "f64",
                      "dt": 1.0, "results": res}))
    return 0


def main():
    args = parse()
    if args.workload == "timeloop":
        return run_timeloop(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "study":
        return run_study(args)
    if args.workload == "c4":
        return run_batched(args)
    if args.workload == "c5adj":
        return run_adjoint(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
