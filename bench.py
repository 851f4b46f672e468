#!/usr/bin/env python
"""Benchmark of the hybrid multigrid hot path on one GB300 (or N replicas).

Workload (default): 2D -div(eps grad u) = f on the unit square, uniform k = 3
spacetree of level 6 (729 x 729 cells, 529,984 DoFs), eps piecewise constant on a
seeded 9 x 9 checkerboard with values {1, 1e-4}, f ~ U[-1, 1] per vertex, BoxMG
prolongation / restriction with Galerkin coarse operators stored as FP64
hierarchical deltas, damped Jacobi V(2,2) (omega 0.6), FP64 throughout, solved to
a 1e-10 relative residual drop.

A step = mg_setup (coarse coefficients, BoxMG, Galerkin R A P, deltas, coarsest
Cholesky) + mg_solve, inputs resident in HBM.  Metric: DoF/s to the 1e-10 drop
(DoFs x solves / time).  The mixed-precision form (FP64 refinement around FP32
V-cycles reading BF16 deltas) is measured on the same workload and reported
beside it.  L2 (126 MB) is flushed by writing a 512 MB buffer before every timed
step.
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

# the CPU oracle legs run on one core; set before numpy loads its BLAS
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synthetic as syn  # noqa: E402

WORKLOADS = {
    "checker2d-l6": dict(dim=2, L=6, eps="checker", eps_seed=0, load_seed=1, transfer="boxmg",
                         coarse="galerkin", tol=1e-10, max_cycles=3000,
                         desc="2D level 6 (729^2 cells, 529,984 DoFs), 9x9 seeded checkerboard {1,1e-4}, "
                              "BoxMG + Galerkin, V(2,2) omega 0.6, to 1e-10"),
    "jump2d-l6": dict(dim=2, L=6, eps="jump", eps_seed=0, load_seed="unit", transfer="boxmg",
                      coarse="galerkin", tol=1e-10, max_cycles=3000,
                      desc="2D level 6, the paper's jump benchmark (eps 1 / 0.1 across x_1 = 0.5, f = 1), "
                           "BoxMG + Galerkin, V(2,2), to 1e-10"),
    "grf2d-l6": dict(dim=2, L=6, eps="grf", eps_seed=1000, load_seed=2000, transfer="boxmg",
                     coarse="galerkin", tol=1e-10, max_cycles=3000,
                     desc="2D level 6, log-normal coefficient sigma 2, lambda 0.1 (the largest problem size "
                          "of the batched workload), BoxMG + Galerkin, V(2,2), to 1e-10"),
    "sin2d-l4": dict(dim=2, L=4, eps="const", eps_seed=0, load_seed=None, transfer="dlinear",
                     coarse="redisc", tol=1e-8, max_cycles=200,
                     desc="2D level 4 (81^2 cells, 6,400 DoFs), sin benchmark, geometric V(2,2), to 1e-8"),
}

# Adaptive 3D workload: uniform to level 4 (81^3 cells), refined to level 5 in a shell
# around the sphere |x - (0.5, 0.5, 0.5)| = 0.3, eps 1e3 inside / 1 outside; the
# composite system of Sect. 3 (level-5 DoFs + unrefined level-4 DoFs), solved to 1e-10
# with BF16 deltas, FP32 composite cycles and FP64 refinement (FP64 beside it).
ADAPTIVE = {
    "sphere3d-l5": dict(dim=3, L=5, radius=0.3, load_seed=2, tol=1e-10, max_cycles=3000,
                        desc="3D adaptive: level 4 (81^3 cells) + level 5 in a shell around r = 0.3, "
                             "eps 1e3 / 1, BoxMG + Galerkin below level 4, composite cycles, "
                             "BF16 deltas + FP32 cycles + FP64 refinement to 1e-10"),
}

# FP64 flops per DoF of the finest 2D in-situ Jacobi sweep (k_sweep2f): two pair sums of
# cell coefficients (the other two are shared with the neighbouring column and the row
# below), the corner products (1 mul + 3 fma), their doubling, the edge products
# (4 fma), b - off (1 fma), (1 - omega) u and the update (1 mul + 1 fma); an fma counts
# 2 flops.  14 FP64 instructions issue these 23 flops.
FLOPS_PER_DOF_SWEEP_2D = 23
FP64_INSTR_PER_DOF_SWEEP_2D = 14
# algorithmic bytes of a finest Jacobi sweep: u, b, eps read and u' written, 8 B each
# (the stored omega / diag(A) adds 8 B read per DoF in this implementation)
BYTES_PER_DOF_SWEEP_FP64 = 32
BYTES_PER_DOF_SWEEP_FP64_IMPL = 40
# DRAM bytes per DoF of k_sweep2f from ncu (dram__bytes_read.sum + dram__bytes_write.sum)
# on the 2D level-7 case (python bench.py --sweep-level 7 --sweep-dim 2 --sweep-prec
# fp64), whose vectors exceed L2
TRAFFIC_PER_DOF_SWEEP_FP64_2D = 38.34
BYTES_PER_DOF_SWEEP_FP32 = 16


def inputs(w):
    L, d = w["L"], w["dim"]
    if w["eps"] == "checker":
        eps = syn.checkerboard_eps(L, d, seed=w["eps_seed"])
    elif w["eps"] == "jump":
        eps = syn.jump_eps(L, d)
    elif w["eps"] == "grf":
        eps = syn.lognormal_grf_eps(L, d, sigma=2.0, seed=w["eps_seed"])
    else:
        eps = syn.constant_eps(L, d)
    if w["load_seed"] == "unit":
        bf = syn.unit_load(L, d)
    else:
        bf = syn.uniform_load(L, d, w["load_seed"]) if w["load_seed"] is not None else syn.sin_load(L, d)
    return eps, bf


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def fp64_peak_tflops(mg, torch, reps=5):
    """FP64 fma rate of this GPU, measured: mg_probe_fp64_fma (8 independent fma chains
    per thread, 16 resident CTAs of 256 threads per SM, four waves) timed with CUDA
    events on the current stream; the best of `reps` launches after two warm-ups."""
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    n_ctas = sms * 8 * 4
    sink = torch.zeros(n_ctas, dtype=torch.float64, device="cuda")
    for _ in range(2):
        mg.probe_fp64_fma(n_ctas, 2048, sink)
    best = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fl = mg.probe_fp64_fma(n_ctas, 2048, sink)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        best = t if best is None or t < best else best
    return fl / best / 1e12


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # raw samples beside the run's other outputs (MG_BENCH_OUT, else the system temp dir)
        out = os.environ.get("MG_BENCH_OUT") or tempfile.gettempdir()
        self.path = os.path.join(out, f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait(timeout=10)
            self.f.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
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


_PROFILER_WARM = False


def measured_launches(step):
    """Kernels of this library (names in namespace mg) that one call of step() launches,
    counted from the CUDA activity trace of torch.profiler (kernels replayed from CUDA
    graphs included); an untimed run beside the timed ones."""
    global _PROFILER_WARM
    import torch
    from torch.profiler import ProfilerActivity, profile

    if not _PROFILER_WARM:  # the first trace of a process misses kernels
        with profile(activities=[ProfilerActivity.CUDA]):
            torch.zeros(8, device="cuda").sum()
            torch.cuda.synchronize()
        _PROFILER_WARM = True
    torch.cuda.synchronize()
    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        step()
        torch.cuda.synchronize()
    return sum(1 for ev in prof.events() if ev.device_type.name == "CUDA" and "mg::" in ev.name)


def adaptive_problem(mg, w):
    """Grid, level-concatenated eps and b, and the composite unknown count."""
    L, d = w["L"], w["dim"]
    T = L - 1
    mask = syn.sphere_shell_mask(T, d, radius=w["radius"])
    grid = mg.Grid(d, L, {T: mask})
    eps_cat = grid.cells_to_concat({L: syn.sphere_eps(L, d, radius=w["radius"]),
                                    T: syn.sphere_eps(T, d, radius=w["radius"])})
    iL, iT = grid.info(L), grid.info(T)
    unref = grid.dof_mask(T) & ((grid.tables(T)["vflags"] & 8) == 0)
    b = np.zeros(grid.n_slots_total())
    b[iL.slot_offset: iL.slot_offset + iL.n_slots] = grid.to_slots(L, syn.uniform_load(L, d, w["load_seed"]))
    b[iT.slot_offset: iT.slot_offset + iT.n_slots] = np.where(
        unref, grid.to_slots(T, syn.uniform_load(T, d, w["load_seed"] + 1)), 0.0)
    return grid, eps_cat, b, int(iL.n_dofs + unref.sum())


def run_adaptive(args):
    import torch

    import paper_1607_00648_gb300 as mg

    torch.cuda.set_device(0)
    w = ADAPTIVE[args.workload]
    L, d = w["L"], w["dim"]
    grid, eps_cat, b, n_dofs = adaptive_problem(mg, w)
    eps_dev = torch.from_numpy(eps_cat).cuda()
    b_dev = torch.from_numpy(b).cuda()
    u_dev = torch.zeros_like(b_dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(H, prec):
        for _ in range(args.warmup):
            H.setup(eps_dev)
            H.solve(u_dev, b_dev, rel_tol=w["tol"], max_cycles=w["max_cycles"])
        total, launches, res = 0.0, 0, None
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            H.setup(eps_dev)
            res = H.solve(u_dev, b_dev, rel_tol=w["tol"], max_cycles=w["max_cycles"])
            e1.record(stream)
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
        launches = args.steps * measured_launches(
            lambda: (H.setup(eps_dev), H.solve(u_dev, b_dev, rel_tol=w["tol"], max_cycles=w["max_cycles"])))
        return total, launches, res

    Hmx = mg.Hierarchy(grid, precision="mixed_bf16")
    H64 = mg.Hierarchy(grid, precision="fp64")
    tiles = {}
    if not args.no_autotune:
        for name, H in (("mixed", Hmx), ("fp64", H64)):
            H.setup(eps_dev)
            tiles[name] = {str(k): v for k, v in H.autotune().items()}
    do64, domx = args.precision in ("both", "fp64"), args.precision in ("both", "mixed")
    with Clocks(torch.cuda.current_device()) as clk:
        if domx:
            tmx, lmx, rmx = timed(Hmx, "mixed")
        if do64:
            t64, l64, r64 = timed(H64, "fp64")
    clocks = clk.summary()
    if not domx:  # FP64 only (profiling runs): the line reports the FP64 solve
        tmx, lmx, rmx = t64, 0, r64
    value = n_dofs * args.steps / (tmx / 1e3)
    value64 = n_dofs * args.steps / (t64 / 1e3) if do64 else None

    # dominant kernel of the mixed solve: the FP32 level-L sweep (hanging entries kept)
    if not domx:
        Hmx.setup(eps_dev)
    nL = grid.info(L).n_slots
    oL = grid.info(L).slot_offset
    u32 = torch.zeros(nL, dtype=torch.float32, device="cuda")
    b32 = b_dev[oL: oL + nL].float()
    for _ in range(5):
        Hmx.smooth_f32(L, u32, b32, 2)
    torch.cuda.synchronize()
    reps = 50
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        Hmx.smooth_f32(L, u32, b32, 2)
    e1.record(stream)
    torch.cuda.synchronize()
    sweep_s = e0.elapsed_time(e1) / 1e3 / (2 * reps)
    hbm_peak, src = peaks()
    nd_L = grid.info(L).n_dofs
    achieved = BYTES_PER_DOF_SWEEP_FP32 * nd_L / sweep_s / 1e9
    roofline = {"bound": "hbm", "kernel": "k_sweep<3,float,0,Jacobi> (level-5 FP32 Jacobi sweep)",
                "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                "peak_source": src, "bytes_per_dof": BYTES_PER_DOF_SWEEP_FP32, "dofs_per_launch": nd_L,
                "launch_us": sweep_s * 1e6, "traffic": None}

    # end to end with host buffers
    eps_h = torch.from_numpy(eps_cat).pin_memory()
    b_h = torch.from_numpy(b).pin_memory()
    u_h = torch.empty_like(b_h).pin_memory()
    e2e_ms = 0.0
    for i in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        eps_dev.copy_(eps_h, non_blocking=True)
        b_dev.copy_(b_h, non_blocking=True)
        Hmx.setup(eps_dev)
        Hmx.solve(u_dev, b_dev, rel_tol=w["tol"], max_cycles=w["max_cycles"])
        u_h.copy_(u_dev, non_blocking=True)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_ms += (time.perf_counter() - t0) * 1e3
    e2e = {"value": n_dofs * args.steps / (e2e_ms / 1e3), "unit": "DoF/s",
           "h2d_bytes_per_step": int(eps_h.numel() * 8 + b_h.numel() * 8), "d2h_bytes_per_step": int(u_h.numel() * 8)}
    out = {
        "metric": "DoF/s to 1e-10 residual drop (mixed; FP64 beside it)",
        "value": value, "unit": "DoF/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tmx / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 cycles + f64 refinement, bf16 deltas", "data": "synthetic",
        "config": {"workload": args.workload, "description": w["desc"], "dofs": n_dofs,
                   "level5_dofs": int(nd_L), "inner_cycles": rmx["cycles"], "outer_steps": rmx["outer_steps"],
                   "rel_residual": rmx["rel_residual"], "parallelism": "replicas1",
                   "l2": "flushed (512 MB write) before every timed step", "setup_included": True,
                   "tiles": tiles or "default rule"},
        "fp64": None if not (do64 and domx) else {
            "value": value64, "unit": "DoF/s", "ms_per_step": t64 / args.steps, "cycles": r64["cycles"],
            "rel_residual": r64["rel_residual"], "mixed_speedup": value / value64},
        "roofline": roofline, "e2e": e2e, "clocks": clocks, "gpu_launches": lmx + (l64 if do64 else 0),
        "cpu_baseline": None,
    }
    print(json.dumps(out))


def run_breakdown(args):
    """Per-kernel device time of one mg_setup + mg_solve of the workload, per solve form,
    from the CUDA activity trace of torch.profiler (kernels at full speed, in the order
    the solve runs them; a diagnostic beside the ncu launch lists)."""
    import collections
    import re

    import torch
    from torch.profiler import ProfilerActivity, profile

    import paper_1607_00648_gb300 as mg

    torch.cuda.set_device(0)
    with profile(activities=[ProfilerActivity.CUDA]):  # the first trace misses kernels
        torch.zeros(8, device="cuda").sum()
        torch.cuda.synchronize()
    if args.workload in ADAPTIVE:
        w = ADAPTIVE[args.workload]
        grid, eps_cat, b, n_dofs = adaptive_problem(mg, w)
        opts = {}
    else:
        w = WORKLOADS[args.workload]
        eps, bf = inputs(w)
        grid = mg.Grid(w["dim"], w["L"])
        eps_cat, b = grid.cells_to_concat({w["L"]: eps}), grid.to_slots(w["L"], bf)
        n_dofs = grid.info(w["L"]).n_dofs
        opts = {"transfer": w["transfer"], "coarse": w["coarse"]}
    if args.smoother != "jacobi":
        opts.update(smoother=args.smoother, gs_sweeps=args.gs_sweeps)
    e = torch.from_numpy(eps_cat).cuda()
    bd = torch.from_numpy(b).cuda()
    u = torch.zeros_like(bd)
    out = {"workload": args.workload, "dofs": n_dofs}
    precs = ("mixed_bf16", "mixed_bpa") if args.precision == "bpa" else ("fp64", "mixed_bf16")
    for prec in precs:
        if args.precision not in ("both", "bpa", prec.split("_")[0]):
            continue
        H = mg.Hierarchy(grid, precision=prec, **opts)
        H.setup(e)
        H.solve(u, bd, rel_tol=w["tol"], max_cycles=w["max_cycles"])
        torch.cuda.synchronize()
        with profile(activities=[ProfilerActivity.CUDA]) as prof:
            H.setup(e)
            res = H.solve(u, bd, rel_tol=w["tol"], max_cycles=w["max_cycles"])
            torch.cuda.synchronize()
        agg = collections.defaultdict(lambda: [0, 0.0])
        for ev in prof.events():
            if ev.device_type.name == "CUDA":
                k = re.sub(r"\(.*", "", ev.name).replace("void ", "").replace("mg::", "")
                agg[k][0] += 1
                agg[k][1] += ev.device_time_total
        tot = sum(v[1] for v in agg.values())
        out[prec] = {"cycles": res["cycles"], "outer_steps": res["outer_steps"], "solve_ms": res["solve_ms"],
                     "kernel_ms": tot / 1e3,
                     "kernels": [{"name": k, "launches": c, "ms": t / 1e3, "share": t / tot}
                                 for k, (c, t) in sorted(agg.items(), key=lambda kv: -kv[1][1])]}
        del H
    print(json.dumps(out))


def max_over_ranks(ms, dist=None, device=None):
    """The slowest rank's time (replicas: the job ends when the last one does)."""
    if dist is None:
        return ms
    import torch

    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank, steps, world, slowest_ms):
    """Whole-job rate of N independent replicas: every rank's units over the slowest time."""
    return units_per_rank * steps * world / (slowest_ms / 1e3)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_ours(args):
    import torch

    import paper_1607_00648_gb300 as mg

    world, rank, local = dist_setup()
    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        dist = dist_mod
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    w = WORKLOADS[args.workload]
    L, d = w["L"], w["dim"]
    eps, bf = inputs(w)
    grid = mg.Grid(d, L)
    n_dofs = grid.info(L).n_dofs
    eps_cat = grid.cells_to_concat({L: eps})
    b = grid.to_slots(L, bf)
    eps_dev = torch.from_numpy(eps_cat).to(dev)
    b_dev = torch.from_numpy(b).to(dev)
    u_dev = torch.zeros_like(b_dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if dist:
            dist.barrier()

    def timed(H, K, W, prec):
        res = None
        for _ in range(W):
            H.setup(eps_dev)
            res = H.solve(u_dev, b_dev, rel_tol=w["tol"], max_cycles=w["max_cycles"])
        total_ms, launches, stats = 0.0, 0, []
        for _ in range(K):
            flush.zero_()
            barrier()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            H.setup(eps_dev)
            res = H.solve(u_dev, b_dev, rel_tol=w["tol"], max_cycles=w["max_cycles"])
            e1.record(stream)
            torch.cuda.synchronize()
            barrier()
            total_ms += e0.elapsed_time(e1)
            stats.append(res)
        launches = K * measured_launches(
            lambda: (H.setup(eps_dev), H.solve(u_dev, b_dev, rel_tol=w["tol"], max_cycles=w["max_cycles"])))
        return max_over_ranks(total_ms, dist, dev), launches, stats

    smo = {} if args.smoother == "jacobi" else {"smoother": args.smoother, "gs_sweeps": args.gs_sweeps}
    cyc = {} if args.cycle == "v" else {"cycle": args.cycle}
    H64 = mg.Hierarchy(grid, transfer=w["transfer"], coarse=w["coarse"], precision="fp64", **smo, **cyc)
    Hmx = mg.Hierarchy(grid, transfer=w["transfer"], coarse=w["coarse"], precision="mixed_bf16", **smo)
    tiles = {}
    if not args.no_autotune:  # slab depths by measurement, once, outside the timed region
        for name, H in (("fp64", H64), ("mixed", Hmx)):
            H.setup(eps_dev)
            tiles[name] = {str(k): v for k, v in H.autotune().items()}
    do64, domx = args.precision in ("both", "fp64"), args.precision in ("both", "mixed")
    if cyc:  # the additive cycle runs on FP64 hierarchies only
        do64, domx = True, False
    with Clocks(torch.cuda.current_device()) as clk:
        if do64:
            t64, launches64, st64 = timed(H64, args.steps, args.warmup, "fp64")
        if domx:
            tmx, launchesmx, stmx = timed(Hmx, args.steps, args.warmup, "mixed")
    clocks = clk.summary()
    if not do64:  # mixed only (profiling runs): the line reports the mixed solve
        t64, launches64, st64 = tmx, 0, stmx
    value = replica_throughput(n_dofs, args.steps, world, t64)
    value_mx = replica_throughput(n_dofs, args.steps, world, tmx) if domx else None

    # the FP64 solve with float-float finest-level sweeps (FP64 vectors and setup)
    ff = None
    if do64 and not cyc and not smo and not args.no_ff:
        Hff = mg.Hierarchy(grid, transfer=w["transfer"], coarse=w["coarse"], precision="fp64", ff_sweeps=1)
        if not args.no_autotune:
            Hff.setup(eps_dev)
            tiles["fp64_ff"] = {str(k): v for k, v in Hff.autotune().items()}
        with Clocks(torch.cuda.current_device()) as clk_ff:
            tff, launchesff, stff = timed(Hff, args.steps, args.warmup, "fp64")
        launches64 += launchesff
        Hff.setup(eps_dev)
        ff = {"value": replica_throughput(n_dofs, args.steps, world, tff), "unit": "DoF/s",
              "dtype": "f64 vectors and setup, float-float finest-level sweeps",
              "ms_per_step": tff / args.steps, "cycles": stff[-1]["cycles"],
              "rel_residual": stff[-1]["rel_residual"], "clocks": clk_ff.summary(),
              "sweep_us": sweep_time(Hff, L, b_dev, stream) * 1e6}
        ff["speedup_vs_fp64"] = ff["value"] / value

    # dominant kernel: finest-level FP64 in-situ Jacobi sweep (two sweeps per call, no copy)
    H64.setup(eps_dev)
    sweep_s = sweep_time(H64, L, b_dev, stream)
    Hmx.setup(eps_dev)
    hbm_peak, peak_src = peaks()
    with Clocks(torch.cuda.current_device()) as clk_peak:
        fp64_peak = fp64_peak_tflops(mg, torch)
    flops = FLOPS_PER_DOF_SWEEP_2D * n_dofs
    achieved = flops / sweep_s / 1e12
    # the binding roofline of the sweep, in DoF/s: min(HBM at the algorithmic bytes,
    # FP64 units at the kernel's flops); the FP64 one binds on GB300
    dofs_hbm = hbm_peak * 1e9 / BYTES_PER_DOF_SWEEP_FP64
    dofs_fp64 = fp64_peak * 1e12 / FLOPS_PER_DOF_SWEEP_2D
    traffic = TRAFFIC_PER_DOF_SWEEP_FP64_2D * n_dofs if TRAFFIC_PER_DOF_SWEEP_FP64_2D else None
    roofline = {"bound": "alu", "kernel": "k_sweep2f<0,Jacobi> (finest FP64 Jacobi sweep, 2D column kernel)",
                "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                "peak_source": "measured: FP64 fma-chain probe (mg_probe_fp64_fma), CUDA events, this run",
                "peak_clocks": clk_peak.summary(),
                "flops_per_dof": FLOPS_PER_DOF_SWEEP_2D, "fp64_instr_per_dof": FP64_INSTR_PER_DOF_SWEEP_2D,
                "fp64_issue_frac": FP64_INSTR_PER_DOF_SWEEP_2D * n_dofs / sweep_s / (fp64_peak * 1e12 / 2),
                "dofs_per_launch": n_dofs, "launch_us": sweep_s * 1e6,
                "l2": "the level-6 vectors (~21 MB) are L2-resident; the kernel is bound by the FP64 units",
                "binding_roofline": {"hbm_dofs_per_s": dofs_hbm, "fp64_dofs_per_s": dofs_fp64,
                                     "bytes_per_dof": BYTES_PER_DOF_SWEEP_FP64,
                                     "achieved_dofs_per_s": n_dofs / sweep_s,
                                     "frac": n_dofs / sweep_s / min(dofs_hbm, dofs_fp64)},
                "hbm_equivalent": {"achieved": BYTES_PER_DOF_SWEEP_FP64 * n_dofs / sweep_s / 1e9,
                                   "peak": hbm_peak, "unit": "GB/s",
                                   "frac": BYTES_PER_DOF_SWEEP_FP64 * n_dofs / sweep_s / 1e9 / hbm_peak,
                                   "peak_source": peak_src},
                "traffic": traffic,
                "traffic_note": "ncu DRAM bytes per DoF of the level-7 case (vectors beyond L2) x DoFs"
                if traffic else "null: no ncu capture of the current kernel yet"}

    # end to end through the public API with host buffers
    eps_h = torch.from_numpy(eps_cat).pin_memory()
    b_h = torch.from_numpy(b).pin_memory()
    u_h = torch.empty_like(b_h).pin_memory()
    e2e_ms = 0.0
    for i in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        eps_dev.copy_(eps_h, non_blocking=True)
        b_dev.copy_(b_h, non_blocking=True)
        H64.setup(eps_dev)
        H64.solve(u_dev, b_dev, rel_tol=w["tol"], max_cycles=w["max_cycles"])
        u_h.copy_(u_dev, non_blocking=True)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_ms += (time.perf_counter() - t0) * 1e3
    e2e_ms = max_over_ranks(e2e_ms, dist, dev)
    e2e = {"value": replica_throughput(n_dofs, args.steps, world, e2e_ms), "unit": "DoF/s",
           "h2d_bytes_per_step": int(eps_h.numel() * 8 + b_h.numel() * 8),
           "d2h_bytes_per_step": int(u_h.numel() * 8)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(w, st64[-1]["cycles"])

    # the batched and served forms (task configs 4 and 5), reduced to finish within the
    # run: the first 128 problems of the batched workload, the first 150 requests of the
    # served stream; mixed against FP64 each
    batched = served = None
    if rank == 0 and world == 1 and not args.no_a13:
        with Clocks(torch.cuda.current_device()) as clk_a13:
            _, probs = batched_problems(mg, torch, 128)
            batched = batched_solves(mg, torch, probs, 1, flush)
            del probs
            torch.cuda.empty_cache()
            served = served_summary(mg, torch, 150, 200.0, 64.0)
        batched["clocks"] = served["clocks"] = clk_a13.summary()

    if rank == 0:
        out = {
            "metric": "DoF/s to 1e-10 residual drop (FP64; mixed beside it)",
            "value": value, "unit": "DoF/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t64 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if do64 else "f32 cycles + f64 refinement, bf16 deltas", "data": "synthetic",
            "config": {"workload": args.workload, "description": w["desc"], "dofs": n_dofs,
                       "cycles_per_solve": st64[-1]["cycles"], "parallelism": f"replicas{world}",
                       "l2": "flushed (512 MB write) before every timed step", "setup_included": True,
                       "tiles": tiles or "default rule",
                       "smoother": "damped Jacobi" if not smo else f"block Jacobi, {args.gs_sweeps} Gauss-Seidel "
                                                                     f"sweep(s) per patch (Sect. 4.2)",
                       "cycle": "V(2,2)" if not cyc else {"additive": "additive (Alg. 2)", "bpx": "BPX (Alg. 3)"}[args.cycle]},
            "mixed": None if not (domx and do64) else {
                "value": value_mx, "unit": "DoF/s", "dtype": "f32 cycles + f64 refinement, bf16 deltas",
                "ms_per_step": tmx / args.steps, "inner_cycles": stmx[-1]["cycles"],
                "outer_steps": stmx[-1]["outer_steps"], "rel_residual": stmx[-1]["rel_residual"],
                "speedup_vs_fp64": value_mx / value},
            "fp64_ff": ff,
            "roofline": roofline, "e2e": e2e, "clocks": clocks,
            "gpu_launches": launches64 + (launchesmx if domx else 0),
            "cpu_baseline": cpu,
            "batched": batched, "served": served,
        }
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def sweep_time(H, L, b_dev, stream, reps=50):
    """Seconds per finest-level Jacobi sweep of H (mg_smooth with two sweeps per call, CUDA
    events on the launching stream, after 5 warm-up calls)."""
    import torch

    uu = torch.zeros_like(b_dev)
    for _ in range(5):
        H.smooth(L, uu, b_dev, 2)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        H.smooth(L, uu, b_dev, 2)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3 / (2 * reps)


def run_codecs(args):
    """Mixed solves with the deltas in BF16 + FP32 scale against the paper's bpa codec
    (Sect. 5) at eps_mf = 1e-2, 1e-4, 1e-8: DoF/s, cycles and stored delta bytes."""
    import torch

    import paper_1607_00648_gb300 as mg

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    w = WORKLOADS[args.workload]
    L, d = w["L"], w["dim"]
    eps, bf = inputs(w)
    grid = mg.Grid(d, L)
    n_dofs = grid.info(L).n_dofs
    eps_dev = torch.from_numpy(grid.cells_to_concat({L: eps})).to(dev)
    b_dev = torch.from_numpy(grid.to_slots(L, bf)).to(dev)
    u_dev = torch.zeros_like(b_dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    n3, n5 = 3 ** d, 5 ** d
    out = {}
    with Clocks(0) as clk:
        for name, kw in (("bf16", {"precision": "mixed_bf16"}),
                         ("bpa_1e-2", {"precision": "mixed_bpa", "eps_mf": 1e-2}),
                         ("bpa_1e-4", {"precision": "mixed_bpa", "eps_mf": 1e-4}),
                         ("bpa_1e-8", {"precision": "mixed_bpa", "eps_mf": 1e-8})):
            H = mg.Hierarchy(grid, transfer=w["transfer"], coarse=w["coarse"], **kw)
            for _ in range(args.warmup):
                H.setup(eps_dev)
                H.solve(u_dev, b_dev, rel_tol=w["tol"], max_cycles=w["max_cycles"])
            ms, res = 0.0, None
            for _ in range(args.steps):
                flush.zero_()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                H.setup(eps_dev)
                res = H.solve(u_dev, b_dev, rel_tol=w["tol"], max_cycles=w["max_cycles"])
                e1.record(stream)
                torch.cuda.synchronize()
                ms += e0.elapsed_time(e1)
            coarse_slots = coarse_dofs = stored = 0
            hist = {}
            for lv in range(H.options.coarsest_level, L):
                inf = grid.info(lv)
                coarse_slots += inf.n_slots
                coarse_dofs += inf.n_dofs
                if kw["precision"] == "mixed_bf16":
                    stored += inf.n_slots * ((n3 + n5) * 2 + 8)
                else:
                    ar = torch.empty(inf.n_slots, dtype=torch.int64, device=dev)
                    pr = torch.empty(inf.n_slots, dtype=torch.int64, device=dev)
                    na, npb = H.get_bpa(lv, a_rec=ar, p_rec=pr)
                    stored += na + npb + inf.n_slots * 16
                    for r in (ar, pr):
                        vals, cnt = np.unique((r.cpu().numpy().view(np.uint64) & np.uint64(15)).astype(int),
                                              return_counts=True)
                        for v, c in zip(vals, cnt):
                            hist[int(v)] = hist.get(int(v), 0) + int(c)
            out[name] = {"dofs_per_s": n_dofs * args.steps / (ms / 1e3), "ms_per_step": ms / args.steps,
                         "inner_cycles": res["cycles"], "outer_steps": res["outer_steps"],
                         "rel_residual": res["rel_residual"], "delta_bytes": stored,
                         "delta_bytes_per_coarse_dof": stored / max(coarse_dofs, 1),
                         "bpa_histogram": hist or None}
            del H
    line = {"metric": "DoF/s to 1e-10 residual drop, mixed path by delta codec", "unit": "DoF/s",
            "value": out["bpa_1e-4"]["dofs_per_s"], "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "dtype": "f32 cycles + f64 refinement", "data": "synthetic",
            "config": {"workload": args.workload, "description": w["desc"], "dofs": n_dofs,
                       "l2": "flushed (512 MB write) before every timed step", "setup_included": True},
            "codecs": out, "clocks": clk.summary()}
    print(json.dumps(line))


def run_sweeps(args):
    """Finest-level in-situ Jacobi sweeps alone on a uniform checkerboard grid of level
    args.sweep_level and dimension args.sweep_dim (2D level 8: 6561^2 cells, 43M DoFs;
    3D level 5: 243^3 cells, 14M DoFs; vectors larger than L2): per-launch time of the
    FP64 and the FP32 sweep kernels and their roofline."""
    import torch

    import paper_1607_00648_gb300 as mg

    torch.cuda.set_device(0)
    L, d = args.sweep_level, args.sweep_dim
    eps = syn.checkerboard_eps(L, d, seed=0)
    grid = mg.Grid(d, L)
    n_dofs = grid.info(L).n_dofs
    eps_dev = torch.from_numpy(grid.cells_to_concat({L: eps})).cuda()
    b64 = torch.from_numpy(grid.to_slots(L, syn.uniform_load(L, d, 1))).cuda()
    H = mg.Hierarchy(grid, precision="mixed_bf16")  # FP32 sweeps
    H.setup(eps_dev)
    H64 = mg.Hierarchy(grid, precision="fp64") if args.sweep_prec in ("both", "fp64") else None
    if H64 is not None:
        H64.setup(eps_dev)
    Hff = mg.Hierarchy(grid, precision="fp64", ff_sweeps=1) if args.sweep_prec in ("both", "ff") else None
    if Hff is not None:
        Hff.setup(eps_dev)
    u64 = torch.zeros_like(b64)
    b32 = b64.float()
    u32 = torch.zeros_like(b32)
    hbm, src = peaks()
    out = {"workload": f"sweep{d}d-l{L}", "dofs": n_dofs}
    if H64 is not None:  # the FP64 setup of this grid (BoxMG, Galerkin R A P, deltas, coarse factor)
        ts = []
        for _ in range(3):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            H64.setup(eps_dev)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        out["setup_fp64_ms"] = min(ts)
    for name, bpd in (("fp64", BYTES_PER_DOF_SWEEP_FP64), ("ff", BYTES_PER_DOF_SWEEP_FP64),
                      ("fp32", BYTES_PER_DOF_SWEEP_FP32)):
        if args.sweep_prec not in ("both", name):
            continue
        fn, u, bb = {"fp64": (H64 and H64.smooth, u64, b64), "ff": (Hff and Hff.smooth, u64, b64),
                     "fp32": (H.smooth_f32, u32, b32)}[name]
        for _ in range(3):
            fn(L, u, bb, 2)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = args.steps
        e0.record()
        for _ in range(reps):
            fn(L, u, bb, 2)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3 / (2 * reps)
        out[name] = {"launch_us": t * 1e6, "GB/s": bpd * n_dofs / t / 1e9, "hbm_frac": bpd * n_dofs / t / 1e9 / hbm,
                     "peak_source": src, "Gdof/s": n_dofs / t / 1e9}
        if name == "fp64" and d == 2:
            out[name]["TFLOP/s"] = FLOPS_PER_DOF_SWEEP_2D * n_dofs / t / 1e12
    if args.sweep_prec in ("both", "fp64"):
        out["fp64_peak_tflops"] = fp64_peak_tflops(mg, torch)
        if "TFLOP/s" in out.get("fp64", {}):
            out["fp64"]["fp64_frac"] = out["fp64"]["TFLOP/s"] / out["fp64_peak_tflops"]
    print(json.dumps(out))


def batched_problems(mg, torch, n, seed=3):
    """The batched workload's first n problems: edge 3^m cells with m ~ U{3,4,5,6}
    (seed 3), log-normal eps (sigma 2, correlation length 0.1, seed 1000+i), f ~ U[-1,1]
    (seed 2000+i); grids shared per size."""
    ms = syn.batch_problem_sizes(n, seed)
    grids = {int(m): mg.Grid(2, int(m)) for m in sorted(set(ms.tolist()))}
    probs = []
    for i, m in enumerate(ms.tolist()):
        g = grids[m]
        eps = syn.lognormal_grf_eps(m, 2, sigma=2.0, seed=1000 + i)
        b = g.to_slots(m, syn.uniform_load(m, 2, 2000 + i))
        probs.append((g, m, torch.from_numpy(g.cells_to_concat({m: eps})).cuda(), torch.from_numpy(b).cuda()))
    return ms, probs


def batched_solves(mg, torch, probs, steps, flush):
    """Setup + solve to 1e-10 of all problems as one batch (mg_batch_setup +
    mg_batch_solve), mixed and FP64: median over `steps` timed batches (CUDA events)."""
    n = len(probs)
    total_dofs = sum(g.info(m).n_dofs for g, m, _, _ in probs)
    out = {}
    for prec, pers in (("mixed_bf16", 0), ("fp64", 0), ("mixed_bf16", 1), ("fp64", 1)):
        Hs = [mg.Hierarchy(g, precision=prec, persistent=pers) for g, m, _, _ in probs]
        us = [torch.zeros_like(b) for _, _, _, b in probs]
        bs = [b for _, _, _, b in probs]
        eps_list = [e for _, _, e, _ in probs]
        for H, e in zip(Hs, eps_list):
            H.setup(e)
        batch = mg.Batch(Hs)
        batch.solve(us, bs, rel_tol=1e-10, max_cycles=3000)  # warm-up (graph capture)
        times, setups = [], []
        stats, status = None, None
        for _ in range(max(1, steps)):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record()
            batch.setup(eps_list)
            e1.record()
            status, stats = batch.solve(us, bs, rel_tol=1e-10, max_cycles=3000)
            e2.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e2))
            setups.append(e0.elapsed_time(e1))
        t = statistics.median(times) / 1e3
        cyc = [st["cycles"] for st in stats]
        out[prec + ("_persistent" if pers else "")] = {"solves_per_s": n / t, "dof_per_s": total_dofs / t, "s_per_batch": t,
                     "setup_s": statistics.median(setups) / 1e3, "status": status,
                     "cycles_median": statistics.median(cyc), "cycles_max": max(cyc),
                     "max_rel_residual": max(st["rel_residual"] for st in stats)}
        del batch, Hs
        torch.cuda.empty_cache()
    out["mixed_speedup"] = out["mixed_bf16"]["solves_per_s"] / out["fp64"]["solves_per_s"]
    out["steps"] = ("lockstep: one graph-captured launch per phase and brick edge; persistent: every step "
                    "in one launch over a work queue with per-problem progress counters")
    out["problems"] = n
    out["dofs"] = total_dofs
    return out


def run_batched(args, n_problems=512, seed=3):
    """Batched workload: n independent 2D problems, edge 3^m cells with m ~ U{3,4,5,6},
    log-normal eps (sigma 2, correlation length 0.1, seed 1000+i), f ~ U[-1,1]
    (seed 2000+i), solved to 1e-10 together (mg_batch_solve): mixed vs FP64."""
    import torch

    import paper_1607_00648_gb300 as mg

    torch.cuda.set_device(0)
    n = args.batch_size or n_problems
    t0 = time.perf_counter()
    ms, probs = batched_problems(mg, torch, n, seed)
    t_inputs = time.perf_counter() - t0
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    with Clocks(0) as clk:
        res = batched_solves(mg, torch, probs, args.steps, flush)
    out = {"workload": f"batch{n}-2d", "inputs_s": t_inputs,
           "sizes": {str(3**m): int((ms == m).sum()) for m in sorted(set(ms.tolist()))}, **res,
           "clocks": clk.summary()}
    print(json.dumps(out))


def served_requests(mg, torch, n, rate, seed=4):
    """The served workload's first n requests: Poisson arrivals at `rate` per second
    (seed 4), 3D edges {27, 81, 243} cells weighted 6:3:1, log-normal eps (sigma 1.5,
    correlation length 0.1, seed 1000+i), f ~ U[-1,1] (seed 2000+i), built on the GPU."""
    arrivals, levels = syn.poisson_arrivals(n, rate, seed)
    grids = {int(L): mg.Grid(3, int(L)) for L in sorted(set(levels.tolist()))}
    reqs = []
    for i, L in enumerate(levels.tolist()):
        g = grids[L]
        inf = g.info(L)
        eps = syn.lognormal_grf_eps_torch(L, 3, sigma=1.5, seed=1000 + i)
        c = torch.from_numpy(g.tables(L)["coords"]).cuda().long()
        ok = c[:, 0] >= 0
        cat = torch.zeros(g.n_slots_total(), dtype=torch.float64, device="cuda")
        sl = torch.zeros(inf.n_slots, dtype=torch.float64, device="cuda")
        sl[ok] = eps[c[ok, 0], c[ok, 1], c[ok, 2]]
        cat[inf.slot_offset: inf.slot_offset + inf.n_slots] = sl
        gen = torch.Generator(device="cuda")
        gen.manual_seed(2000 + i)
        f = torch.rand(inf.n_slots, generator=gen, device="cuda", dtype=torch.float64) * 2 - 1
        dof = torch.from_numpy(g.dof_mask(L)).cuda()
        b = torch.where(dof, f * (3.0**-L) ** 3, torch.zeros_like(f))
        reqs.append((g, L, cat, b))
    torch.cuda.synchronize()
    return arrivals, levels, reqs


def serve_stream(mg, torch, reqs, arrivals, levels, precision, budget, tol=1e-8):
    """Submit the requests at their arrival times (scaled to the stream's rate) to an
    mg_server of the given precision; latency from submission to completion."""
    us = [torch.zeros_like(b) for _, _, _, b in reqs]
    sv = mg.Server(budget, precision=precision)
    start = time.perf_counter()
    tickets = []
    for (g, L, e, b), u, ta in zip(reqs, us, arrivals.tolist()):
        now = time.perf_counter() - start
        if ta > now:
            time.sleep(ta - now)
        tickets.append(sv.submit(g, e, b, u, rel_tol=tol, max_cycles=2000))
    res = [sv.poll(t, wait=True) for t in tickets]
    wall = time.perf_counter() - start
    sv.close()
    del us
    lat = sorted(r["latency_ms"] for r in res)
    by_edge = {}
    for L in sorted(set(levels.tolist())):
        ls = sorted(r["latency_ms"] for r, lv in zip(res, levels.tolist()) if lv == L)
        by_edge[str(3**L)] = {"n": len(ls), "p50_ms": ls[len(ls) // 2],
                              "p99_ms": ls[min(len(ls) - 1, int(0.99 * len(ls)))]}
    n = len(reqs)
    return {"solves_per_s": n / wall, "dof_per_s": sum(g.info(L).n_dofs for g, L, _, _ in reqs) / wall,
            "p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
            "max_ms": lat[-1], "wall_s": wall, "arrival_span_s": float(arrivals[-1]),
            "failed": sum(1 for r in res if r["status"] != 0),
            "max_rel_residual": max(r["rel_residual"] for r in res), "latency_by_edge": by_edge}


def served_summary(mg, torch, n, rate, budget_gb):
    """Both arms (mixed, FP64) at the offered rate, then both at a rate one GPU sustains:
    half the requests per second the mixed arm completed under the offered load."""
    budget = int(budget_gb * (1 << 30))
    arrivals, levels, reqs = served_requests(mg, torch, n, rate)
    # untimed warm-up: one request of each size through each arm (first use of the 3D
    # kernels loads their code)
    first = sorted({int(L): i for i, L in reversed(list(enumerate(levels.tolist())))}.values())
    for prec in ("mixed_bf16", "fp64"):
        serve_stream(mg, torch, [reqs[i] for i in first], np.zeros(len(first)), levels[first], prec, budget)
    out = {"requests": n, "budget_gb": budget_gb,
           "sizes": {str(3**L): int((levels == L).sum()) for L in sorted(set(levels.tolist()))}}
    offered = {}
    for prec in ("mixed_bf16", "fp64"):
        offered[prec] = serve_stream(mg, torch, reqs, arrivals, levels, prec, budget)
    out["offered"] = {"rate_per_s": rate, **offered,
                      "mixed_speedup": offered["mixed_bf16"]["solves_per_s"] / offered["fp64"]["solves_per_s"]}
    sustain = max(1.0, round(0.5 * min(offered["mixed_bf16"]["solves_per_s"], rate), 1))
    arr_s = arrivals * (rate / sustain)  # the same stream, stretched to the sustainable rate
    sus = {}
    for prec in ("mixed_bf16", "fp64"):
        sus[prec] = serve_stream(mg, torch, reqs, arr_s, levels, prec, budget)
    out["sustainable"] = {"rate_per_s": sustain,
                          "rule": "half the solves/s the mixed arm completed under the offered rate", **sus}
    return out


def run_serve(args, seed=4):
    """Served workload: Poisson arrivals (mean 200 req/s) of 3D solves with edges
    {27, 81, 243} cells (weights 6:3:1), log-normal eps (sigma 1.5, correlation length
    0.1), f ~ U[-1,1], tolerance 1e-8 each, served by mg_server with an HBM budget, mixed
    and FP64 arms; reports solves/s and p50 / p99 latency from submission, at the offered
    rate and at a rate one GPU sustains."""
    import torch

    import paper_1607_00648_gb300 as mg

    torch.cuda.set_device(0)
    with Clocks(0) as clk:
        res = served_summary(mg, torch, args.serve_requests, args.serve_rate, args.serve_budget_gb)
    print(json.dumps({"workload": f"serve{args.serve_requests}-3d", **res, "clocks": clk.summary()}))


def cpu_baseline(w, gpu_cycles, sample_cycles=15):
    """The oracle as it stands on one host core: setup + a bounded number of V-cycles of
    the full workload, extrapolated to the cycle count of the solve."""
    from oracle import multigrid
    from oracle import spacetree as stt

    L, d = w["L"], w["dim"]
    eps, bf = inputs(w)
    t0 = time.perf_counter()
    tree = stt.Spacetree(d, L)
    O = multigrid.Hierarchy(tree, {L: eps}, transfer=w["transfer"], coarse=w["coarse"])
    t_setup = time.perf_counter() - t0
    b = tree.vertices_to_slots(L, bf)
    u = np.zeros_like(b)
    t0 = time.perf_counter()
    for _ in range(sample_cycles):
        u = O.vcycle(u, b)
        np.linalg.norm(O.residual(L, u, b))
    t_cycle = (time.perf_counter() - t0) / sample_cycles
    n_dofs = int(tree.levels[L].dof.sum())
    t_solve = t_setup + gpu_cycles * t_cycle
    return {"value": n_dofs / t_solve, "unit": "DoF/s", "cores": 1, "kind": "oracle",
            "sample": f"oracle setup + {sample_cycles} V(2,2) cycles of the full workload "
                      f"({t_setup:.2f} s + {sample_cycles} x {t_cycle * 1e3:.1f} ms), extrapolated to "
                      f"{gpu_cycles} cycles", "setup_s": t_setup, "cycle_s": t_cycle}


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    from oracle import multigrid
    from oracle import spacetree as stt

    w = WORKLOADS[args.workload]
    L, d = w["L"], w["dim"]
    eps, bf = inputs(w)
    tree = stt.Spacetree(d, L)
    b = tree.vertices_to_slots(L, bf)
    n_dofs = int(tree.levels[L].dof.sum())
    # cycles to the tolerance, once (untimed): the iteration is deterministic
    O = multigrid.Hierarchy(tree, {L: eps}, transfer=w["transfer"], coarse=w["coarse"])
    _, hist = O.solve(b, w["tol"], w["max_cycles"])
    cycles = len(hist) - 1
    sample = 5
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        O = multigrid.Hierarchy(tree, {L: eps}, transfer=w["transfer"], coarse=w["coarse"])
        ts = time.perf_counter() - t0
        u = np.zeros_like(b)
        t1 = time.perf_counter()
        for _ in range(sample):
            u = O.vcycle(u, b)
            np.linalg.norm(O.residual(L, u, b))
        tc = (time.perf_counter() - t1) / sample
        if i >= args.warmup:
            times.append(ts + cycles * tc)
    t = sum(times)
    value = n_dofs * len(times) / t
    out = {"impl": "reference", "metric": "DoF/s to 1e-10 residual drop (FP64; mixed beside it)",
           "value": value, "unit": "DoF/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": t / len(times) * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "description": w["desc"], "dofs": n_dofs,
                      "cycles_per_solve": cycles},
           "cpu_baseline": {"value": value, "unit": "DoF/s", "cores": 1, "kind": "oracle",
                            "sample": f"per step: oracle setup + {sample} V(2,2) cycles, extrapolated to "
                                      f"{cycles} cycles"},
           "e2e": {"value": value, "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="checker2d-l6", choices=sorted(WORKLOADS) + sorted(ADAPTIVE))
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline leg")
    ap.add_argument("--no-ff", action="store_true",
                    help="skip the FP64 solve with float-float finest-level sweeps")
    ap.add_argument("--no-a13", action="store_true",
                    help="skip the reduced batched and served measurements of the default line")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default slab depths (no mg_autotune)")
    ap.add_argument("--precision", default="both", choices=("both", "fp64", "mixed", "bpa"),
                    help="which solve forms to time (profiling runs; the default times both; "
                         "bpa: --breakdown of the BF16 and bpa mixed forms)")
    ap.add_argument("--smoother", default="jacobi", choices=("jacobi", "block"),
                    help="smoother of the timed solves (the workloads are defined with damped Jacobi)")
    ap.add_argument("--gs-sweeps", type=int, default=1, help="block smoother: Gauss-Seidel sweeps per patch")
    ap.add_argument("--cycle", default="v", choices=("v", "additive", "bpx"),
                    help="multigrid cycle of the timed FP64 solve (additive: Alg. 2, bpx: Alg. 3; FP64 only)")
    ap.add_argument("--codecs", action="store_true",
                    help="mixed solves with BF16 deltas against the bpa codec at eps_mf 1e-2 / 1e-4 / 1e-8")
    ap.add_argument("--batched", action="store_true", help="512 uneven 2D problems solved as one batch: mixed vs FP64")
    ap.add_argument("--serve", action="store_true", help="a Poisson stream of 3D solve requests through mg_server: p50 / p99 latency")
    ap.add_argument("--serve-requests", type=int, default=300)
    ap.add_argument("--serve-budget-gb", type=float, default=64.0)
    ap.add_argument("--serve-rate", type=float, default=200.0, help="offered arrivals per second")
    ap.add_argument("--batch-size", type=int, default=0)
    ap.add_argument("--breakdown", action="store_true",
                    help="per-kernel device time of one setup + solve of the workload (torch.profiler trace)")
    ap.add_argument("--sweep-level", type=int, default=0,
                    help="time only the finest-level FP64 / FP32 sweeps on a uniform grid of this level")
    ap.add_argument("--sweep-dim", type=int, default=2, choices=(2, 3))
    ap.add_argument("--sweep-prec", default="both", choices=("both", "fp64", "fp32", "ff"),
                    help="both = fp64 + fp32 + ff (float-float finest sweeps of an FP64 hierarchy)")
    args = ap.parse_args()
    if args.precision == "bpa" and not args.breakdown:
        ap.error("--precision bpa goes with --breakdown (bench.py --codecs times the codecs)")
    if args.breakdown:
        run_breakdown(args)
    elif args.serve:
        run_serve(args)
    elif args.batched:
        run_batched(args)
    elif args.codecs:
        run_codecs(args)
    elif args.sweep_level:
        run_sweeps(args)
    elif args.workload in ADAPTIVE:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times the uniform workloads only"}))
        else:
            run_adaptive(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
