#!/usr/bin/env python
"""Throughput of the PPM+PPB sweeps: cell-updates/s per 3-D step.

Workload: the 1024^3 sphere-in-cube (n=3 polytrope under central gravity,
heating shell, damping zones, light-fluid layer at r=0.6R, rms Mach 0.03),
advanced by Strang double steps (X Y Z [sources] Z Y X [sources]) in the FP32
base-state-deviation form, in place on one 9 x 1024^3 FP32 state (~39 GB),
dt from the CFL maximum fused into each step's last pass.  The FP64 plain
form runs on the same grid for comparison.

One "step" = one double step = two 3-D steps; value = 2 * cells * steps /
time.  Inputs (39 GB) are far larger than L2 (129 MB), so no flush is needed
between timed steps.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the reference arm of this
program) on the host cores on a bounded sample of the same workload.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per 3-D step"
UNIT = "cell-updates/s"
BYTES_PER_CELL_PASS = {"f32": 72, "f64": 144}   # 9 values read + written per pass
SWEEP_SRC = os.path.join(ROOT, "paper_1810_13416_gb300", "csrc", "sweep.cuh")
TILE_SRC = os.path.join(ROOT, "paper_1810_13416_gb300", "csrc", "tile.cuh")
TRAFFIC_JSON = os.path.join(ROOT, "profiles", "sweep_traffic.json")
FP32_LANES_PER_SM = 128


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


def _src_hash() -> str:
    """Hash of the FP32 passes as compiled: the sources of both designs and
    their nvcc flags."""
    import importlib
    _b = importlib.import_module("paper_1810_13416_gb300.build")
    src = b""
    for path in (SWEEP_SRC, TILE_SRC):
        with open(path, "rb") as f:
            src += f.read()
    flags = repr((_b.UNIT_FLAGS.get("sweep_f32"), _b.UNIT_FLAGS.get("tile_f32")))
    return hashlib.sha256(src + flags.encode()).hexdigest()[:16]


def _traffic_per_cell(prec: str, designs):
    """DRAM bytes per cell and pass of the pass kernels the step runs (design
    per axis), averaged over the six passes of a double step (two x passes,
    four y/z passes), from the committed ncu summary; None when absent or
    taken on another kernel source."""
    try:
        with open(TRAFFIC_JSON) as f:
            d = json.load(f)
        e = d[prec]
        if e.get("src_sha256_16") != _src_hash():
            return None
        name = lambda dd: "tile" if dd == 1 else "march"
        bx = float(e["dram_bytes_per_cell_pass"][name(designs[0])]["x"])
        by = float(e["dram_bytes_per_cell_pass"][name(designs[1])]["yz"])
        bz = float(e["dram_bytes_per_cell_pass"][name(designs[2])]["yz"])
        return (2.0 * bx + 2.0 * by + 2.0 * bz) / 6.0
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "100", "-i", str(self.index)],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.p is None:
            return
        time.sleep(0.25)
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out = ""
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                self.rows.append(f)

    def summary(self):
        rows = getattr(self, "rows", [])
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def shard(n_items: int, rank: int, world: int):
    """Independent units (ensemble boxes) owned by one rank: round robin, no
    data-path communication between ranks."""
    return [i for i in range(n_items) if i % world == rank]


def reduce_max(x: float, dist=None, device="cpu") -> float:
    """Slowest rank's time: the job's time."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job rate: units of all ranks over the slowest rank's time."""
    return units_per_rank * world / seconds


def _upload(ctx, p, torch, slab=64):
    import workloads
    nz = p.shape[2]
    for z0 in range(0, nz, slab):
        z1 = min(nz, z0 + slab)
        qs = [t.contiguous() for t in workloads.initial_state(p, device="cuda", z_lo=z0, z_hi=z1)]
        # ten-value PPB: second and mixed moments start at zero
        qs += [torch.zeros_like(qs[0]) for _ in range(ctx.nvar - len(qs))]
        ctx.set_region((0, 0, z0), (p.shape[0], p.shape[1], z1), qs, device=True)
        del qs
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def _cpu_baseline(n_cpu: int, steps: int, warmup: int):
    """The oracle as it stands, on the host cores, on an n_cpu^3 sample of
    the same sphere recipe."""
    import oracle
    import workloads
    oracle.build()
    threads = os.cpu_count() or 1
    oracle.Oracle.set_threads(threads)
    p = workloads.sphere(n=n_cpu)
    q = workloads.build(p)
    o = oracle.Oracle(p)
    for _ in range(warmup):
        o.double_step(q, o.cfl_dt(q, p.cfl))
    t0 = time.perf_counter()
    for _ in range(steps):
        o.double_step(q, o.cfl_dt(q, p.cfl))
    t = time.perf_counter() - t0
    return {"value": 2.0 * p.ncell * steps / t, "unit": UNIT, "cores": oracle.Oracle.threads(),
            "kind": "oracle", "sample": f"sphere recipe at {n_cpu}^3, {steps} double steps after {warmup} warm-up",
            "seconds": t}


def _cpu_single_thread(n_cpu: int):
    """The oracle on one host core, one double step of an n_cpu^3 sample of
    the same recipe after one warm-up."""
    import oracle
    import workloads
    before = oracle.Oracle.threads()
    oracle.Oracle.set_threads(1)
    try:
        p = workloads.sphere(n=n_cpu)
        q = workloads.build(p)
        o = oracle.Oracle(p)
        o.double_step(q, o.cfl_dt(q, p.cfl))
        t0 = time.perf_counter()
        o.double_step(q, o.cfl_dt(q, p.cfl))
        t = time.perf_counter() - t0
    finally:
        oracle.Oracle.set_threads(before)
    return {"value": 2.0 * p.ncell / t, "unit": UNIT, "cores": 1,
            "sample": f"sphere recipe at {n_cpu}^3, 1 double step after 1 warm-up"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    cb = _cpu_baseline(args.cpu_n, args.steps, args.warmup)
    t_step = cb["seconds"] / args.steps
    line = {"metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"sphere-in-cube {args.cpu_n}^3 sample of the 1024^3 sphere (oracle, host cores)",
                       "cells": args.cpu_n ** 3, "precision": "FP64 CPU oracle"},
            "cpu_baseline": {k: cb[k] for k in ("kind", "cores", "sample", "value", "unit")},
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _time_steps(ctx, torch, stream, steps, pass_ms=None):
    """Device time of `steps` double steps (CUDA events on the library's
    stream).  With pass_ms (a list), each step's six pass durations, from the
    events the library records inside its step graph, are appended to it; the
    host then waits for each step before queueing the next (the waits are
    inside the timed region)."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ctx.step(0.0)
        if pass_ms is not None:
            pass_ms.append(ctx.pass_times())
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) * 1e-3


def run_ours(args):
    import numpy as np
    import torch
    import paper_1810_13416_gb300 as ppm
    import workloads

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    ppm.build()
    hbm_peak, sm_max_mhz, peak_src = _peaks()
    n = args.n
    p = workloads.sphere(n=n)
    ncell = p.ncell
    stream = torch.cuda.Stream()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    def max_over_ranks(x):
        return reduce_max(x, dist, "cuda")

    # ---------------- FP32 deviation form: the headline -----------------
    ctx = ppm.Context.from_problem(p, precision=ppm.FP32_DEVIATION, stream=stream, device=local)
    if args.design == "tile":
        ctx.set_pass_design(ppm.PASS_TILE)
    _upload(ctx, p, torch)
    tune_info = None
    if args.design == "auto":
        # the autotuner picks the pass design per axis on this state (or from
        # its cache); outside the timed region
        cache = os.environ.get("PPM_AUTOTUNE_CACHE", os.path.join(tempfile.gettempdir(), "ppm_autotune.txt"))
        t_tune = time.perf_counter()
        from_cache = ctx.tune(cache)
        tune_info = {"designs_xyz": ["tile" if d == ppm.PASS_TILE else "march" for d in ctx.pass_designs],
                     "from_cache": from_cache, "tune_s": time.perf_counter() - t_tune}
    ctx.cfl_dt(p.cfl, fetch=False)
    # evolve the state first, so that the timed steps see a realistic mix of
    # the data-dependent branches (constraints, limiters, wave directions)
    for _ in range(args.pre_evolve):
        ctx.step(0.0)
    host_q = None
    if not args.no_e2e:
        # pinned host copy of the evolved state for the end-to-end leg
        host_q = [torch.empty((p.shape[2], p.shape[1], p.shape[0]), dtype=torch.float64, pin_memory=True)
                  for _ in range(9)]
        ctx.get_state_into([t.numpy() for t in host_q])
        ctx.cfl_dt(p.cfl, fetch=False)
    for _ in range(args.warmup):
        ctx.step(0.0)
    barrier()
    l0 = ctx.launch_count
    pass_rec = []
    with Clocks(local) as clk:
        t = _time_steps(ctx, torch, stream, args.steps, pass_rec)
    launches = ctx.launch_count - l0
    t = max_over_ranks(t)
    ctx.sync()
    pr = np.array(pass_rec)                      # steps x 6 (X Y Z Z Y X), ms
    ctx_designs = ctx.pass_designs
    tot, _, mach = ctx.diagnostics()
    ok_state = bool(np.isfinite(tot).all()) and 0.0 < mach < 1.0
    value = job_throughput(2.0 * ncell * args.steps, ws, t)
    ms = 1e3 * t / args.steps
    # dominant kernel: the fused pass (6 of the 7 launches of a step; the
    # 7th is a one-thread dt kernel).  Its average launch duration comes from
    # the events recorded between the passes inside every timed step.
    pass_s = float(pr.mean()) * 1e-3
    achieved = BYTES_PER_CELL_PASS["f32"] * ncell / pass_s / 1e9
    tr = _traffic_per_cell("f32", ctx.pass_designs)
    flops_cell = args.flops_per_cell
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    alu_peak = n_sm * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12
    alu_achieved = flops_cell * ncell / pass_s / 1e12
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak,
                "traffic": (tr * ncell if tr is not None else None),
                "kernel": "fused PPM+PPB pass, per axis: " + ", ".join(
                    f"{ax}: " + ("ppm::tile::tile_pass_kernel<AX,FULL> (cell-parallel tiles, TMA)" if d == ppm.PASS_TILE
                                 else "ppm::sweep_kernel<float,0,VEC,0,0,0,128,0,NSRC> (register-window march)")
                    for ax, d in zip("xyz", ctx_designs)),
                "tuned": tune_info,
                "algorithmic_bytes_per_launch": BYTES_PER_CELL_PASS["f32"] * ncell,
                "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_src})",
                "pass_ms": {"avg_in_step": 1e3 * pass_s, "x": float(pr[:, [0, 5]].mean()),
                            "y": float(pr[:, [1, 4]].mean()), "z": float(pr[:, [2, 3]].mean()),
                            "step_over_6": 1e3 * t / args.steps / 6.0,
                            "how": "CUDA events recorded inside the step graph between its six passes, "
                                   "every timed step"},
                "alu": {"flops_per_cell_pass": flops_cell, "achieved_tflops": alu_achieved,
                        "peak_tflops": alu_peak, "frac": alu_achieved / alu_peak,
                        "peak_source": f"{n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max_mhz:.0f} MHz "
                                       f"(unit counts and the maximum SM clock)"}}
    clocks = clk.summary()

    # ---------------- end to end through the C ABI with host buffers -----
    e2e = None
    if host_q is not None:
        hq = [t_.numpy() for t_ in host_q]
        barrier()
        t0 = time.perf_counter()
        ctx.set_state(hq)                       # H2D of the initial state
        dt = ctx.cfl_dt(p.cfl)                  # D2H of dt
        for _ in range(args.steps):
            ctx.step(dt)
            ctx.diagnostics()                   # D2H of the conserved totals and max Mach
            dt = ctx.cfl_dt(p.cfl)
        ctx.get_state_into(hq)                  # D2H of the final state
        te = max_over_ranks(time.perf_counter() - t0)
        state_bytes = 9 * 8 * ncell
        e2e = {"value": 2.0 * ncell * args.steps * ws / te, "unit": UNIT,
               "h2d_bytes_per_step": int(state_bytes / args.steps) + 8,
               "d2h_bytes_per_step": int(state_bytes / args.steps) + 8 * 8 + 2 * 8,
               "includes": "set_state(host pinned FP64) + per step: cfl_dt->host, step, diagnostics->host; "
                           "get_state(host pinned FP64)"}
        del hq
        host_q = None
    ctx.close()
    del ctx
    torch.cuda.empty_cache()

    # ---------------- FP64 plain form on the same grid -------------------
    fp64 = None
    if not args.no_fp64:
        c64 = ppm.Context.from_problem(p, precision=ppm.FP64_PLAIN, stream=stream, device=local)
        _upload(c64, p, torch)
        c64.cfl_dt(p.cfl, fetch=False)
        c64.step(0.0)
        barrier()
        t64 = max_over_ranks(_time_steps(c64, torch, stream, args.fp64_steps))
        v64 = 2.0 * ncell * args.fp64_steps * ws / t64
        fp64 = {"value": v64, "unit": UNIT, "ms_per_step": 1e3 * t64 / args.fp64_steps,
                "steps": args.fp64_steps, "fp32_over_fp64": value / v64,
                "achieved_gbs": BYTES_PER_CELL_PASS["f64"] * ncell / (t64 / args.fp64_steps / 6.0) / 1e9}
        c64.close()
        del c64
        torch.cuda.empty_cache()

    # ---------------- confining sphere (FP32, same grid) ------------------
    conf = None
    if not args.no_confined:
        pc = workloads.sphere(n=n, confine=True)
        cc = ppm.Context.from_problem(pc, precision=ppm.FP32_DEVIATION, stream=stream, device=local)
        _upload(cc, pc, torch)
        cc.cfl_dt(pc.cfl, fetch=False)
        for _ in range(args.warmup):
            cc.step(0.0)
        barrier()
        tc = max_over_ranks(_time_steps(cc, torch, stream, args.confined_steps))
        nflu = math.pi / 6.0 * n ** 3   # fluid cells ~ volume of the inscribed sphere
        conf = {"workload": f"star confined in the sphere inscribed in the {n}^3 cube, gravity tapered "
                            f"to zero inside it, FP32", "cells": ncell,
                "value": 2.0 * ncell * args.confined_steps * ws / tc, "unit": UNIT,
                "fluid_cell_updates_per_s": 2.0 * nflu * args.confined_steps * ws / tc,
                "ms_per_step": 1e3 * tc / args.confined_steps, "steps": args.confined_steps}
        cc.close()
        del cc
        torch.cuda.empty_cache()

    # ---------------- ten-value PPB (FP32, same grid) ---------------------
    ten = None
    if not args.no_ppb10:
        import copy as _copy
        pt = _copy.copy(p)
        pt.nmom = 9
        ct = ppm.Context.from_problem(pt, precision=ppm.FP32_DEVIATION, stream=stream, device=local)
        _upload(ct, pt, torch)
        ct.cfl_dt(pt.cfl, fetch=False)
        for _ in range(args.warmup):
            ct.step(0.0)
        barrier()
        tt = max_over_ranks(_time_steps(ct, torch, stream, args.ppb10_steps))
        ten = {"workload": f"sphere-in-cube {n}^3, FP32, FV with 9 moments (15 values per cell)",
               "cells": ncell, "value": 2.0 * ncell * args.ppb10_steps * ws / tt, "unit": UNIT,
               "ms_per_step": 1e3 * tt / args.ppb10_steps, "steps": args.ppb10_steps,
               "algorithmic_bytes_per_cell_pass": 120}
        ct.close()
        del ct
        torch.cuda.empty_cache()

    # ---------------- 3-D shock dissipation on (FP32, same grid) -----------
    shock = None
    if not args.no_shock:
        import copy as _copy
        ps = _copy.copy(p)
        ps.shock_k = 0.1
        cs = ppm.Context.from_problem(ps, precision=ppm.FP32_DEVIATION, stream=stream, device=local)
        _upload(cs, ps, torch)
        cs.cfl_dt(ps.cfl, fetch=False)
        for _ in range(args.warmup):
            cs.step(0.0)
        barrier()
        l0s = cs.launch_count
        tsk = max_over_ranks(_time_steps(cs, torch, stream, args.shock_steps))
        shock = {"workload": f"sphere-in-cube {n}^3, FP32, 3-D shock dissipation on (K = 0.1; inactive in "
                             f"this Mach-0.03 flow: the cost of the divergence pass and the dissipative "
                             f"flux terms)", "cells": ncell,
                 "value": 2.0 * ncell * args.shock_steps * ws / tsk, "unit": UNIT,
                 "ms_per_step": 1e3 * tsk / args.shock_steps, "steps": args.shock_steps,
                 "launches_per_step": (cs.launch_count - l0s) / args.shock_steps}
        cs.close()
        del cs
        torch.cuda.empty_cache()

    # ---------------- batched ensemble of uneven boxes (FP32) -------------
    ens_out = None
    if not args.no_ensemble:
        boxes = workloads.ensemble_boxes(nbox=args.ens_boxes)
        mine = [boxes[i] for i in shard(len(boxes), rank, ws)]   # independent boxes shard over ranks
        ens = ppm.Ensemble(mine, precision=ppm.FP32_DEVIATION, stream=stream, device=local)
        for i, bp in enumerate(mine):
            qs = workloads.initial_state(bp, device="cuda")
            ens.set_region(i, (0, 0, 0), bp.shape, [t.contiguous() for t in qs], device=True)
            del qs
        torch.cuda.synchronize()
        cache = os.environ.get("PPM_AUTOTUNE_CACHE",
                               os.path.join(tempfile.gettempdir(), "ppm_autotune.txt"))
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        t_tune = time.perf_counter()
        from_cache = ens.tune(cache)
        t_tune = time.perf_counter() - t_tune
        ens.cfl_dt(0.7, fetch=False)
        for _ in range(args.warmup):
            ens.step(0.0)
        barrier()
        l0 = ens.launch_count
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            ens.step(0.0)
        e1.record(stream)
        e1.synchronize()
        te = max_over_ranks(e0.elapsed_time(e1) * 1e-3)
        ens.sync()
        cells = sum(b.ncell for b in boxes)
        mode = "one launch per double step" if ens.launch_mode == ppm.ENS_ONE_LAUNCH else "one launch per pass"
        ens_out = {"workload": f"{len(boxes)} stratified boxes, extents 48..192 (seeded), FP32",
                   "launch_mode": mode + " (tuned)",
                   "cells": cells, "value": 2.0 * cells * args.steps / te, "unit": UNIT,
                   "ms_per_step": 1e3 * te / args.steps, "scaling": "strong (boxes shared over ranks)",
                   "launches_per_step": (ens.launch_count - l0) / args.steps,
                   "tuned": ens.config(), "tune_from_cache": from_cache, "tune_s": t_tune}
        ens.close()
        del ens
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and not args.no_cpu:
        cb = _cpu_baseline(args.cpu_n, args.cpu_steps, 1)
        cpu = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
        cpu["single_thread"] = _cpu_single_thread(128)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"sphere-in-cube {n}^3, FP32 base-state-deviation form, in place",
                           "cells": ncell, "state_bytes": 9 * 4 * ncell, "cfl": p.cfl,
                           "step": "Strang double step X Y Z [src] Z Y X [src] = 2 3-D steps",
                           "pre_evolved_double_steps": args.pre_evolve,
                           "l2": f"inputs larger than L2 ({9 * 4 * ncell / 1e9:.2f} GB vs 129 MB); no flush"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clocks, "fp64": fp64, "confined": conf, "ppb10": ten, "shock": shock, "ensemble": ens_out,
                "state_ok": ok_state}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--cpu-n", type=int, default=256,
                    help="edge of the sphere sample the oracle runs for the CPU baseline")
    ap.add_argument("--cpu-steps", type=int, default=6,
                    help="timed oracle double steps of the CPU baseline (about 10 s on 16 cores)")
    ap.add_argument("--flops-per-cell", type=float, default=464.0,
                    help="algorithmic FP32 flops per cell and pass (oracle census)")
    ap.add_argument("--pre-evolve", type=int, default=20,
                    help="double steps taken before the warm-up (not timed)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-confined", action="store_true")
    ap.add_argument("--no-ppb10", action="store_true")
    ap.add_argument("--ppb10-steps", type=int, default=3)
    ap.add_argument("--confined-steps", type=int, default=3)
    ap.add_argument("--no-shock", action="store_true")
    ap.add_argument("--shock-steps", type=int, default=3)
    ap.add_argument("--ens-boxes", type=int, default=24)
    ap.add_argument("--design", default="auto", choices=["auto", "march", "tile"],
                    help="form of the FP32 pass kernel for the headline (auto: the autotuner's choice per axis)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
