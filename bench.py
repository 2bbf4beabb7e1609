#!/usr/bin/env python
"""Benchmark of the shell pressure-correction Poisson solve on one GB300 (or N replicas).

A step is one whole solve from a cold start (x = 0) to 1e-10 relative
residual of the 128 x 128 x 256 tanh-stretched sphere workload (RHS on the
device, hierarchy set up before timing), with L2 flushed (256 MB write)
before every step.  Prints one JSON line (rank 0).

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

``--impl reference`` times the FP64 CPU oracle on the host cores instead
(a bounded sample of the same workload per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fine-grid DOF/s to 1e-10 rel. residual, FP32-refined vs FP64 MG; HBM GB/s; p99 ms"
UNIT = "DOF/s"
PREC = {"fp64": 0, "fp32": 1, "fp16": 2}
SMOOTHER = {"gs": 0, "jacobi": 1, "line": 2, "xline": 3, "alt": 4, "plane": 5}
PREC_NAME = {0: "plain FP64 multigrid", 1: "FP32 V-cycles inside FP64 refinement",
             2: "FP16-coefficient FP32 V-cycles inside FP64 refinement"}
L2_FLUSH_BYTES = 256 << 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="single_sphere_128")
    p.add_argument("--scale", type=int, default=1, help="single workloads: shrink every dimension by this factor "
                                                         "(small cases for profiling; not a bench line)")
    p.add_argument("--precision", default="fp32", choices=list(PREC))
    p.add_argument("--tol", type=float, default=1e-10)
    p.add_argument("--smoother", default="gs", choices=list(SMOOTHER),
                   help="gs: multicolour Gauss-Seidel; jacobi; line: radial-line Gauss-Seidel; "
                        "xline: longitude-line Gauss-Seidel; alt: radial then longitude lines; "
                        "plane: semi-coarsening multigrid with zebra plane relaxation, V(1,1)")
    p.add_argument("--no-compare", action="store_true", help="skip the plain FP64 multigrid leg")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-c3", action="store_true", help="skip the 256 x 256 x 512 oblate-shell leg")
    p.add_argument("--requests", type=int, default=200, help="serve_stream: requests per offered rate")
    p.add_argument("--rates", default="50,100,200,500,1000,2000",
                   help="serve_stream: Poisson arrival rates (1/s), comma separated")
    return p.parse_args()


# ----------------------------------------------------------------- peaks / profiles
def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


BATCH_SOURCES = ("batch.cu", "mg_internal.cuh", "mg_kernels.h", "line_smooth.cuh", "xline_smooth.cuh",
                 "plane_smooth.cuh")
SWEEP_SOURCES = ("sweep.cu", "mg_internal.cuh", "mg_kernels.h")


def kernel_source_hash(sources=BATCH_SOURCES):
    """Hash of the source files a kernel is built from (the batched level
    kernels by default; the one-pass sweeps: SWEEP_SOURCES)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2305_17875_gb300", "csrc")
    for fn in sources:
        with open(os.path.join(csrc, fn), "rb") as fh:
            h.update(fn.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(workload, precision, slot, one_pass=False):
    """DRAM bytes per launch of the slot's kernel from the committed ncu
    summary, or None when absent or taken on different kernel sources.  The
    level-0 smoother's entry is that of the colour passes, or with one_pass
    that of the one-pass sweep (key suffix /sweep)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    suffix = "/sweep" if (one_pass and slot == "smooth0") else ""
    e = d.get(f"{workload}/{precision}/{slot}{suffix}")
    scale = 1.0
    if not e:
        # a workload too large to capture: its half-size capture (every
        # dimension halved, the same kernels), scaled by the cell count, since
        # a level kernel's traffic per cell does not depend on the grid size
        e = d.get(f"{workload}/2/{precision}/{slot}{suffix}")
        scale = 8.0
    if not e or e.get("source_hash") != kernel_source_hash(tuple(e.get("sources", BATCH_SOURCES))):
        return None
    return e.get("dram_bytes_per_launch") * scale


def coef_components(stencil, axi):
    """Metric arrays the operator stores: 3 for 7 points, 9 for 19 points, 5
    for 19 points on an axisymmetric mapping (the longitude cross terms
    vanish there and are not stored)."""
    return (5 if axi else 9) if stencil == 19 else 3


def sweep_bytes_per_cell(stencil, prec, smoother=0, axi=False, ncomp=None):
    """Minimum HBM bytes of one whole smoothing sweep (all colours) per cell:
    x read and written, b read, every stored coefficient array read once;
    line smoothers add their factor arrays (radial 3, longitude 4 values per
    cell; the alternating smoother's sweeps are radial and longitude in
    turn: their mean)."""
    vb = 8 if prec == 0 else 4
    cb = {0: 8, 1: 4, 2: 2}[prec]
    nc = coef_components(stencil, axi) if ncomp is None else ncomp
    base = 3 * vb + nc * cb
    fac = {2: 3 * vb, 3: 4 * vb, 4: 3.5 * vb}.get(smoother, 0.0)
    return base + fac


def algorithmic_bytes(slot, stencil, prec, n_fine, n_next, smoother=0, axi=False, passes_per_sweep=None,
                      ncomp=None):
    """Minimum HBM bytes one launch of the slot's kernel must move: each array
    it needs read or written once, neighbour re-reads served on chip.  A
    colour pass is charged 1/C of a whole sweep (C = 2 colours for 7 points, 4
    for 19 points); a one-pass sweep (all colours in one launch,
    passes_per_sweep = 1) the whole sweep.  ncomp overrides the stored
    coefficient count (9 for 19 points: every component of the general
    mapping, the model the 19-point byte counts were first planned on)."""
    vb = 8 if prec == 0 else 4
    cb = {0: 8, 1: 4, 2: 2}[prec]
    nc = coef_components(stencil, axi) if ncomp is None else ncomp
    N = float(n_fine)
    if slot == "smooth0":
        ncol = 4 if stencil == 19 else 2
        if smoother == 1:
            ncol = 1                        # weighted Jacobi: one pass per sweep
        per = ncol if passes_per_sweep is None else passes_per_sweep
        return sweep_bytes_per_cell(stencil, prec, smoother, axi, nc) * N / per
    if slot == "residual":
        # x64, b64, the FP64 face coefficients; in FP32 / FP16 cycles the
        # FP32 residual out and the fine FP32 correction cleared for the next
        # cycle
        return N * (8 + 8 + 8 * nc + (0 if prec == 0 else 8))
    if slot == "restrict0":
        # x, b, coefficients of every fine cell; the coarse right side out
        return N * (2 * vb + nc * cb) + vb * n_next
    if slot == "prolong0":
        return 2 * vb * N + vb * n_next
    if slot == "update":
        return 20 * N                       # e32 read, x64 read and written
    return float("nan")                     # many small launches; no single per-launch count


# ----------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- CPU oracle leg
def _oracle_solve_job(args):
    """Runs in a spawned process with single-threaded BLAS: one oracle solve of
    the sample grid; returns (cells, seconds of the solve, iterations)."""
    g, tol, kind = args
    import numpy as np
    import workloads as W
    from oracle import mg as omg
    f = W.rhs_modes(g, seed=0)
    hier, fm = omg.setup(g, 7 if g["mapping"] == 0 else 19)
    t0 = time.perf_counter()
    x, info = omg.solve(g, f.ravel(), tol=tol, hier=hier, fm=fm, max_iters=200, kind=kind)
    dt = time.perf_counter() - t0
    return g["nr"] * g["nth"] * g["nph"], dt, info["iters"]


def sample_grid(g, factor=2):
    s = dict(g)
    s.update(nr=g["nr"] // factor, nth=g["nth"] // factor, nph=g["nph"] // factor)
    return s


def cpu_baseline(g, tol, repeats=1, kind=0, all_cores=False):
    """The oracle on the host: one single-threaded process (the baseline line),
    or, with all_cores, one such process per core solving the same sample at
    once (throughput of the whole host: cells of all solves / the median
    solve time)."""
    env_keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    old = {k: os.environ.get(k) for k in env_keys}
    for k in env_keys:
        os.environ[k] = "1"
    ncores = max(1, os.cpu_count() or 1) if all_cores else 1
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(ncores) as pool:
            res = pool.map(_oracle_solve_job, [(sample_grid(g), tol, kind)] * (ncores if all_cores else repeats))
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    cells, dts, iters = zip(*res)
    dt = statistics.median(dts)
    s = sample_grid(g)
    if all_cores:
        return {"value": ncores * cells[0] / dt, "unit": UNIT, "cores": ncores, "kind": "oracle",
                "sample": (f"{ncores} single-threaded oracle processes at once, each solving the "
                           f"{s['nr']}x{s['nth']}x{s['nph']} sample to {tol:g} (setup excluded; "
                           f"median solve {dt:.1f} s)")}
    return {"value": cells[0] / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"oracle FP64 multigrid (numpy/scipy, 1 thread) solving the same workload "
                       f"at {s['nr']}x{s['nth']}x{s['nph']} (1/8 of the cells) to {tol:g}, "
                       f"setup excluded: {iters[0]} V-cycles in {dt:.1f} s")}


# ----------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    import workloads as W
    if rank != 0:
        return
    if args.workload not in W.SINGLE:
        print(json.dumps({"impl": "reference", "unavailable": f"the oracle arm times single solves only; "
                                                              f"{args.workload} is not one"}), flush=True)
        return
    w = W.single(args.workload)
    g = w["grid"]
    ctx = mp.get_context("spawn")
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    s = sample_grid(g)
    with ctx.Pool(1) as pool:
        for _ in range(args.warmup):
            pool.map(_oracle_solve_job, [(s, args.tol, SMOOTHER[args.smoother])])
        t0 = time.perf_counter()
        res = [pool.map(_oracle_solve_job, [(s, args.tol, SMOOTHER[args.smoother])])[0] for _ in range(args.steps)]
        wall = time.perf_counter() - t0
    cells = res[0][0]
    ms = [r[1] * 1e3 for r in res]
    value = cells / (statistics.mean(ms) / 1e3)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(ms),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_of(args, g, None, None),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"oracle FP64 multigrid, 1 thread, same workload at "
                                   f"{s['nr']}x{s['nth']}x{s['nph']} to {args.tol:g} per step, "
                                   f"setup excluded"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": wall,
    }
    print(json.dumps(line), flush=True)


def config_of(args, g, rep, stencil):
    name = args.workload if getattr(args, "scale", 1) == 1 else f"{args.workload}/{args.scale}"
    c = {"workload": name, "grid": f"{g['nr']}x{g['nth']}x{g['nph']}",
         "mapping": ["sphere", "oblate", "triaxial"][g["mapping"]], "stretch": g["stretch"],
         "flattening": g["flattening"], "tol": args.tol, "precision": PREC_NAME[PREC[args.precision]],
         "l2": "flushed (256 MB write) before every step", "parallelism": f"replicas x{args.gpus}",
         "smoother": getattr(args, "smoother", "gs")}
    if rep is not None:
        c.update(stencil=stencil, levels=rep["levels"], iters=rep["iters"])
    return c


# ----------------------------------------------------------------- ranks
def sync_ranks():
    """Barrier across the ranks of a distributed run (no-op otherwise)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def max_over_ranks(value):
    """The largest value over the job's ranks after a barrier (the job is as
    slow as its slowest rank); the value itself when not distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.barrier()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------- our arm
def time_solves(mgs, h, fd, xd, steps, flush, torch):
    ms, reps = [], []
    for _ in range(steps):
        xd.zero_()
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        rep = mgs.mg_solve(h, fd, xd, tol=TOL)
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        reps.append(rep)
    return ms, reps


TOL = 1e-10
SLOT_NAMES = (("smooth0", 0), ("residual", 1), ("restrict0", 2), ("prolong0", 3), ("update", 4), ("tail", 5),
              ("other", 6))


def profile_solves(mgs, h, fd, xd, steps, flush, torch, stencil, prec, N, n_next, smoother, axi, one_pass):
    """A separate profiled run of the same solves (every launch records its
    own start and end on the GPU's global timer; the launches run as in the
    headline): device time per slot and per level, and the roofline of the
    level-0 kernel with the largest device time."""
    mgs.mg_profile_enable(h, True)
    ms, _ = time_solves(mgs, h, fd, xd, steps, flush, torch)
    slots = {name: mgs.mg_profile_read(h, slot) for name, slot in SLOT_NAMES}
    levels = {}
    for l in range(1, mgs.PROF_SLOTS - mgs.PROF_LEVEL_BASE):
        t, n = mgs.mg_profile_read(h, mgs.PROF_LEVEL_BASE + l)
        if n:
            levels[l] = {"ms_per_solve": t / steps, "launches_per_solve": n / steps}
    gap_ms, _ = mgs.mg_profile_read(h, mgs.PROF_GAPS)
    # cross-check of the clocks: the same solves with CUDA events around
    # every launch (eager launches, host loop: the events break the launches'
    # overlap, so these spans include some launch latency)
    mgs.mg_profile_enable(h, 2)
    ev_steps = max(2, min(steps, 3))
    ev_ms, _ = time_solves(mgs, h, fd, xd, ev_steps, flush, torch)
    ev_slots = {name: mgs.mg_profile_read(h, slot) for name, slot in SLOT_NAMES}
    mgs.mg_profile_enable(h, False)
    kernels = {}
    for k, (t, n) in slots.items():
        avg = t / max(n, 1)
        ab = algorithmic_bytes(k, stencil, prec, N, n_next, smoother, axi,
                               passes_per_sweep=1 if (k == "smooth0" and one_pass) else None)
        kernels[k] = {"ms_per_solve": t / steps, "launches_per_solve": n / steps, "avg_ms": avg if n else None,
                      "alg_GBps": ab / (avg * 1e-3) / 1e9 if n and ab == ab else None}
    attributed = sum(v["ms_per_solve"] for v in kernels.values()) + sum(v["ms_per_solve"] for v in levels.values())
    live = statistics.mean(ms)
    # device time no kernel covers, within a program run (an outer
    # iteration, the prologue, the epilogue): launch latency between kernels
    gaps = gap_ms / steps
    events = {k: {"ms_per_solve": t / ev_steps, "avg_ms": t / n if n else None} for k, (t, n) in ev_slots.items()}
    return {"profiled_ms_per_solve": live, "attributed_ms_per_solve": attributed,
            "launch_gaps_ms_per_solve": gaps,
            "events_ms_per_solve": statistics.mean(ev_ms), "events": events,
            # the rest: between program runs (stop tests, copies, host calls)
            "between_programs_ms_per_solve": live - attributed - gaps,
            "kernels": kernels, "levels": levels}, slots


def add_event_check(roof, prof, name):
    """The kernel's mean launch time from the CUDA-event pass beside the
    clocks' (same bytes, the events' duration)."""
    ev = prof["events"].get(name, {}).get("avg_ms")
    if ev:
        roof["avg_launch_ms_events"] = ev
        roof["frac_events"] = roof["algorithmic_bytes_per_launch"] / (ev * 1e-3) / 1e9 / roof["peak"]


def roofline_of(name, slots, steps, stencil, prec, N, n_next, smoother, axi, one_pass, traffic):
    tot_ms, nl = slots[name]
    per_launch_ms = tot_ms / max(nl, 1)
    pps = 1 if (name == "smooth0" and one_pass) else None
    abytes = algorithmic_bytes(name, stencil, prec, N, n_next, smoother, axi, passes_per_sweep=pps)
    peak, peak_kind = peaks()
    achieved = abytes / (per_launch_ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": peak_kind, "traffic": traffic,
            "algorithmic_bytes_per_launch": abytes, "avg_launch_ms": per_launch_ms,
            "cells": N, "sweep_bytes_per_cell": sweep_bytes_per_cell(stencil, prec, smoother, axi)
            if name == "smooth0" else None,
            "launches_per_sweep": (1 if one_pass else (1 if smoother == 1 else (4 if stencil == 19 else 2)))
            if name == "smooth0" else None}
    if stencil == 19 and axi:
        # the same bytes with all nine coefficient arrays of the general mapping
        sb = algorithmic_bytes(name, stencil, prec, N, n_next, smoother, axi, passes_per_sweep=pps, ncomp=9)
        roof["frac_nine_component_model"] = sb / (per_launch_ms * 1e-3) / 1e9 / peak
    return roof


def single_leg(args, mgs, torch, workload, scale, prec, smoother, steps, warmup, flush, traffic_key=None):
    """Set-up, warm-up and `steps` timed solves (profiling off) of one single
    workload, then a profiled run of the same solves for the kernel
    breakdown.  Returns the leg's record, the handle and its device buffers."""
    import workloads as W
    w = W.single(workload, scale)
    g, f = w["grid"], w["f"]
    N = g["nr"] * g["nth"] * g["nph"]
    sopts = dict(precision=prec, smoother=smoother)
    if "max_levels" in w:
        sopts["max_levels"] = w["max_levels"]
    if "max_iters" in w:
        sopts["max_iters"] = w["max_iters"]
    if w.get("coarsen") == "full":
        sopts["coarsen"] = 1
    t_setup = time.perf_counter()
    h = mgs.mg_setup(g, sopts)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    fd = torch.from_numpy(f).cuda()
    xd = torch.zeros_like(fd)
    for _ in range(warmup):
        xd.zero_()
        mgs.mg_solve(h, fd, xd, tol=TOL)
    torch.cuda.synchronize()
    ms, reps = time_solves(mgs, h, fd, xd, steps, flush, torch)
    rep = reps[-1]
    info0 = mgs.mg_get_level_info(h, 0)
    info1 = mgs.mg_get_level_info(h, 1) if info0["levels"] > 1 else info0
    n_next = info1["nr"] * info1["nth"] * info1["nph"]
    stencil = rep["stencil"]
    axi = stencil == 19 and g["mapping"] != 2
    sched = mgs.mg_get_schedule(h)
    one_pass = bool(sched.get("one_pass_tiles", 0)) and smoother == 0
    prof, slots = profile_solves(mgs, h, fd, xd, max(2, min(steps, 10)), flush, torch, stencil, prec, N, n_next,
                                 smoother, axi, one_pass)
    name = max(((k, v) for k, v in slots.items() if k in ("smooth0", "residual", "restrict0", "prolong0", "update")),
               key=lambda kv: kv[1][0])[0]
    pname = [k for k, v in PREC.items() if v == prec][0]
    roof = roofline_of(name, slots, steps, stencil, prec, N, n_next, smoother, axi, one_pass,
                       ncu_traffic(traffic_key or workload, pname, name, one_pass))
    # the kernel's share of all device time of the profiled solves (every
    # slot and every coarse level): comparable with an ncu launch list
    roof["share_of_step"] = prof["kernels"][name]["ms_per_solve"] / max(prof["attributed_ms_per_solve"], 1e-30)
    add_event_check(roof, prof, name)
    prof["attributed_over_headline"] = prof["attributed_ms_per_solve"] / statistics.mean(ms)
    prof["device_over_headline"] = (prof["attributed_ms_per_solve"] + prof["launch_gaps_ms_per_solve"]) / statistics.mean(ms)
    leg = {"workload": workload if scale == 1 else f"{workload}/{scale}", "grid": f"{g['nr']}x{g['nth']}x{g['nph']}",
           "value": N / (statistics.mean(ms) / 1e3), "ms_per_step": statistics.mean(ms),
           "p99_ms": float(__import__("numpy").percentile(ms, 99)), "iters": rep["iters"], "rel_res": rep["rel_res"],
           "levels": rep["levels"], "stencil": stencil, "setup_s": t_setup, "schedule": sched,
           "roofline": roof, "profile": prof, "gpu_launches": int(sum(r["launches"] for r in reps)), "ms": ms}
    return leg, h, g, f, fd, xd, rep


def fp64_compare(args, mgs, torch, g, sopts, fd, xd, flush, world, ms_step, steps):
    """Plain FP64 multigrid on the same workload: the speedup reference."""
    N = g["nr"] * g["nth"] * g["nph"]
    h64 = mgs.mg_setup(g, dict(sopts, precision=0))
    xd.zero_()
    mgs.mg_solve(h64, fd, xd, tol=TOL)
    ms64, reps64 = time_solves(mgs, h64, fd, xd, steps, flush, torch)
    v64 = world * N / (statistics.mean(ms64) / 1e3)
    h64.close()
    return {"value": v64, "ms_per_step": statistics.mean(ms64), "iters": reps64[-1]["iters"],
            "speedup": statistics.mean(ms64) / ms_step}


def c3_leg(args, mgs, torch, flush, world):
    """The 256 x 256 x 512 oblate shell (19 points): FP32 cycles, FP16
    coefficients, and plain FP64 multigrid, each to the bench tolerance."""
    steps = max(3, min(args.steps, 8))
    out = {}
    for pname in ("fp32", "fp16"):
        leg, h, g, f, fd, xd, rep = single_leg(args, mgs, torch, "single_oblate_256", 1, PREC[pname], 0, steps,
                                               max(1, min(args.warmup, 2)), flush)
        leg.pop("ms")
        if pname == "fp32":
            out.update(leg)
            if not args.no_compare:
                out["fp64_mg"] = fp64_compare(args, mgs, torch, g, dict(precision=0), fd, xd, flush, world,
                                              leg["ms_per_step"], max(2, steps // 3))
        else:
            out["fp16_coefficients"] = {k: leg[k] for k in ("value", "ms_per_step", "iters", "rel_res", "roofline",
                                                            "setup_s")}
        h.close()
        del fd, xd
        torch.cuda.empty_cache()
    return out


def run_ours(args, rank, world, local_rank):
    global TOL
    TOL = args.tol
    import numpy as np
    import torch
    import paper_2305_17875_gb300 as mgs
    import workloads as W

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
    prec = PREC[args.precision]
    smoother = SMOOTHER[args.smoother]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    w = W.single(args.workload, args.scale)
    g, f = w["grid"], w["f"]
    N = g["nr"] * g["nth"] * g["nph"]
    sopts = dict(precision=prec, smoother=smoother)
    if smoother == SMOOTHER["plane"]:
        sopts.update(nu1=1, nu2=1)          # the semi-coarsening multigrid's V(1,1)
    if "max_levels" in w:
        sopts["max_levels"] = w["max_levels"]
    if "max_iters" in w:
        sopts["max_iters"] = w["max_iters"]
    if w.get("coarsen") == "full":
        sopts["coarsen"] = 1
    t_setup = time.perf_counter()
    h = mgs.mg_setup(g, sopts)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    fd = torch.from_numpy(f).cuda()
    xd = torch.zeros_like(fd)
    for _ in range(args.warmup):
        xd.zero_()
        mgs.mg_solve(h, fd, xd, tol=TOL)

    # the headline: timed with profiling off
    clocks = Clocks(local_rank)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0 = time.perf_counter()
    ms, reps = time_solves(mgs, h, fd, xd, args.steps, flush, torch)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms_step = max_over_ranks(statistics.mean(ms))
    rep = reps[-1]
    info0 = mgs.mg_get_level_info(h, 0)
    info1 = mgs.mg_get_level_info(h, 1) if info0["levels"] > 1 else info0
    n_next = info1["nr"] * info1["nth"] * info1["nph"]
    stencil = rep["stencil"]
    axi = stencil == 19 and g["mapping"] != 2
    sched = mgs.mg_get_schedule(h)
    one_pass = bool(sched.get("one_pass_tiles", 0)) and smoother == 0

    # kernel breakdown: a separate profiled run of the same solves
    prof, slots = profile_solves(mgs, h, fd, xd, max(2, min(args.steps, 10)), flush, torch, stencil, prec, N,
                                 n_next, smoother, axi, one_pass)
    name = max(((k, v) for k, v in slots.items() if k in ("smooth0", "residual", "restrict0", "prolong0", "update")),
               key=lambda kv: kv[1][0])[0]
    roof = roofline_of(name, slots, args.steps, stencil, prec, N, n_next, smoother, axi, one_pass,
                       ncu_traffic(args.workload if args.smoother == "gs" else f"{args.workload}/{args.smoother}",
                                   args.precision, name, one_pass))
    roof["share_of_step"] = prof["kernels"][name]["ms_per_solve"] / max(prof["attributed_ms_per_solve"], 1e-30)
    add_event_check(roof, prof, name)
    prof["attributed_over_headline"] = prof["attributed_ms_per_solve"] / ms_step
    # kernels plus the launch gaps between them: the device time of the
    # solve's program runs
    prof["device_over_headline"] = (prof["attributed_ms_per_solve"] + prof["launch_gaps_ms_per_solve"]) / ms_step

    # end to end through the public host-buffer call (pinned host memory)
    fh = torch.from_numpy(f.copy()).pin_memory()
    xh = torch.zeros_like(fh).pin_memory()
    # warm-up (untimed): the first call allocates the handle's staging
    # buffers
    for _ in range(max(1, min(args.warmup, 2))):
        xh.zero_()
        mgs.mg_solve_host(h, fh.numpy(), xh.numpy(), tol=TOL)
    e2e_ms = []
    for _ in range(max(2, min(args.steps, 5))):
        xh.zero_()
        flush.fill_(2.0)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        mgs.mg_solve_host(h, fh.numpy(), xh.numpy(), tol=TOL)
        e2e_ms.append((time.perf_counter() - t1) * 1e3)
    e2e = {"value": world * N / (statistics.mean(e2e_ms) / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": 2 * 8 * N, "d2h_bytes_per_step": 8 * N,
           "ms_per_step": statistics.mean(e2e_ms)}

    # the steps either side of the solve in the pressure correction
    # (Section 3.6): right side of Eq. PC_6 and correction of Eq. PC_7 from a
    # random staggered velocity, device time per call
    pc_step = None
    if world == 1:
        u = torch.randn(9 * N, dtype=torch.float64, device="cuda")
        fpc = torch.empty(N, dtype=torch.float64, device="cuda")
        mgs.mg_pc_rhs(h, u, fpc)                       # first call builds the face C
        def _ev_time(fn, reps=5):
            flush.fill_(3.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                fn()
            e1.record()
            e1.synchronize()
            return e0.elapsed_time(e1) / reps
        t_rhs = _ev_time(lambda: mgs.mg_pc_rhs(h, u, fpc))
        t_cor = _ev_time(lambda: mgs.mg_pc_correct(h, xd, u))
        b_rhs, b_cor = 160.0 * N, (8 + 216 + 24 + 144) * N
        pc_step = {"rhs_ms": t_rhs, "correct_ms": t_cor,
                   "rhs_alg_GBps": b_rhs / (t_rhs * 1e-3) / 1e9, "correct_alg_GBps": b_cor / (t_cor * 1e-3) / 1e9,
                   "step_ms": t_rhs + ms_step + t_cor,
                   "note": "right side + solve + correction of one pressure-correction step"}
        del u, fpc

    # the line solves of Section 3.5 on this grid's field: every radial line
    # (plain Thomas) and every longitude line (periodic Thomas) of random
    # diagonally dominant systems, FP64; algorithmic bytes = a, b, c, g read
    # and x written once (40 B per unknown)
    line_solves = None
    if world == 1:
        shape = (g["nr"], g["nth"], g["nph"])
        gen = torch.Generator(device="cuda").manual_seed(3)
        la = -torch.rand(shape, generator=gen, device="cuda", dtype=torch.float64)
        lc = -torch.rand(shape, generator=gen, device="cuda", dtype=torch.float64)
        lb = 2.2 + torch.rand(shape, generator=gen, device="cuda", dtype=torch.float64)
        lg = torch.randn(shape, generator=gen, device="cuda", dtype=torch.float64)
        lx = torch.empty_like(lg)
        lw = torch.empty(2 * N, dtype=torch.float64, device="cuda")
        line_solves = {}
        for key, axis, per in (("radial", 0, False), ("longitude_periodic", 2, True)):
            L = mgs.lines_along(shape, axis)
            mgs.mg_thomas(L, la, lb, lc, lg, lx, periodic=per, work=lw)
            t = _ev_time(lambda: mgs.mg_thomas(L, la, lb, lc, lg, lx, periodic=per, work=lw))
            gbs = 40.0 * N / (t * 1e-3) / 1e9
            line_solves[key] = {"ms": t, "alg_GBps": gbs, "frac": gbs / peaks()[0],
                                "lines": L["n1"] * L["n2"], "n": L["n"]}
        del la, lb, lc, lg, lx, lw

    # one ADI-CN sub-step of Section 3.4 (three implicit sweeps, Eqs.
    # solve_2-solve_4) on this grid: diffusion number kappa G / J up to 10,
    # no-slip walls; algorithmic bytes 136 per cell (u^n, s, J, three G read
    # and u written in the first sweep; u, u^n, J, one G read and u written in
    # each of the other two)
    adi_step = None
    if world == 1:
        Jd = torch.empty(N, dtype=torch.float64, device="cuda")
        mgs.mg_get_metric(h, 0, 9, Jd)
        uo = torch.empty(N, dtype=torch.float64, device="cuda")
        gmax = 0.0
        for comp in (0, 4, 8):
            mgs.mg_get_metric(h, 0, comp, uo)
            gmax = max(gmax, uo.abs().max().item())
        kappa = 10.0 * Jd.min().item() / gmax
        gen = torch.Generator(device="cuda").manual_seed(5)
        un = [torch.randn(N, generator=gen, device="cuda", dtype=torch.float64) for _ in range(3)]
        src = [0.01 * torch.randn(N, generator=gen, device="cuda", dtype=torch.float64) * Jd for _ in range(3)]
        uo = [uo] + [torch.empty_like(uo) for _ in range(2)]
        mgs.mg_adi_substep(h, kappa, un[0], uo[0], src=src[0])
        t1 = _ev_time(lambda: mgs.mg_adi_substep(h, kappa, un[0], uo[0], src=src[0]))
        mgs.mg_adi_substep(h, kappa, un, uo, src=src)
        t3 = _ev_time(lambda: mgs.mg_adi_substep(h, kappa, un, uo, src=src))
        gbs = 136.0 * N / (t1 * 1e-3) / 1e9
        gbs3 = 3 * 136.0 * N / (t3 * 1e-3) / 1e9
        adi_step = {"ms": t1, "alg_GBps": gbs, "frac": gbs / peaks()[0],
                    "ms_3_fields": t3, "alg_GBps_3_fields": gbs3, "frac_3_fields": gbs3 / peaks()[0],
                    "kappa": kappa,
                    "note": "three FP64 line-solve sweeps (2 plain, 1 periodic), no-slip walls; one field, "
                            "and the three velocity components in one call"}
        del Jd, un, src, uo

    # plain FP64 multigrid on the same workload (the speedup reference)
    compare = None
    if not args.no_compare and prec != 0:
        compare = fp64_compare(args, mgs, torch, g, sopts, fd, xd, flush, world, ms_step, max(3, args.steps // 3))
    h.close()
    del fd, xd
    torch.cuda.empty_cache()

    # the 19-point oblate shell (C3) in the same line, when the headline is the
    # default workload
    c3 = None
    if world == 1 and args.workload == "single_sphere_128" and args.scale == 1 and not args.no_c3:
        c3 = c3_leg(args, mgs, torch, flush, world)

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": world * N / (ms_step / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "p99_ms": float(np.percentile(ms, 99)), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if prec else "f64", "data": "synthetic",
        "config": config_of(args, g, rep, stencil),
        "rel_res": rep["rel_res"], "iters": rep["iters"],
        "roofline": roof, "profile": prof,
        "setup_s": t_setup, "schedule": sched, "pc_step": pc_step,
        "line_solves": line_solves, "adi_substep": adi_step,
        "e2e": e2e,
        "gpu_launches": int(sum(r["launches"] for r in reps)),
        "clocks": clk, "fp64_mg": compare, "wall_s": wall, "c3": c3,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(g, TOL, kind=sopts["smoother"])
        line["cpu_baseline_all_cores"] = cpu_baseline(g, TOL, kind=sopts["smoother"], all_cores=True)
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- batch of uneven shells
def run_batch(args, rank, world, local_rank):
    """64 shells of uneven size solved together (one launch per level
    operation over all shells, captured outer iterations); value = fine cells
    of all shells / batch solve time.  Also times the same shells solved one
    after another and the plain FP64 multigrid batch."""
    import torch
    import paper_2305_17875_gb300 as mgs
    import workloads as W
    torch.cuda.set_device(local_rank)
    items = W.batch_shells(64)
    prec = PREC[args.precision]
    hs, fds, xds, cells = [], [], [], 0
    for it in items:
        g = it["grid"]
        hs.append(mgs.mg_setup(g, dict(precision=prec)))
        fds.append(torch.from_numpy(W.batch_rhs(it)).cuda())
        xds.append(torch.zeros_like(fds[-1]))
        cells += g["nr"] * g["nth"] * g["nph"]
    tols = [args.tol] * len(hs)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def batch_once(handles):
        for x in xds:
            x.zero_()
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        reps = mgs.mg_solve_batch(handles, fds, xds, tols)
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1), reps

    for _ in range(args.warmup):
        batch_once(hs)
    clocks = Clocks(local_rank)
    torch.cuda.synchronize()
    sync_ranks()
    clocks.start()
    mgs.mg_profile_enable(hs[0], True)
    runs = [batch_once(hs) for _ in range(args.steps)]
    mgs.mg_profile_enable(hs[0], False)
    clk = clocks.stop()
    ms = [r[0] for r in runs]
    reps = runs[-1][1]
    ms_step = max_over_ranks(statistics.mean(ms))
    # the same shells one after another
    seq = 0.0
    for h, f, x in zip(hs, fds, xds):
        x.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        mgs.mg_solve(h, f, x, tol=args.tol)
        e1.record()
        e1.synchronize()
        seq += e0.elapsed_time(e1)
    compare = None
    if not args.no_compare and prec != 0:
        h64 = [mgs.mg_setup(it["grid"], dict(precision=0)) for it in items]
        batch_once(h64)
        ms64 = [batch_once(h64)[0] for _ in range(max(1, args.steps // 3))]
        compare = {"value": world * cells / (statistics.mean(ms64) / 1e3), "ms_per_step": statistics.mean(ms64),
                   "speedup": statistics.mean(ms64) / ms_step}
        for h in h64:
            h.close()
    if rank != 0:
        return
    iters = [r["iters"] for r in reps]
    line = {
        "metric": METRIC, "value": world * cells / (ms_step / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "p99_ms": float(__import__("numpy").percentile(ms, 99)), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if prec else "f64", "data": "synthetic",
        "config": {"workload": "batch_64", "shells": len(hs), "cells": cells, "tol": args.tol,
                   "precision": PREC_NAME[prec], "l2": "flushed (256 MB write) before every step",
                   "parallelism": f"replicas x{world}"},
        "iters": {"min": min(iters), "max": max(iters)}, "max_rel_res": max(r["rel_res"] for r in reps),
        "sequential_ms": seq, "batching_speedup": seq / ms_step,
        "gpu_launches": int(reps[0]["launches"]) * args.steps, "clocks": clk, "fp64_mg": compare,
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- serve stream
def serve_rate(mgs, sv, reqs, prec):
    """Submit the requests at their Poisson arrival times; poll until every
    result is back.  Returns (wall s, latencies ms, cells)."""
    import numpy as np
    tickets, out = [], {}
    t0 = time.perf_counter()
    nxt = 0
    while len(out) < len(reqs):
        now = time.perf_counter() - t0
        while nxt < len(reqs) and reqs[nxt]["t_arrive"] <= now:
            r = reqs[nxt]
            tickets.append(mgs.mg_serve_submit(sv, r["grid"], r["f"], r["tol"], dict(precision=prec)))
            nxt += 1
        for q, tk in enumerate(tickets):
            if q in out:
                continue
            res = mgs.mg_serve_poll(sv, tk, None)
            if res is not None:
                out[q] = res[1]
        time.sleep(0.0002)
    wall = time.perf_counter() - t0
    lat = np.array([out[q]["seconds"] * 1e3 for q in range(len(reqs))])
    cells = sum(r["grid"]["nr"] * r["grid"]["nth"] * r["grid"]["nph"] for r in reqs)
    return wall, lat, cells


def run_serve(args, rank, world, local_rank):
    """The serve stream at every offered rate of the workload (Poisson
    arrivals into the continuous-batching serve loop; every request a new
    grid, its right side from the host, its solution back to the host);
    latency = submit to result, throughput = requests (and fine cells) / wall
    time.  Compared with plain FP64 set-up + solve of the same requests one
    after another."""
    import numpy as np
    import torch
    import paper_2305_17875_gb300 as mgs
    import workloads as W
    torch.cuda.set_device(local_rank)
    prec = PREC[args.precision]
    rates = [float(r) for r in args.rates.split(",")]
    pool = {}   # two right sides per size (the sizes are a small discrete set)

    def with_rhs(reqs):
        for q, r in enumerate(reqs):
            key = r["grid"]["nr"]
            if key not in pool:
                pool[key] = [W.rhs_modes(r["grid"], seed=2000 + key), W.rhs_modes(r["grid"], seed=3000 + key)]
            r["f"] = pool[key][q & 1]
        return reqs

    sv = mgs.mg_serve_create(max_slots=64, setup_threads=8)
    g0 = W.grid_desc(32, r_out=2.0, mapping=1, flattening=0.05)     # warm-up request
    t = mgs.mg_serve_submit(sv, g0, W.rhs_modes(g0), 1e-8, dict(precision=prec))
    while mgs.mg_serve_poll(sv, t, None) is None:
        time.sleep(0.001)
    sync_ranks()
    per_rate = []
    for rate in rates:
        reqs = with_rhs(W.serve_stream(n=args.requests, rate=rate, seed=int(rate)))
        wall, lat, cells = serve_rate(mgs, sv, reqs, prec)
        wall = max_over_ranks(wall)
        per_rate.append({"rate_per_s": rate, "requests": len(reqs), "req_per_s": len(reqs) / wall,
                         "dof_per_s": world * cells / wall, "p50_ms": float(np.percentile(lat, 50)),
                         "p99_ms": float(np.percentile(lat, 99)), "wall_s": wall,
                         "mean_cells": cells / len(reqs)})
    stats = mgs.mg_serve_stats(sv)
    sv.close()
    # sequential plain FP64 (set-up + solve per request) on a prefix of a stream
    seq_reqs = with_rhs(W.serve_stream(n=min(args.requests, 40), rate=rates[0], seed=int(rates[0])))
    t1 = time.perf_counter()
    seq_cells = 0
    for r in seq_reqs:
        h = mgs.mg_setup(r["grid"], dict(precision=0, autotune=0))   # a new grid: no tuning, as in the server
        fd = torch.from_numpy(r["f"]).cuda()
        x = torch.zeros_like(fd)
        mgs.mg_solve(h, fd, x, tol=r["tol"])
        x.cpu()
        h.close()
        seq_cells += r["grid"]["nr"] * r["grid"]["nth"] * r["grid"]["nph"]
    seq_wall = time.perf_counter() - t1
    seq = {"requests": len(seq_reqs), "req_per_s": len(seq_reqs) / seq_wall, "value": seq_cells / seq_wall,
           "includes": "set-up (default schedule, no tuning), host-to-device copy, solve and "
                       "device-to-host copy per request"}
    for pr in per_rate:
        pr["throughput_vs_sequential_fp64"] = pr["req_per_s"] / seq["req_per_s"]
    if rank != 0:
        return
    best = max(per_rate, key=lambda pr: pr["dof_per_s"])
    nreq = sum(pr["requests"] for pr in per_rate)
    line = {
        "metric": METRIC, "value": best["dof_per_s"], "unit": UNIT, "n_gpus": world, "steps": nreq, "warmup": 1,
        "ms_per_step": best["wall_s"] * 1e3 / best["requests"], "p50_ms": best["p50_ms"], "p99_ms": best["p99_ms"],
        "req_per_s": best["req_per_s"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if prec else "f64", "data": "synthetic",
        "config": {"workload": "serve_stream", "requests_per_rate": args.requests, "rates_per_s": rates,
                   "precision": PREC_NAME[prec], "sizes": sorted(pool), "parallelism": f"replicas x{world}",
                   "note": f"{args.requests} requests per offered rate (the specified stream has 10000)"},
        "per_rate": per_rate, "serve_stats": stats, "sequential_fp64": seq,
        "e2e": {"value": best["dof_per_s"], "unit": UNIT, "h2d_bytes_per_step": int(8 * best["mean_cells"]),
                "d2h_bytes_per_step": int(8 * best["mean_cells"])},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batch_64":
        run_batch(args, rank, world, local_rank)
    elif args.workload == "serve_stream":
        run_serve(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
