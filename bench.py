#!/usr/bin/env python3
"""Benchmark of the single-level comoving gas advance on GB300.

One step = ghost fill + fused advance + CFL dt of the whole level (every
box), i.e. one pass of the hot path over one synthetic level.  Default
workload: the large batched mixed-precision level, a periodic 512^3 domain
cut into 4096 boxes of 32^3 plus 410 independent 64^3 boxes at half the
cell width (2.42e8 valid cells), lognormal comoving field with sigma = 1.0,
a from 1/51 to 1/31.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle, as it stands, on a bounded sample of the same workload.
N > 1 (torchrun): every rank advances its own replica of the level on its
own GPU (replicas, weak scaling); timing is the max over ranks.
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

from paper_1301_4498_gb300 import workloads as W  # noqa: E402

METRIC = "zone-updates/s per level step on 1 GB300 + HBM-roofline fraction, FP32-batched vs FP64"
ALG_BYTES_PER_ZONE = 120  # read S (6 x 8 B) + g (3 x 8 B), write S (6 x 8 B)
# Standalone corrector (Step 6 with g^{n+1}): read rho, m at t^n (4 x 8 B), the
# predictor (6 x 8 B), g^n and g^{n+1} (2 x 3 x 8 B); write m, rhoE, rhoe (5 x 8 B).
CORRECT_BYTES_PER_ZONE = 168
# Its FP64 operations per zone (option (i)): momentum corrector 3 x 6, energy
# corrector 16 (two dot products and the weighted difference), dual-energy
# sync 10 (kinetic energy with its division, the switch test, the
# subtraction).  FP64 division and square root run at a small fraction of the
# FP32 rate here.
CORRECT_FP64_FLOPS_PER_ZONE = 44
# The shock-flattening pass reads five state components of every cell (rho,
# the three momenta, rho e; 40 B, the +-3 stencil's reuse coming from the
# caches) and writes one coefficient (float for mixed plans, double for
# FP64 ones), per zone.
FLATTEN_BYTES_PER_ZONE = {"mixed": 44, "fp64": 48}
# 4 pi G of the self-gravity workloads in code units (mean density 1, sound
# speed 1, box length 1): a free-fall time of order the sound crossing time.
COSMO_FOUR_PI_G = 1.0
# Algorithmic floating-point operations per zone-update (+ - * / sqrt counted
# once each, comparisons not counted): 3196 for primitives, PPM + tracing in 3
# directions, 12 Riemann set-ups/samplings, 18 corner-coupling corrections and
# the FP64 update (165 in the FP64 forms), plus 480 per mean Newton iteration
# of the 12 two-shock solves.  The FP64 oracle on the large level's 64^3
# boxes, in the initial state every timed phase starts from, averages 3.14
# iterations at the mixed path's tolerance (1e-6) and 3.83 at the FP64 one
# (1e-10).
ALG_FLOPS_PER_ZONE = {"mixed": 3196 + 480 * 3.14, "fp64": 3196 + 480 * 3.83}
# The mixed path splits them over two pipes.  FP64: the update as written
# (flux differences and divergence 48, predictor 2 + 1 + 18, reciprocal of
# the density 3, m.g 5, total energy 8, internal energy 7, gravity corrector
# 20, dual-energy sync with the kinetic energy 10): 122.  FP32: the rest
# (the FP64 forms' update of 165 taken out).
ALG_FP64_FLOPS_MIXED = 122
ALG_FP32_FLOPS_MIXED = ALG_FLOPS_PER_ZONE["mixed"] - 165
# DRAM bytes per zone of the task-form kernel at 16 x 8 tiles on the large
# level's box sizes, from one ncu capture of the large128 workload (the same
# box sizes on a 128^3 domain); traffic scales with the cells of boxes of the
# same sizes.  Reported only for that kernel, workload and shape, and only
# while the kernel is the one captured.
NOMINAL_HBM_GBS = 7900.0   # HBM3e nominal rate of the part, beside the measured copy rate
TRAFFIC_BYTES_PER_ZONE = {("large", 3): 154.3, ("large128", 3): 154.3}
# Unit-count peaks (152 SMs at the 2070 MHz maximum clock; 128 FP32 and 2
# FP64 FMA lanes per SM per clock), reported beside the measured ones.
NOMINAL_FP32_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
NOMINAL_FP64_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def measure_alu(stream=None):
    """FP32 and FP64 multiply-add peaks of this GPU, measured by the
    library's own throughput probe (nyx_alu_peak), in TFLOP/s (FMA = 2)."""
    from paper_1301_4498_gb300 import hydro as H
    f32 = H.alu_peak("fp32", 0.25, stream)
    f64 = H.alu_peak("fp64", 0.25, stream)
    return {"fp32_tflops": 2 * f32 / 1e12, "fp64_tflops": 2 * f64 / 1e12,
            "fp32_fma_per_s": f32, "fp64_fma_per_s": f64,
            "nominal_fp32_tflops": NOMINAL_FP32_TFLOPS, "nominal_fp64_tflops": NOMINAL_FP64_TFLOPS,
            "how": "nyx_alu_peak: 8 independent FMA chains per thread, 8 x 256 threads per SM, "
                   "best of 5 timed launches (CUDA events)"}


def roofline_of(kernel_ms, cells, precision, peaks, peak_src, alu, kernel, traffic=None):
    """Roofline of one launch of the advance over `cells` zones: the time
    each roof (HBM at the measured copy rate, the FP32 and the FP64 pipe at
    their measured FMA rates) allows for the algorithmic work, and the
    achieved fraction of the binding (slowest) one."""
    sec = kernel_ms / 1e3
    if precision == "mixed":
        work = {"fp32": ALG_FP32_FLOPS_MIXED, "fp64": ALG_FP64_FLOPS_MIXED}
    else:
        work = {"fp64": ALG_FLOPS_PER_ZONE["fp64"]}
    roofs = {"hbm": {"bound": "hbm", "alg_per_zone": ALG_BYTES_PER_ZONE, "unit": "GB/s",
                     "achieved": ALG_BYTES_PER_ZONE * cells / sec / 1e9,
                     "peak": peaks["hbm_gbs"], "peak_source": f"hbm_gbs {peak_src}"}}
    for pipe, fz in work.items():
        roofs[pipe] = {"bound": pipe, "alg_per_zone": fz, "unit": "TFLOP/s",
                       "achieved": fz * cells / sec / 1e12,
                       "peak": alu[f"{pipe}_tflops"], "peak_source": "measured (nyx_alu_peak)"}
    for r in roofs.values():
        r["frac"] = r["achieved"] / r["peak"]
        r["roof_ms"] = kernel_ms * r["frac"]
    bind = max(roofs, key=lambda k: roofs[k]["roof_ms"])
    b = roofs[bind]
    out = {"bound": b["bound"], "achieved": b["achieved"], "peak": b["peak"], "unit": b["unit"],
           "frac": b["frac"], "traffic": traffic, "traffic_unit": "bytes per launch",
           "kernel": kernel, "kernel_ms": kernel_ms, "peak_source": b["peak_source"],
           "binding": "the roof allowing the longest time for the algorithmic work",
           "roofs": roofs}
    return out


def make_workload(name: str, sample_only: bool = False):
    """The named workload with its prescribed scale-factor schedule (the
    bench takes the first K+1 values of it)."""
    if name == "large":  # a from 1/51 to 1/31 over 100 steps
        if sample_only:  # the independent 64^3 boxes only: what the CPU sample uses
            return W.large_level(nsteps=100, coarse_select=[], fine_select=range(16))
        return W.large_level(nsteps=100)
    if name == "large128":  # the large level's box sizes on a 128^3 domain (profiling case)
        return W.large_level(n=128, box=32, nfine=6, nsteps=100)
    if name == "comoving128":
        return W.comoving_box(n=128, sigma=0.5, seed=1, nsteps=10)
    if name == "uneven512":
        return W.uneven_boxes(nbox=512, nsteps=10)
    if name == "uneven64":  # the first 64 boxes of the 512-box level (profiling case)
        return W.uneven_boxes(nbox=512, boxes=list(range(64)), nsteps=10)
    if name == "mixed256":
        return W.comoving_box(n=256, sigma=1.0, seed=4, nsteps=50, mixed=True)
    if name == "sod":
        return W.sod()
    if name == "amr":  # the large level with its 10% refined boxes coupled (ratio 2)
        if sample_only:
            return W.amr_level(n=64, box=32, nfine=1, nsteps=100, a0=1.0 / 51, aN=1.0 / 31)
        return W.amr_large(nsteps=100)
    if name == "amr128":  # the same structure on a 128^3 domain (profiling case)
        return W.amr_large(n=128, box=32, nfine=6, nsteps=100)
    if name == "cosmo":  # gas + dark matter + self-gravity on the 512^3 level (Steps 1-6)
        return W.cosmo_level(n=64 if sample_only else 512, box=32, nsteps=100)
    if name == "cosmo128":
        return W.cosmo_level(n=128, box=32, nsteps=100)
    raise SystemExit(f"unknown workload {name}")


def a_schedule_for(w, nsteps):
    """a_0..a_nsteps: the workload's schedule, continued linearly (never
    cycled back) if more steps are asked for than it prescribes."""
    a = np.asarray(w.a_sched, dtype=np.float64)
    if len(a) >= nsteps + 1:
        return a[: nsteps + 1].copy()
    step = (a[-1] - a[0]) / max(1, len(a) - 1)
    extra = a[-1] + step * np.arange(1, nsteps + 2 - len(a))
    return np.concatenate([a, extra])


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
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
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus):
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, ws: int) -> float:
    """Max of a host scalar over all ranks (timing only; no data-path exchange)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if (torch.cuda.is_available() and dist.get_backend() == "nccl") else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------- CPU oracle timing

def oracle_sample(workload_name, w, budget_s=12.0, max_boxes=None, threads=0):
    """Time the FP64 CPU oracle on a bounded sample of the workload: whole
    independent boxes (periodic domains of their own) advanced one step,
    added one at a time until ``budget_s`` of CPU time is spent.  threads:
    OpenMP threads (0: all host cores)."""
    import oracle
    oracle.set_threads(threads)
    P = oracle.OracleParams(gamma=w.gamma, cfl=w.cfl)
    lev = w.level
    # boxes that are their own domain (all of them for single-box levels)
    dom_count = np.bincount(lev.dom)
    own = [b for b in range(lev.nbox) if dom_count[lev.dom[b]] == 1]
    if not own:
        own = list(range(lev.nbox))
    cells = 0
    elapsed = 0.0
    used = 0
    a0, a1 = float(w.a_sched[0]), float(w.a_sched[1])
    for b in own:
        sub = lev.subset([b])
        st = [w.state[b]]
        gr = None if w.grav is None else [w.grav[b]]
        t0 = time.perf_counter()
        dt = oracle.estdt(sub, P, st, a0)
        oracle.advance(sub, P, st, gr, a_old=a0, a_new=a1, dt=dt)
        elapsed += time.perf_counter() - t0
        cells += int(np.prod(sub.hi[0] - sub.lo[0] + 1))
        used += 1
        if elapsed >= budget_s or (max_boxes and used >= max_boxes):
            break
    oracle.set_threads(0)
    where = f"{threads} host thread(s)" if threads > 0 else "OpenMP on all host cores"
    return {"value": cells / elapsed, "unit": "zone-updates/s",
            "cores": threads if threads > 0 else os.cpu_count(),
            "kind": "oracle", "elapsed_s": elapsed,
            "sample": f"{used} whole box(es) of the '{workload_name}' workload ({cells} cells), "
                      f"1 step each, FP64 oracle, {where}; {elapsed:.1f} s"}


def run_reference(args, w):
    ws, rank, _ = dist_setup(args.gpus)
    if rank != 0:
        return
    # each step: one oracle step on a bounded sample of the workload
    per_step = []
    info = None
    for s in range(args.warmup + args.steps):
        r = oracle_sample(args.workload, w, budget_s=args.ref_budget, max_boxes=args.ref_boxes)
        if s >= args.warmup:
            per_step.append(r)
        info = r
    value = statistics.median(x["value"] for x in per_step)
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "zone-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.median(x["elapsed_s"] for x in per_step) * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "level": w.name, "sample": info["sample"]},
        "cpu_baseline": {"value": value, "unit": "zone-updates/s", "cores": info["cores"],
                         "kind": "oracle", "sample": info["sample"]},
        "e2e": {"value": value, "unit": "zone-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------- GPU path

def field_errors(plan, spec, got, ref):
    """Per conserved field, normwise relative L-inf and L1 differences of two
    level states over the valid cells, taken on strided views of runs of
    equally shaped, consecutive boxes."""
    off, st = plan.layout(6)
    runs, b0 = [], 0
    for b in range(1, spec.nbox + 1):
        if b == spec.nbox or spec.extent(b) != spec.extent(b0) or st[b] != st[b0]:
            runs.append((b0, b))
            b0 = b
    g_ng = spec.ng
    ninf, dinf, n1, d1 = [0.0] * 6, [0.0] * 6, [0.0] * 6, [0.0] * 6
    for r0, r1 in runs:
        nx, ny, nz = spec.extent(r0)
        shp = (nz + 2 * g_ng, ny + 2 * g_ng, nx + 2 * g_ng)
        vol = shp[0] * shp[1] * shp[2]
        s = int(st[r0])
        v = slice(g_ng, -g_ng)

        def view(x):
            return x[int(off[r0]):int(off[r1])].view(r1 - r0, 6, s)[:, :, :vol] \
                .reshape(r1 - r0, 6, *shp)[:, :, v, v, v]
        G, R = view(got), view(ref)
        for c in range(6):
            d = (G[:, c] - R[:, c]).abs()
            ra = R[:, c].abs()
            ninf[c] = max(ninf[c], float(d.max()))
            dinf[c] = max(dinf[c], float(ra.max()))
            n1[c] += float(d.sum())
            d1[c] += float(ra.sum())
            del d, ra
    names = ["rho", "m_x", "m_y", "m_z", "rhoE", "rhoe"]
    return {n: {"linf": ninf[c] / max(dinf[c], 1e-300), "l1": n1[c] / max(d1[c], 1e-300)}
            for c, n in enumerate(names)}


def mixed256_errors(H, torch):
    """256^3 periodic box, sigma = 1.0, a 1/51 -> 1/49 over 50 steps: the mixed
    and the FP64 persistent forms from the same initial state, each with its
    own CFL steps; per conserved field the normwise relative L-inf and L1
    difference after step 50, and each form's rate over the 50 steps."""
    w = make_workload("mixed256")
    cells = w.level.valid_cells()
    out = {"workload": w.name, "steps": w.nsteps, "cells": cells}
    states = {}
    for prec in ("mixed", "fp64"):
        plan = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl, precision=prec, batching="persistent",
                      autotune=1)
        lev = H.make_level(plan, w.state, w.grav)
        snap = lev.state[0].clone()
        a = torch.tensor(a_schedule_for(w, w.nsteps), dtype=torch.float64, device="cuda")
        dt = torch.zeros(w.nsteps + 1, dtype=torch.float64, device="cuda")
        plan.run(lev, a, dt, w.nsteps, compute_dt0=True, use_graph=True)
        torch.cuda.synchronize()
        lev.state[0].copy_(snap)
        lev.cur = 0
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(plan.torch_stream)
        plan.run(lev, a, dt, w.nsteps, compute_dt0=True, use_graph=True)
        e1.record(plan.torch_stream)
        torch.cuda.synchronize()
        rc, flags = plan.status()
        out[prec] = {"status": rc, "value": cells * w.nsteps / (e0.elapsed_time(e1) / 1e3),
                     "unit": "zone-updates/s", "dt_last": float(dt[w.nsteps - 1])}
        states[prec] = lev.state[lev.cur].clone()
        keep = plan
        del lev, snap
        if prec == "fp64":
            out["fields"] = field_errors(keep, w.level, states["mixed"], states["fp64"])
        keep.close()
    out["metric"] = "normwise relative over the valid cells: max|d|/max|ref| and sum|d|/sum|ref|"
    del states
    torch.cuda.empty_cache()
    return out


def run_ours(args, w):
    import torch
    from paper_1301_4498_gb300 import hydro as H
    ws, rank, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    peaks, peak_src = load_peaks()
    K, Wm = args.steps, args.warmup
    cells = w.level.valid_cells()

    plan = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl, precision=args.precision,
                  batching="persistent", autotune=1 if args.autotune else 0)
    if args.tile_shape >= 0:
        plan.set_tile_shape(args.tile_shape)
    lev = H.make_level(plan, w.state, w.grav)
    a_host = a_schedule_for(w, max(K, Wm) + 1)
    a = torch.tensor(a_host, dtype=torch.float64, device="cuda")
    dt = torch.zeros(len(a_host), dtype=torch.float64, device="cuda")
    stream = plan.torch_stream

    # Every measured phase starts from the initial state (restored outside the
    # timed regions), so each runs the same first steps of the evolution.
    snap = lev.state[lev.cur].clone()

    def restore():
        lev.state[lev.cur].copy_(snap)

    # measured ALU peaks of this GPU (the roofline's FP32 and FP64 denominators)
    alu = measure_alu(stream.cuda_stream)
    # warm-up: W eager steps (the first one also runs the tile autotuner)
    plan.run(lev, a, dt, Wm, compute_dt0=True, use_graph=False)
    restore()
    # capture the K-step graph (first launch also warms it)
    plan.run(lev, a, dt, K, compute_dt0=True, use_graph=True)
    torch.cuda.synchronize()
    rc, flags = plan.status()
    if rc != H.NYX_OK:
        raise SystemExit(f"device status after warm-up: {rc} flags {flags}")
    plan.counters(reset=True)
    restore()

    # timed: K steps (one graph replay), inputs (>= 20 GB) far larger than L2
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.4)
    barrier(ws)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.run(lev, a, dt, K, compute_dt0=True, use_graph=True)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    launches = plan.counters(reset=True)["launches"]
    ms_max = max_over_ranks(ms, ws)
    value = ws * cells * K / (ms_max / 1e3)
    rc, flags = plan.status()
    if rc != H.NYX_OK:
        raise SystemExit(f"device status after the timed steps: {rc} flags {flags}")

    # dominant kernel: the fused advance, timed with events on its own stream
    restore()
    plan.profile(True)
    plan.run(lev, a, dt, K, compute_dt0=True, use_graph=False)
    prof = plan.counters(reset=True)
    plan.profile(False)
    rc, flags = plan.status()
    if rc != H.NYX_OK:
        raise SystemExit(f"device status after the profiled steps: {rc} flags {flags}")
    restore()
    adv_ms = prof["advance_ms"] / max(1, prof["timed_advances"])
    fill_ms = prof["fill_ms"] / max(1, prof["timed_fills"])
    flops = ALG_FLOPS_PER_ZONE[args.precision]
    shape, (tx, ty) = plan.tile_shape()
    tcls, ttrials, tlaunches = plan.tune_info()
    tuning = {"box_size_classes": tcls, "trial_launches": ttrials,
              "fused_launches_per_advance": tlaunches,
              "how": "per box-size class, one wave of work items per candidate (tile shape x "
                     "resident CTAs per SM); choices cached in a JSON file keyed by GPU, SM count, "
                     "precision, scheme variant and box extent (0 trials: all from the cache)"}

    # the workload's whole prescribed run (the large level: 100 steps, a from
    # 1/51 to 1/31) in one CUDA-graph replay from the initial state, with the
    # device status read at its end
    prescribed = None
    if not args.no_prescribed and w.nsteps > K:
        restore()
        nps = w.nsteps
        a_all = torch.tensor(a_schedule_for(w, nps), dtype=torch.float64, device="cuda")
        dt_all = torch.zeros(nps + 1, dtype=torch.float64, device="cuda")
        plan.run(lev, a_all, dt_all, nps, compute_dt0=True, use_graph=True)  # capture + first run
        torch.cuda.synchronize()
        restore()
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        plan.run(lev, a_all, dt_all, nps, compute_dt0=True, use_graph=True)
        p1.record(stream)
        torch.cuda.synchronize()
        pms = p0.elapsed_time(p1)
        prc, pflags = plan.status()
        prescribed = {"steps": nps, "a_first": float(a_all[0]), "a_last": float(a_all[nps]),
                      "status": prc, "status_flags": pflags,
                      "value": cells * nps / (pms / 1e3), "unit": "zone-updates/s",
                      "ms_per_step": pms / nps, "dt_first": float(dt_all[0]),
                      "dt_last": float(dt_all[nps - 1]),
                      "how": "one CUDA-graph replay of every step (ghost fill, fused advance, CFL "
                             "dt) from the initial state, timed with CUDA events"}
        if prc != H.NYX_OK:
            raise SystemExit(f"device status after the prescribed run: {prc} flags {pflags}")
        del a_all, dt_all
        restore()

    # end to end through the C ABI with pinned host buffers: the level's valid
    # cells in, the new valid cells and dt out, every step
    e2e = None
    if not args.no_e2e:
        restore()
        host_in = torch.from_numpy(plan.pack_valid(w.state)).pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        e2e_steps = max(1, min(3, K))
        d = plan.step_host_valid(lev, host_in, host_out, float(a_host[0]), float(a_host[1]), 0.0)
        torch.cuda.synchronize()
        barrier(ws)
        t0 = time.perf_counter()
        for s in range(e2e_steps):
            d = plan.step_host_valid(lev, host_in, host_out, float(a_host[s]), float(a_host[s + 1]),
                                     d)
        t_e2e = max_over_ranks(time.perf_counter() - t0, ws)
        state_bytes = host_in.numel() * 8
        e2e = {"value": ws * cells * e2e_steps / t_e2e, "unit": "zone-updates/s",
               "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes + 8,
               "steps": e2e_steps, "call": "nyx_hydro_step_host_valid (valid cells only)"}
        del host_in, host_out

    # scheme variants on the same level: the standalone corrector with a second
    # gravity field (Step 6 with g^{n+1}) and the fused advance with energy
    # option (ii) (Sec. 3.2), each timed with events on its plan's stream
    variants = {}
    if not args.no_variants:
        restore()
        g_new = lev.grav.clone()
        a1 = a[:2]
        dtv = dt[:1]
        plan.predict(lev, a1[:1], a1[1:], dtv, lev.grav)
        torch.cuda.synchronize()
        pred_snap = lev.state[1 - lev.cur].clone()
        reps = 3
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        tot = 0.0
        for r in range(reps):
            lev.state[1 - lev.cur].copy_(pred_snap)
            torch.cuda.synchronize()
            ev[0].record(stream)
            plan.correct(lev, a1[:1], a1[1:], dtv, lev.grav, g_new)
            ev[1].record(stream)
            torch.cuda.synchronize()
            tot += ev[0].elapsed_time(ev[1])
            lev.cur = 1 - lev.cur          # keep the state at t^n current
        c_ms = tot / reps
        gbs = CORRECT_BYTES_PER_ZONE * cells / (c_ms / 1e3) / 1e9
        f64 = CORRECT_FP64_FLOPS_PER_ZONE * cells / (c_ms / 1e3) / 1e12
        variants["corrector"] = {"ms": c_ms, "bound": "fp64",
                                 "alg_fp64_flops_per_zone": CORRECT_FP64_FLOPS_PER_ZONE,
                                 "achieved": f64, "peak": alu["fp64_fma_per_s"] / 1e12,
                                 "unit": "TFLOP/s", "frac": f64 / (alu["fp64_fma_per_s"] / 1e12),
                                 "peak_source": "measured FP64 instruction rate (nyx_alu_peak; "
                                                "one flop per non-FMA instruction)",
                                 "hbm": {"alg_bytes_per_zone": CORRECT_BYTES_PER_ZONE,
                                         "achieved_gbs": gbs, "peak_gbs": peaks["hbm_gbs"],
                                         "frac": gbs / peaks["hbm_gbs"]}}
        del pred_snap, g_new
        def one_advance(graph_steps=0, **kw):
            p2 = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl, precision=args.precision,
                        batching="persistent", **kw)
            p2.set_tile_shape(shape)
            l2 = H.Level(lev.state[0], lev.state[1], lev.grav, lev.cur)
            p2.advance(l2, a1[:1], a1[1:], dtv)
            torch.cuda.synchronize()
            l2.cur = lev.cur
            p2.profile(True)
            p2.advance(l2, a1[:1], a1[1:], dtv)
            pr2 = p2.counters(reset=True)
            p2.profile(False)
            torch.cuda.synchronize()
            rc2 = p2.status()
            step = None
            if graph_steps:
                # whole steps as the timed run takes them: a graph replay of
                # graph_steps steps (box groups: each group's ghost fill and
                # coefficient pass beside the other groups' advances)
                ag = a[:graph_steps + 1]
                dg = torch.zeros(graph_steps + 1, dtype=torch.float64, device="cuda")
                cur0 = l2.cur
                p2.run(l2, ag, dg, graph_steps, compute_dt0=True, use_graph=True)
                torch.cuda.synchronize()
                l2.cur = cur0
                g0 = torch.cuda.Event(enable_timing=True)
                g1 = torch.cuda.Event(enable_timing=True)
                g0.record(p2.torch_stream)
                p2.run(l2, ag, dg, graph_steps, compute_dt0=True, use_graph=True)
                g1.record(p2.torch_stream)
                torch.cuda.synchronize()
                gms = g0.elapsed_time(g1) / graph_steps
                step = {"ms_per_step": gms, "zone_updates_per_s": cells / (gms / 1e3),
                        "steps": graph_steps, "status": p2.status()[0],
                        "how": "graph replay of whole steps (CFL dt, ghost fill, coefficient "
                               "pass, advance), timed with CUDA events"}
            p2.close()
            ms2 = pr2["advance_ms"] / max(1, pr2["timed_advances"])
            out = {"advance_ms": ms2, "zone_updates_per_s": cells / (ms2 / 1e3),
                   "vs_default_advance_ms": adv_ms, "status": rc2[0]}
            if step is not None:
                out["graph_step"] = step
            if pr2["timed_flattens"]:
                fms = pr2["flatten_ms"] / pr2["timed_flattens"]
                fb = FLATTEN_BYTES_PER_ZONE[args.precision]
                gbs = fb * cells / (fms / 1e3) / 1e9
                out["zone_updates_per_s"] = cells / ((ms2 + fms) / 1e3)
                out["flatten_pass"] = {"ms": fms, "bound": "hbm", "alg_bytes_per_zone": fb,
                                       "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                       "frac": gbs / peaks["hbm_gbs"]}
            return out

        r2 = one_advance(grav_energy=1)
        rf2 = roofline_of(r2["advance_ms"], cells, args.precision, peaks, peak_src, alu,
                          "fused advance, energy option (ii)")
        r2.update(bound=rf2["bound"], achieved=rf2["achieved"], peak=rf2["peak"],
                  unit=rf2["unit"], frac=rf2["frac"])
        variants["energy_option_ii"] = r2
        # PLM and the linearised solver do fewer operations than the
        # algorithmic count above, so only their times and rates are reported
        variants["plm"] = one_advance(reconstruction="plm")
        variants["linearised_riemann"] = one_advance(riemann_solver="linear")
        # shock flattening: the coefficient pass, then the advance reading it
        variants["flattening"] = one_advance(graph_steps=K, flattening=True)

    # FP64 forms on the same workload (one step each), for the FP32-vs-FP64
    # comparison; the mixed step's per-field error against the FP64 step from
    # the same state with the same dt
    side = {}
    errors = None
    if not args.no_fp64:
        restore()
        lm = H.Level(lev.state[0], lev.state[1], lev.grav, lev.cur)
        plan.run(lm, a, dt, 1, compute_dt0=True, use_graph=False)
        torch.cuda.synchronize()
        mixed_new = lm.state[lm.cur].clone()
        dt0 = dt[:1].clone()
        for label, batching in (("fp64_persistent", "persistent"), ("fp64_per_box", "per_box")):
            restore()
            p64 = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl, precision="fp64", batching=batching)
            l64 = H.Level(lev.state[0], lev.state[1], lev.grav, lev.cur)
            dt[:1].copy_(dt0)
            p64.run(l64, a, dt, 1, compute_dt0=False, use_graph=False)
            torch.cuda.synchronize()
            if label == "fp64_persistent":
                errors = {"reference": "the FP64 persistent form, one step from the same state "
                                       "and dt (bit for bit the FP64 oracle's arithmetic)",
                          "metric": "normwise relative over the valid cells: max|d|/max|ref| "
                                    "and sum|d|/sum|ref|",
                          "fields": field_errors(plan, w.level, mixed_new, l64.state[l64.cur])}
                del mixed_new
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            f0.record(p64.torch_stream)
            p64.run(l64, a, dt, 1, compute_dt0=True, use_graph=False)
            f1.record(p64.torch_stream)
            torch.cuda.synchronize()
            zps = cells / (f0.elapsed_time(f1) / 1e3)
            tf = ALG_FLOPS_PER_ZONE["fp64"] * zps / 1e12
            side[label] = {"value": zps, "unit": "zone-updates/s", "steps": 1,
                           "roofline": {"bound": "fp64", "achieved": tf,
                                        "peak": alu["fp64_tflops"], "unit": "TFLOP/s",
                                        "frac": tf / alu["fp64_tflops"],
                                        "peak_source": "measured (nyx_alu_peak)",
                                        "alg_flops_per_zone": ALG_FLOPS_PER_ZONE["fp64"],
                                        "note": "whole step (fill, advance, dt) timed"}}
            p64.close()

    # the 256^3 sigma = 1 box over its 50 prescribed steps: the mixed path's
    # per-field error against the FP64 path (itself the oracle's arithmetic,
    # bit for bit), both persistent and graph-captured
    m256 = None
    if not args.no_mixed256 and args.workload == "large" and args.precision == "mixed":
        m256 = mixed256_errors(H, torch)

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = oracle_sample(args.workload, w, budget_s=args.cpu_budget)
        one = oracle_sample(args.workload, w, budget_s=0.5 * args.cpu_budget, threads=1)
        cpu["single_thread"] = {"value": one["value"], "unit": one["unit"], "cores": 1,
                                "sample": one["sample"]}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "zone-updates/s", "n_gpus": ws,
            "steps": K, "warmup": Wm, "ms_per_step": ms_max / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": args.workload, "level": w.name, "valid_cells": cells,
                       "boxes": w.level.nbox, "precision": args.precision,
                       "batching": "persistent + CUDA graph; box groups, each group's ghost "
                                   "fill beside the other groups' advances",
                       "tile": [tx, ty],
                       "l2": "inputs larger than L2 (state + gravity > 20 GB)",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU"},
            "roofline": roofline_of(
                adv_ms, cells, args.precision, peaks, peak_src, alu,
                ("k_fused2 (task form)" if shape >= 3 else
                 f"k_fused<{'float' if args.precision == 'mixed' else 'double'}>"),
                traffic=(args.traffic_per_zone * cells if args.traffic_per_zone else
                         (TRAFFIC_BYTES_PER_ZONE[(args.workload, shape)] * cells
                          if args.precision == "mixed" and
                          (args.workload, shape) in TRAFFIC_BYTES_PER_ZONE else None))),
            "alu_peaks": alu,
            "hbm_nominal": {"peak": NOMINAL_HBM_GBS,
                            "frac": ALG_BYTES_PER_ZONE * cells / (adv_ms / 1e3) / 1e9 /
                            NOMINAL_HBM_GBS},
            "kernel_ms": {"advance": adv_ms, "ghost_fill": fill_ms},
            "variants": variants,
            "fp64_comparison": side,
            "mixed_vs_fp64": errors,
            "prescribed_run": prescribed,
            "autotune": tuning,
            "mixed256_50_steps": m256,
            "clocks": clk,
            "e2e": e2e,
            "gpu_launches": launches,
            "cpu_baseline": cpu,
        }
        print(json.dumps(out), flush=True)
    plan.close()


# ---------------------------------------------------------------------- two levels

# Algorithmic bytes of the coupling kernels: interpolation writes the 6
# doubles of a fine ghost cell (the coarse cells it reads are shared by 8 fine
# cells: 6 more bytes); reflux reads 4 fine and 1 coarse flux of 6 doubles and
# reads and writes the coarse cell (336 B per coarse face); average down reads
# 8 fine cells and writes one coarse cell (432 B per coarse cell).
AMR_BYTES = {"interp": 54, "reflux": 336, "avgdown": 432}
# One cycle of the self-gravity solve per fine cell.  FP64: 4 red-black
# sweeps (read phi and f, write phi: 24 B each), the residual restriction
# (16 B), the prolongation (24 B) and the residual norm (16 B), times 8/7 for
# the coarser grids: 174 B.  Mixed (iterative refinement): the FP32 V-cycle
# (4 sweeps of 12 B, restriction 8 B, prolongation 12 B, times 8/7: 78 B),
# the FP64 residual with its float copy and e = 0 (24 B), the FP64 update of
# phi (20 B): 122 B.
VCYCLE_BYTES_PER_CELL = {"fp64": 174, "mixed": 122}


def oracle_amr_sample(w, budget_s=12.0):
    """Time the FP64 CPU oracle's two-level step on a bounded sample: a
    64^3 periodic coarse level (8 boxes of 32^3) with one of them refined by
    2 (the large coupled level's box sizes), steps until the budget."""
    import oracle
    cw = w.coarse
    P = oracle.OracleParams(gamma=cw.gamma, cfl=cw.cfl)
    cs = [s.copy() for s in cw.state]
    oracle.fill_ghosts(cw.level, cs)
    fs = oracle.amr_interp(cw.level, cs, w.fine,
                           [np.zeros(w.fine.shape(b, 6)) for b in range(w.fine.nbox)], "all")
    cg = [g.copy() for g in cw.grav]
    oracle.fill_ghosts(cw.level, cg)
    fg = oracle.amr_interp(cw.level, cg, w.fine,
                           [np.zeros(w.fine.shape(b, 3)) for b in range(w.fine.nbox)], "all")
    cells = cw.level.valid_cells() + w.fine.valid_cells()
    a0, a1 = float(cw.a_sched[0]), float(cw.a_sched[1])
    elapsed, steps = 0.0, 0
    while elapsed < budget_s:
        t0 = time.perf_counter()
        dt = oracle.amr_estdt(cw.level, w.fine, P, cs, fs, a0)
        cs, fs, _, _ = oracle.amr_step(cw.level, w.fine, P, cs, fs, cg, fg, a_old=a0, a_new=a1,
                                       dt=dt)
        elapsed += time.perf_counter() - t0
        steps += 1
    return {"value": cells * steps / elapsed, "unit": "zone-updates/s", "cores": os.cpu_count(),
            "kind": "oracle", "elapsed_s": elapsed / steps,
            "sample": f"{steps} two-level step(s) of a 64^3 coarse level (8 boxes of 32^3) with one "
                      f"box refined by 2 ({cells} cells), FP64 oracle, OpenMP on all host cores; "
                      f"{elapsed:.1f} s"}


def run_reference_amr(args, w):
    ws, rank, _ = dist_setup(args.gpus)
    if rank != 0:
        return
    per = []
    info = None
    for s in range(args.warmup + args.steps):
        r = oracle_amr_sample(w, budget_s=args.ref_budget)
        if s >= args.warmup:
            per.append(r)
        info = r
    value = statistics.median(x["value"] for x in per)
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "zone-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.median(x["elapsed_s"] for x in per) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "level": w.name, "sample": info["sample"]},
        "cpu_baseline": {"value": value, "unit": "zone-updates/s", "cores": info["cores"],
                         "kind": "oracle", "sample": info["sample"]},
        "e2e": {"value": value, "unit": "zone-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def run_amr(args, aw):
    """Two-level steps (coarse advance, fine ghosts from the coarse level,
    fine advance, reflux, average down, shared CFL dt) of a coupled
    hierarchy; zone-updates count the valid cells of both levels."""
    import torch
    from paper_1301_4498_gb300 import hydro as H
    ws, rank, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    peaks, peak_src = load_peaks()
    K, Wm = args.steps, args.warmup
    cw = aw.coarse
    cells_c, cells_f = cw.level.valid_cells(), aw.fine.valid_cells()
    cells = cells_c + cells_f
    kw = dict(gamma=cw.gamma, cfl=cw.cfl, precision=args.precision, batching="persistent",
              autotune=1 if args.autotune else 0, keep_fluxes=args.keep_fluxes)
    cp = H.Plan(cw.level, **kw)
    fp = H.Plan(aw.fine, stream=cp.torch_stream, coarse_fine=1, **kw)
    if args.tile_shape >= 0:
        cp.set_tile_shape(args.tile_shape)
        fp.set_tile_shape(args.tile_shape)
    amr = H.Amr(cp, fp)
    lc = H.make_level(cp, cw.state, cw.grav)
    cp.fill(lc.current, 6)
    fs0 = fp.empty_field(6)
    amr.interp(lc.current, fs0, 6, "all")       # newly refined data: interpolated (Sec. 4.1)
    fg = fp.empty_field(3)
    amr.interp(lc.grav, fg, 3, "all")
    lf = H.Level(fs0, fp.empty_field(6), fg)
    a_host = a_schedule_for(cw, max(K, Wm) + 1)
    a = torch.tensor(a_host, dtype=torch.float64, device="cuda")
    dt = torch.zeros(len(a_host), dtype=torch.float64, device="cuda")
    stream = cp.torch_stream

    amr.run(lc, lf, a, dt, Wm, compute_dt0=True, use_graph=False)
    amr.run(lc, lf, a, dt, K, compute_dt0=True, use_graph=True)
    torch.cuda.synchronize()
    for p in (cp, fp):
        rc, flags = p.status()
        if rc != H.NYX_OK:
            raise SystemExit(f"device status after warm-up: {rc} flags {flags}")
    cp.counters(reset=True)
    fp.counters(reset=True)

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.4)
    barrier(ws)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    amr.run(lc, lf, a, dt, K, compute_dt0=True, use_graph=True)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    launches = cp.counters(reset=True)["launches"] + fp.counters(reset=True)["launches"]
    ms_max = max_over_ranks(ms, ws)
    value = ws * cells * K / (ms_max / 1e3)

    # the fused advances (both levels) and the coupling kernels, each timed
    # with events on the plans' stream in eager steps
    cp.profile(True)
    fp.profile(True)
    amr.run(lc, lf, a, dt, K, compute_dt0=True, use_graph=False)
    pc, pf = cp.counters(reset=True), fp.counters(reset=True)
    cp.profile(False)
    fp.profile(False)
    adv_c = pc["advance_ms"] / max(1, pc["timed_advances"])
    adv_f = pf["advance_ms"] / max(1, pf["timed_advances"])

    def timed(fn, reps=5):
        fn()
        q0 = torch.cuda.Event(enable_timing=True)
        q1 = torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        for _ in range(reps):
            fn()
        q1.record(stream)
        torch.cuda.synchronize()
        return q0.elapsed_time(q1) / reps

    scratch_c = lc.state[1 - lc.cur].clone()
    scratch_f = lf.current.clone()
    t_interp = timed(lambda: amr.interp(lc.current, scratch_f, 6, "ghosts"))
    t_reflux = timed(lambda: amr.reflux(scratch_c))
    t_avg = timed(lambda: amr.average_down(lf.current, scratch_c, 6))
    del scratch_c, scratch_f
    nghost = sum(int(np.prod(np.array(aw.fine.shape(b, 1)[1:]))) - int(np.prod(aw.fine.extent(b)))
                 for b in range(aw.fine.nbox))
    nface = 0
    for b in range(aw.fine.nbox):
        hx, hy, hz = (e // 2 for e in aw.fine.extent(b))
        nface += 2 * (hy * hz + hx * hz + hx * hy)   # coarse faces around the fine box
    ncov = cells_f // 8
    coupling = {}
    for name, ms_k, units in (("interp", t_interp, nghost), ("reflux", t_reflux, nface),
                              ("avgdown", t_avg, ncov)):
        gbs = AMR_BYTES[name] * units / (ms_k / 1e3) / 1e9
        coupling[name] = {"ms": ms_k, "units": units, "alg_bytes_per_unit": AMR_BYTES[name],
                          "achieved_gbs": gbs, "frac_hbm": gbs / peaks["hbm_gbs"]}
    # self-gravity of the coarse level (one periodic 512^3 domain): a cold
    # solve and a warm re-solve; the V-cycle cost is their difference per cycle
    gravity = None
    if not args.no_variants:
        ps = H.Poisson(cp, four_pi_G=1.0, precision=args.precision)
        gtmp = cp.empty_field(3)
        ps.solve(lc.current, float(a_host[0]), gtmp, warm_start=False)   # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cyc, res = ps.solve(lc.current, float(a_host[0]), gtmp, warm_start=False)
        t_cold = time.perf_counter() - t0
        t0 = time.perf_counter()
        cyc0, _ = ps.solve(lc.current, float(a_host[0]), gtmp, warm_start=True)
        t_warm = time.perf_counter() - t0
        per_cycle = (t_cold - t_warm) / max(1, cyc)
        vb = VCYCLE_BYTES_PER_CELL[args.precision]
        gbs = vb * cells_c / per_cycle / 1e9
        gravity = {"cells": cells_c, "cold_solve_ms": t_cold * 1e3, "cycles": cyc,
                   "relative_residual": res, "warm_resolve_ms": t_warm * 1e3,
                   "warm_cycles": cyc0, "vcycle_ms": per_cycle * 1e3,
                   "vcycle_alg_bytes_per_cell": vb, "precision": args.precision,
                   "achieved_gbs": gbs, "frac_hbm": gbs / peaks["hbm_gbs"], "bound": "hbm"}
        ps.close()
        del gtmp
    adv_ms = adv_c + adv_f
    alu = measure_alu(stream.cuda_stream)
    shape, (tx, ty) = cp.tile_shape()

    e2e = None
    if not args.no_e2e:
        hc_in = lc.current.cpu().pin_memory()
        hf_in = lf.current.cpu().pin_memory()
        hc_out = torch.empty_like(hc_in).pin_memory()
        hf_out = torch.empty_like(hf_in).pin_memory()
        e2e_steps = max(1, min(3, K))
        torch.cuda.synchronize()
        barrier(ws)
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for s in range(e2e_steps):
                lc.current.copy_(hc_in, non_blocking=True)
                lf.current.copy_(hf_in, non_blocking=True)
                amr.step(lc, lf, a[s:s + 1], a[s + 1:s + 2], dt[s:s + 1], dt[s + 1:s + 2])
                hc_out.copy_(lc.current, non_blocking=True)
                hf_out.copy_(lf.current, non_blocking=True)
            stream.synchronize()
        t_e2e = max_over_ranks(time.perf_counter() - t0, ws)
        nbytes = (hc_in.numel() + hf_in.numel()) * 8
        e2e = {"value": ws * cells * e2e_steps / t_e2e, "unit": "zone-updates/s",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "steps": e2e_steps}
        del hc_in, hf_in, hc_out, hf_out

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = oracle_amr_sample(make_workload(args.workload, sample_only=True),
                                budget_s=args.cpu_budget)
        cpu.pop("elapsed_s", None)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "zone-updates/s", "n_gpus": ws,
            "steps": K, "warmup": Wm, "ms_per_step": ms_max / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": args.workload, "level": aw.name, "valid_cells": cells,
                       "coarse_cells": cells_c, "fine_cells": cells_f,
                       "boxes": [cw.level.nbox, aw.fine.nbox], "precision": args.precision,
                       "batching": "persistent + CUDA graph, two levels, no subcycling",
                       "keep_fluxes": args.keep_fluxes, "tile": [tx, ty],
                       "l2": "inputs larger than L2 (state + gravity > 20 GB)",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU"},
            "roofline": roofline_of(adv_ms, cells, args.precision, peaks, peak_src, alu,
                                    "fused advance of both levels"),
            "alu_peaks": alu,
            "kernel_ms": {"advance_coarse": adv_c, "advance_fine": adv_f,
                          "ghost_fill_coarse": pc["fill_ms"] / max(1, pc["timed_fills"]),
                          "ghost_fill_fine": pf["fill_ms"] / max(1, pf["timed_fills"])},
            "coupling": coupling,
            "self_gravity": gravity,
            "clocks": clk,
            "e2e": e2e,
            "gpu_launches": launches,
            "cpu_baseline": cpu,
        }
        print(json.dumps(out), flush=True)
    amr.close()
    fp.close()
    cp.close()


# ---------------------------------------------------------------------- self-gravity + dark matter

def oracle_cosmo_step(w, P, PP, cs, x, u, m, phi, a0, a1, gd0=None):
    """One step of the single-level algorithm with gas, dark matter and
    self-gravity on the oracle (Steps 1-6; Step 1 from scratch when gd0 is
    None).  Returns (state, x, u, phi, dense g at t^{n+1})."""
    import oracle
    n = tuple(int(v) for v in (w.level.dom_hi[0] - w.level.dom_lo[0] + 1))
    dx = float(w.level.dx[0][0])
    ah = 0.5 * (a0 + a1)
    rho0 = oracle.pm_deposit(n, dx, x, m)
    phi, gl0, _, gd0 = oracle.poisson_solve(w.level, PP, cs, a0, phi, rho_dm=rho0,
                                            want_dense_g=True)
    oracle.fill_ghosts(w.level, gl0)
    dt = min(oracle.estdt(w.level, P, cs, a0), oracle.pm_estdt(n, dx, gd0, x, u, a0))
    pred, _ = oracle.predict(w.level, P, cs, gl0, a_old=a0, a_new=a1, dt=dt)
    x1, uh = oracle.pm_kick_drift(n, dx, gd0, x, u, a_old=a0, a_half=ah, dt=dt)
    rho1 = oracle.pm_deposit(n, dx, x1, m)
    phi, gl1, _, gd1 = oracle.poisson_solve(w.level, PP, pred, a1, phi, rho_dm=rho1,
                                            want_dense_g=True)
    oracle.fill_ghosts(w.level, gl1)
    u1 = oracle.pm_kick(n, dx, gd1, x1, uh, a_half=ah, a_new=a1, dt=dt)
    new, _ = oracle.correct(w.level, P, cs, pred, gl0, gl1, a_old=a0, a_new=a1, dt=dt)
    return new, x1, u1, phi, gd1


def oracle_cosmo_sample(budget_s=12.0):
    """The oracle's full step on a 64^3 sample (gas + 64^3 particles)."""
    import oracle
    w = make_workload("cosmo", sample_only=True)
    x, u, m = w.level.meta["dm"]
    P = oracle.OracleParams(gamma=w.gamma, cfl=w.cfl)
    PP = oracle.PoissonParams(four_pi_G=COSMO_FOUR_PI_G)
    cs, phi = w.state, None
    a0, a1 = float(w.a_sched[0]), float(w.a_sched[1])
    elapsed, steps = 0.0, 0
    while elapsed < budget_s:
        t0 = time.perf_counter()
        cs, x, u, phi, _ = oracle_cosmo_step(w, P, PP, cs, x, u, m, phi, a0, a1)
        elapsed += time.perf_counter() - t0
        steps += 1
    cells = w.level.valid_cells()
    return {"value": cells * steps / elapsed, "unit": "zone-updates/s", "cores": os.cpu_count(),
            "kind": "oracle", "elapsed_s": elapsed / steps,
            "sample": f"{steps} step(s) of gas + dark matter + self-gravity on a 64^3 level "
                      f"(8 boxes of 32^3, {m.size} particles), FP64 oracle, OpenMP on all host "
                      f"cores; {elapsed:.1f} s"}


def run_reference_cosmo(args, w):
    ws, rank, _ = dist_setup(args.gpus)
    if rank != 0:
        return
    per = []
    info = None
    for s in range(args.warmup + args.steps):
        r = oracle_cosmo_sample(budget_s=args.ref_budget)
        if s >= args.warmup:
            per.append(r)
        info = r
    value = statistics.median(x["value"] for x in per)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "zone-updates/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": statistics.median(x["elapsed_s"] for x in per) * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": args.workload, "level": w.name, "sample": info["sample"]},
           "cpu_baseline": {"value": value, "unit": "zone-updates/s", "cores": info["cores"],
                            "kind": "oracle", "sample": info["sample"]},
           "e2e": {"value": value, "unit": "zone-updates/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_cosmo(args, w):
    """The single-level algorithm with gas, dark matter and self-gravity
    (Sec. 3.6 Steps 1-6): per step the particle and gas time steps, the gas
    predictor with g^n, kick-drift, deposit at x^{n+1}, the Poisson solve on
    rho_b^{n+1,*} + rho_dm^{n+1} (warm start), kick, the gas corrector with
    g^{n+1}; g^n of the next step is this step's g^{n+1} (Step 1 shortcut).
    Host-driven: the solve reads its residual after every V-cycle."""
    import torch
    from paper_1301_4498_gb300 import hydro as H
    ws, rank, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    peaks, peak_src = load_peaks()
    K, Wm = args.steps, args.warmup
    cells = w.level.valid_cells()
    x, u, m = w.level.meta["dm"]
    npart = m.size
    plan = H.Plan(w.level, gamma=w.gamma, cfl=w.cfl, precision=args.precision,
                  batching="persistent", autotune=1 if args.autotune else 0)
    if args.tile_shape >= 0:
        plan.set_tile_shape(args.tile_shape)
    lev = H.make_level(plan, w.state, None)
    # mixed plans solve by iterative refinement (FP64 residual and update
    # around FP32 V-cycles), to the same FP64 stopping test
    ps = H.Poisson(plan, four_pi_G=COSMO_FOUR_PI_G, precision=args.precision)
    xd, ud, md = (torch.tensor(v, device="cuda") for v in (x, u, m))
    rho = ps.dense(1)[0]
    gd = ps.dense(3)
    g_old, g_new = plan.empty_field(3), plan.empty_field(3)
    a_host = a_schedule_for(w, Wm + K + 1)
    a = torch.tensor(a_host, dtype=torch.float64, device="cuda")
    dts = torch.zeros(3, dtype=torch.float64, device="cuda")
    stream = plan.torch_stream
    # Step 1 of the first step: g^0 from scratch
    ps.pm_deposit(xd, md, rho)
    ps.solve(lev.current, float(a_host[0]), g_old, warm_start=False, rho_dm=rho, g_dense=gd)
    timing = {"gas_advance": 0.0, "particles": 0.0, "solve": 0.0, "corrector": 0.0}
    cyc_total = 0

    pdt_ready = [False]   # dts[1] holds this step's particle dt (from the last kick)

    def step(s, record):
        nonlocal g_old, g_new, cyc_total
        a0, a1 = float(a_host[s]), float(a_host[s + 1])
        ah = 0.5 * (a0 + a1)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        plan.estdt(lev, a[s:s + 1], dts[0:1])
        if not pdt_ready[0]:
            ps.pm_estdt(xd, ud, gd, a0, dts[1:2])
        torch.minimum(dts[0:1], dts[1:2], out=dts[2:3])
        dt = float(dts[2].item())
        ev[0].record(stream)
        plan.predict(lev, a[s:s + 1], a[s + 1:s + 2], dts[2:3], g_old)
        ev[1].record(stream)
        ps.pm_kick_drift(xd, ud, gd, a0, ah, dt)
        ps.pm_deposit(xd, md, rho)
        ev[2].record(stream)
        cyc, _ = ps.solve(lev.state[1 - lev.cur], a1, g_new, warm_start=True, rho_dm=rho,
                          g_dense=gd)
        ev[3].record(stream)
        # Step 5 with the next step's particle dt from the kicked particles
        ps.pm_kick_estdt(xd, ud, gd, ah, a1, dt, dts[1:2])
        pdt_ready[0] = True
        ev[4].record(stream)
        plan.correct(lev, a[s:s + 1], a[s + 1:s + 2], dts[2:3], g_old, g_new)
        ev[5].record(stream)
        g_old, g_new = g_new, g_old
        if record:
            torch.cuda.synchronize()
            timing["gas_advance"] += ev[0].elapsed_time(ev[1])
            timing["particles"] += ev[1].elapsed_time(ev[2]) + ev[3].elapsed_time(ev[4])
            timing["solve"] += ev[2].elapsed_time(ev[3])
            timing["corrector"] += ev[4].elapsed_time(ev[5])
            cyc_total += cyc

    for s in range(Wm):
        step(s, False)
    torch.cuda.synchronize()
    rc, flags = plan.status()
    if rc != H.NYX_OK:
        raise SystemExit(f"device status after warm-up: {rc} flags {flags}")
    plan.counters(reset=True)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.4)
    barrier(ws)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in range(Wm, Wm + K):
        step(s, True)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    launches = plan.counters(reset=True)["launches"]
    ms_max = max_over_ranks(ms, ws)
    value = ws * cells * K / (ms_max / 1e3)
    adv_ms = timing["gas_advance"] / K
    alu = measure_alu(plan.torch_stream.cuda_stream)
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = oracle_cosmo_sample(budget_s=args.cpu_budget)
        cpu.pop("elapsed_s", None)
    shape, (tx, ty) = plan.tile_shape()
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "zone-updates/s", "n_gpus": ws,
            "steps": K, "warmup": Wm, "ms_per_step": ms_max / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": args.workload, "level": w.name, "valid_cells": cells,
                       "particles": npart, "boxes": w.level.nbox, "precision": args.precision,
                       "step": "Sec. 3.6 Steps 1-6 (g^n from the previous Step 4)",
                       "poisson": ("iterative refinement: FP64 residual and update, FP32 "
                                   "V-cycles" if args.precision == "mixed"
                                   else "FP64 V-cycles"),
                       "tile": [tx, ty], "l2": "inputs larger than L2",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU"},
            "particle_updates_per_s": ws * npart * K / (ms_max / 1e3),
            "roofline": roofline_of(adv_ms, cells, args.precision, peaks, peak_src, alu,
                                    "fused gas predictor (k_fused2)"),
            "alu_peaks": alu,
            "breakdown_ms_per_step": {k: v / K for k, v in timing.items()},
            "poisson_cycles_per_step": cyc_total / K,
            "clocks": clk, "e2e": None, "gpu_launches": launches, "cpu_baseline": cpu,
        }
        print(json.dumps(out), flush=True)
    ps.close()
    plan.close()


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="large",
                    choices=["large", "large128", "comoving128", "uneven512", "uneven64", "mixed256",
                             "sod", "amr", "amr128", "cosmo", "cosmo128"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--autotune", type=int, default=1)
    ap.add_argument("--tile-shape", type=int, default=-1,
                    help="fix the fused kernel's tile shape (see nyx_hydro_tile_shape)")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-prescribed", action="store_true",
                    help="skip the workload's whole prescribed run (100 steps on the large level)")
    ap.add_argument("--no-mixed256", action="store_true",
                    help="skip the 256^3 sigma = 1 box's 50-step mixed-vs-FP64 error leg")
    ap.add_argument("--traffic-per-zone", type=float, default=0.0,
                    help="DRAM bytes per zone of the advance kernel from an ncu capture")
    ap.add_argument("--keep-fluxes", type=int, default=1,
                    help="two-level workloads: 1 keep every face's flux, 2 box faces only")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--ref-budget", type=float, default=6.0)
    ap.add_argument("--ref-boxes", type=int, default=0)
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    w = make_workload(args.workload, sample_only=args.impl == "reference")
    if "dm" in w.level.meta if hasattr(w, "level") else False:
        if args.impl == "reference":
            run_reference_cosmo(args, w)
        else:
            run_cosmo(args, w)
    elif isinstance(w, W.AmrWorkload):
        if args.impl == "reference":
            run_reference_amr(args, w)
        else:
            run_amr(args, w)
    elif args.impl == "reference":
        run_reference(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
