"""Benchmark of the sliding-mesh SD hot path: SSP-RK3 steps of the residual
(SP->FP interpolation, ALE fluxes, Rusanov faces, curved dynamic mortars,
divergence, RK update) on one GPU per rank, through the C ABI.

Workload (default): vortex through a rotor -- periodic [-20,20]^2, rotating
disk r<=4 at omega=0.5, 246,900 quads, N=6 (p=5), Euler, strength-5
isentropic vortex; 8.9M solution points x 4 variables.  The state (284 MB)
is larger than L2, so no flush is needed between steps.

One step = three SSP-RK3 stages; metric = DOF-updates/s = E * N^2 * 4 *
steps / time.  ``--impl reference`` times the plain C FP64 oracle on the host
cores instead (a bounded sample of the same workload family).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from ssd_inputs import fields, meshes  # noqa: E402
from ssd_inputs.workloads import FlowParams, build_workload  # noqa: E402

METRIC = "DOF-updates/s (FP32 & batched vs FP64 GPU) at stated L2 error; % HBM roofline"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
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
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# DRAM bytes (read + write) per launch of the FP32 volume kernel on this
# workload (mean of the three stage launches of one step), from one ncu
# capture of dram__bytes_read.sum + dram__bytes_write.sum; valid only for the
# kernel source it was taken on: SHA-256 of the engine text that k_volume is
# built from (its helpers, the ElemGeo metrics and VolCfg, from the start of
# the engine header through the end of k_volume); otherwise null.
PROFILED_TRAFFIC = {"bytes": (389.3e6 + 329.1e6 + 673.7e6 + 330.8e6 + 673.6e6 + 329.5e6) / 3,
                    "kernel_sha256": "08c0c761564d75e3ec7ff3855a811e014f811251ac5c17f80dc192a794330087"}


def volume_kernel_source():
    path = os.path.join(ROOT, "paper_1503_02198_gb300", "csrc", "ssd_engine.cuh")
    try:
        text = open(path, encoding="utf-8").read()
    except OSError:
        return None
    d = text.index('#include "ssd_viscous.cuh"')
    return text[:d]


def profiled_traffic():
    import hashlib
    src = volume_kernel_source()
    if src is None:
        return None
    h = hashlib.sha256(src.encode("utf-8")).hexdigest()
    return PROFILED_TRAFFIC["bytes"] if h == PROFILED_TRAFFIC["kernel_sha256"] else None


def volume_bytes_per_element(N, w_c, w_s=8):
    """Algorithmic bytes one volume launch moves per element (see design
    notes): state read + write (w_s bytes per value: 8 for the FP64 or
    double-float state, 4 for FP32 state storage), the Runge-Kutta base read
    on two of the three stages, the common-flux read and the new traces
    written (16 N values each in the compute word), 4 corner nodes (16 B each)
    and the zone tag."""
    state = 4 * N * N * w_s
    return state * (2 + 2.0 / 3.0) + 2 * 16 * N * w_c + 4 * 16 + 4


def volume_flops_per_element(N):
    """FP64 floating-point operations one element takes in the volume kernel
    in a Runge-Kutta stage with a base state, counted from the kernel (an FMA
    counts 2).  Per SP line (2 N of them): at each of the N - 1 interior flux
    points the rotated metric vector (6), the interpolation of 4 variables
    (8 N) and the transformed ALE flux (28: pressure 7, normal velocity 4,
    the four flux components 3 + 5 + 5 + 4, besides one reciprocal); at all
    N + 1 flux points the divergence into N SPs (8 N); the face traces of the
    new state (16 N).  Per SP: the residual and the Runge-Kutta combination
    of 4 variables (7 each) and the positivity check (6, besides one
    division).  Divisions / reciprocals, (N - 1) per line and one per SP, are
    not counted."""
    per_line = (N - 1) * (6 + 8 * N + 28) + (N + 1) * 8 * N + 16 * N
    return 2 * N * per_line + N * N * 34


def interface_fraction(prof):
    """Share of a step spent on sliding-interface work, the paper's
    "interface" time (Tables 3-10): the stage clock and mortar merge and the
    mortar projections with their common flux, each timed as its own launch
    by sd_profile_step (per stage; three stages a step; the sum over each
    face's mortars runs inside the volume kernel and is not counted)."""
    return (prof["merge"] + prof["mortar"]) * 3 / prof["step"]


def launches_per_step(mesh, viscous=0):
    """Kernels of one captured SSP-RK3 step: on the side branch, beside the
    whole step, the merge of the next step's three stages (clocks and mortar
    tables), the launch forming their mortar offsets (Eq. xz) and the clock
    advance; per stage the face kernel (conforming and boundary points, and
    the mortar flux when the mesh has an interface, in one launch) and the
    volume kernel (which sums the mortar contributions of its interface faces
    itself), plus for a viscous stage the common-solution face kernel (with
    its mortar flux) and the gradient-trace kernel.  (Each sd_step call adds
    the two launches merging its first step.)"""
    per_stage = 2 + (2 if viscous else 0)
    return 3 + 3 * per_stage


SAMPLE_LADDER = (  # (n_cart, n_hole, n_core, n_ring_in, n_ring_out) of the rotor family
    (90, 22, 10, 4, 2), (60, 16, 8, 3, 2), (40, 12, 6, 2, 2), (28, 10, 4, 2, 1))


def sample_workload(level=0):
    """Bounded sample of the rotor workload family for the CPU oracle: same
    generator and N, coarser mesh (level 0: 7,950 quads)."""
    nc, nh, nk, ri, ro = SAMPLE_LADDER[level]
    return meshes.rotor_mesh(half_width=20.0, n_cart=nc, n_hole=nh, r_interface=4.0, n_core=nk,
                             core_half=2.0, n_ring_in=ri, n_ring_out=ro)


def cpu_oracle_rate(steps, warmup, dt, budget_s=None):
    """Oracle SSP-RK3 steps on a sample mesh; with a time budget the sample
    is the largest ladder mesh whose estimated (steps + warmup) time fits."""
    import oracle
    oracle.build()
    w = build_workload("rotor_n6")
    level = 0
    if budget_s is not None:
        probe = sample_workload(len(SAMPLE_LADDER) - 1)
        op = oracle.Oracle(probe, w.N, w.params)
        Qp = op.state_from(lambda x, y: fields.isentropic_vortex(x, y))
        t0 = time.perf_counter()
        op.step(Qp, 0.0, dt, 1)
        per_elem = (time.perf_counter() - t0) / len(probe["elem_nodes"])
        level = len(SAMPLE_LADDER) - 1
        for lv in range(len(SAMPLE_LADDER)):
            nc, nh = SAMPLE_LADDER[lv][0], SAMPLE_LADDER[lv][1]
            est_E = nc * nc - nh * nh + 4 * nh * SAMPLE_LADDER[lv][4] + (SAMPLE_LADDER[lv][2] ** 2) * 5
            if est_E * per_elem * (steps + warmup) <= budget_s:
                level = lv
                break
    mesh = sample_workload(level)
    orc = oracle.Oracle(mesh, w.N, w.params)
    Q = orc.state_from(lambda x, y: fields.isentropic_vortex(x, y))
    t = 0.0
    for _ in range(warmup):
        Q, t = orc.step(Q, t, dt, 1)
    t0 = time.perf_counter()
    for _ in range(steps):
        Q, t = orc.step(Q, t, dt, 1)
    el = time.perf_counter() - t0
    E = len(mesh["elem_nodes"])
    rate = E * w.N * w.N * 4 * steps / el
    return rate, el, E, level


def _oracle_sample(args):
    """Worker of the all-cores CPU baseline (a process of its own): warmup +
    steps oracle SSP-RK3 steps on the rotor-family sample mesh at a ladder
    level; returns (DOF-updates done in the timed steps, their seconds)."""
    steps, warmup, dt, level, N, prm = args
    import oracle
    mesh = sample_workload(level)
    orc = oracle.Oracle(mesh, N, prm)
    Q = orc.state_from(lambda x, y: fields.isentropic_vortex(x, y))
    t = 0.0
    for _ in range(warmup):
        Q, t = orc.step(Q, t, dt, 1)
    t0 = time.perf_counter()
    for _ in range(steps):
        Q, t = orc.step(Q, t, dt, 1)
    return len(mesh["elem_nodes"]) * N * N * 4 * steps, time.perf_counter() - t0


def cpu_oracle_rate_all_cores(steps, warmup, dt, level, N, prm, nproc=None):
    """The oracle, as it stands, on every host core: one independent sample
    per process (a spawn-started pool, safe after CUDA use).  Returns
    (aggregate DOF-updates/s = summed work / slowest worker's time, that
    time, processes)."""
    import multiprocessing as mp
    import oracle
    oracle.build()  # compiled once, before the workers load it
    nproc = nproc or os.cpu_count() or 1
    with mp.get_context("spawn").Pool(nproc) as pool:
        res = pool.map(_oracle_sample, [(steps, warmup, dt, level, N, prm)] * nproc)
    el = max(r[1] for r in res)
    return sum(r[0] for r in res) / el, el, nproc


def aggregate_ranks(ms, work):
    """Replicas: every rank advances its own copy of the workload.  Returns
    (max elapsed ms over ranks, total work over ranks); plain values on one
    process, all-reduces over torch.distributed when a group is initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(work)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    w = torch.tensor([float(work)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = build_workload(args.workload)
    # sample size from a one-core probe (one sample fits the time budget),
    # then the same sample on every host core at once
    r1, _, E, level = cpu_oracle_rate(1, 0, w.cfl_dt, budget_s=150.0 / max(1, args.steps + args.warmup))
    rate, el, nproc = cpu_oracle_rate_all_cores(args.steps, args.warmup, w.cfl_dt, level, w.N, w.params)
    sample = (f"{args.steps} SSP-RK3 steps of the rotor family at {E} quads, N={w.N}, on each of {nproc} "
              f"processes (one per host core)")
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "DOF-updates/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "sample": f"same generator at {E} quads, N={w.N}"},
        "cpu_baseline": {"value": rate, "unit": "DOF-updates/s", "cores": nproc, "kind": "oracle",
                         "sample": sample, "single_core": r1},
        "e2e": {"value": rate, "unit": "DOF-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_batched(ssd, ncases, steps, max_cells=50000):
    """Batched form (config 3): a seeded mix of independent cases (Couette,
    rotor and rotating-ellipse families, 1k-50k cells, p = 2..5, omega in
    [0.1, 1]) advanced together -- one launch per phase for all cases of a
    class (equal N and viscous flag), one CUDA graph per step -- on the FP32
    path with autotuned launch shapes and, for the speedup and the accuracy,
    on the FP64 path (default shapes); against the same FP32 cases stepped
    through their own handles (each its own graph and stream, issued one
    after another, so they run concurrently).  Wall-clock time around
    synchronised calls."""
    from ssd_inputs.workloads import batch_cases
    t_gen = time.perf_counter()
    cases = batch_cases(ncases, max_cells=max_cells)
    t_gen = time.perf_counter() - t_gen
    dts = [c[4] for c in cases]

    def start(b, k, name, prm):
        if name.startswith("ellipse"):
            return b.cases[k].state_from(lambda x, y: fields.uniform(x, y, rho=prm.rho_inf, u=prm.u_inf,
                                                                    v=prm.v_inf, p=prm.p_inf))
        if prm.viscous:
            return b.cases[k].state_from(lambda x, y: fields.uniform(x, y, rho=1.0, p=prm.Rgas))
        return b.cases[k].state_from(lambda x, y: fields.isentropic_vortex(x, y))

    def run(precision, tune_dt, separate=False):
        t0 = time.perf_counter()
        b = ssd.Batch([c[1] for c in cases], [c[2] for c in cases], [c[3] for c in cases], precision=precision,
                      tune_dt=tune_dt)
        t_create = time.perf_counter() - t0
        states = [start(b, k, c[0], c[3]) for k, c in enumerate(cases)]
        for k, q in enumerate(states):
            b.cases[k].sd_set_state(q)
        dofs = sum(c.n_dofs for c in b.cases)
        b.sd_batch_step(dts, 5)
        b.sd_batch_sync()
        for k, q in enumerate(states):
            b.cases[k].sd_set_state(q)
            b.cases[k].sd_set_time(0.0)
        t0 = time.perf_counter()
        b.sd_batch_step(dts, steps)
        b.sd_batch_sync()
        el = time.perf_counter() - t0
        finals = [c.sd_get_state() for c in b.cases]
        info = b.class_info()
        el_sep = None
        if separate:
            for k, c in enumerate(b.cases):
                c.sd_set_state(states[k])
                c.sd_step(dts[k], 5)
            for c in b.cases:
                c.sd_sync()
            for k, c in enumerate(b.cases):
                c.sd_set_state(states[k])
            t1 = time.perf_counter()
            for k, c in enumerate(b.cases):
                c.sd_step(dts[k], steps)
            for c in b.cases:
                c.sd_sync()
            el_sep = time.perf_counter() - t1
        b.close()
        return dofs, el, el_sep, finals, info, t_create

    dofs, el, el_sep, q32, info, t_create = run(ssd.SD_PREC_FP32, 1e-5, separate=True)
    _, el64, _, q64, _, _ = run(ssd.SD_PREC_FP64, 0.0)
    worst = max(float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2))) for a, b in zip(q32, q64))
    cells = [int(len(c[1]["elem_nodes"])) for c in cases]
    return {"value": dofs * steps / el, "unit": "DOF-updates/s", "cases": len(cases), "dofs": dofs,
            "cells": int(sum(cells)), "cells_min": min(cells), "cells_max": max(cells), "steps": steps,
            "ms_per_step": el / steps * 1e3, "precision": "f32", "autotuned": True, "classes": info,
            "fp64_value": dofs * steps / el64, "fp64_ms_per_step": el64 / steps * 1e3, "fp64_autotuned": False,
            "speedup_vs_fp64": el64 / el, "fp32_rel_l2_vs_fp64_worst_case": worst,
            "concurrent_handles_ms_per_step": el_sep / steps * 1e3, "speedup_vs_concurrent_handles": el_sep / el,
            "timing": "wall clock around synchronised calls", "mesh_generation_s": t_gen,
            "create_and_tune_s": t_create}


def start_field(w):
    """Initial state of a workload's main leg: the strength-5 vortex for the
    periodic vortex / rotor meshes, the smooth no-slip start for the
    ellipse, fluid at rest for the tank and the Couette annulus."""
    prm = w.params
    if w.name.startswith("ellipse"):
        return lambda x, y: fields.ellipse_start(x, y, prm.rho_inf, prm.u_inf, prm.v_inf, prm.p_inf, prm.omega,
                                                 gamma=prm.gamma)
    if w.name.startswith(("tank", "couette")):
        return lambda x, y: fields.uniform(x, y, rho=1.0, p=prm.Rgas)
    return lambda x, y: fields.isentropic_vortex(x, y)


def run_config(ssd, stream, name, steps, warmup, start, start_label, other_start=None):
    """One of the paper's named configurations at full size: FP32 and FP64
    paths over ``steps`` steps from ``start`` (CUDA-event throughput of each,
    per-kernel times of the FP32 step, FP32-vs-FP64 state difference after the
    steps) and, if given, the same difference from ``other_start``."""
    import torch
    w = build_workload(name)
    prm = w.params
    out = {"workload": w.name, "elements": int(len(w.mesh["elem_nodes"])), "N": w.N, "steps": steps,
           "dt": w.cfl_dt, "start": start_label}

    def run(prec, q_fn, timed):
        s = ssd.Solver(w.mesh, w.N - 1, prm, precision=prec, stream=stream.cuda_stream)
        s.sd_set_state(s.state_from(q_fn))
        res = {}
        if timed:
            s.sd_step(w.cfl_dt, warmup)
            s.sd_sync()
            s.sd_set_state(s.state_from(q_fn))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s.sd_step(w.cfl_dt, steps)
            b.record(stream)
            b.synchronize()
            s.sd_sync()
            ms = a.elapsed_time(b)
            res = {"value": s.n_dofs * steps / (ms * 1e-3), "unit": "DOF-updates/s", "ms_per_step": ms / steps}
            q = s.sd_get_state()  # before sd_profile_step, which advances the solution
            if prec == ssd.SD_PREC_FP32:
                prof = s.sd_profile_step(w.cfl_dt, reps=5)
                res["kernel_ms"] = prof
                res["interface_fraction"] = interface_fraction(prof)
        else:
            s.sd_step(w.cfl_dt, steps)
            s.sd_sync()
            q = s.sd_get_state()
        s.close()
        return res, q

    def rel(a, b):
        return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))

    out["fp32"], q32 = run(ssd.SD_PREC_FP32, start, True)
    out["fp64"], q64 = run(ssd.SD_PREC_FP64, start, True)
    out["fp32_rel_l2_vs_fp64"] = rel(q32, q64)
    out["fp32_speedup"] = out["fp32"]["value"] / out["fp64"]["value"]
    if other_start is not None:
        label, fn = other_start
        _, i32 = run(ssd.SD_PREC_FP32, fn, False)
        _, i64 = run(ssd.SD_PREC_FP64, fn, False)
        out[label + "_fp32_rel_l2_vs_fp64"] = rel(i32, i64)
    return out


def run_ellipse(ssd, stream, steps, warmup):
    """Flow past the rotating ellipse (20096 cells, N = 5, Navier-Stokes,
    slip / inlet / outlet, cubic cells) from a smooth start that meets the
    no-slip condition, and the FP32-vs-FP64 difference from the impulsively
    started free stream."""
    prm = build_workload("ellipse_n5").params
    smooth = lambda x, y: fields.ellipse_start(x, y, prm.rho_inf, prm.u_inf, prm.v_inf, prm.p_inf, prm.omega,
                                               gamma=prm.gamma)
    impulsive = lambda x, y: fields.uniform(x, y, rho=prm.rho_inf, u=prm.u_inf, v=prm.v_inf, p=prm.p_inf)
    return run_config(ssd, stream, "ellipse_n5", steps, warmup, smooth,
                      "free stream blended to the body rotation (no-slip at t = 0)", ("impulsive_start", impulsive))


def run_couette(ssd, stream, steps, warmup):
    """Taylor-Couette flow (288 cells, N = 3, Navier-Stokes, rotating inner
    wall) for the configuration's 200 steps from the quiescent uniform state."""
    prm = build_workload("couette_n3").params
    rest = lambda x, y: fields.uniform(x, y, rho=1.0, p=prm.Rgas)
    return run_config(ssd, stream, "couette_n3", steps, warmup, rest, "uniform fluid at rest, T = T_wall")


def run_tank(ssd, stream, steps, warmup):
    """Stirred tank (14752 cells, N = 4, Navier-Stokes, rotating hub and
    adiabatic blades, baffles) started at rest, as in Sec. 4."""
    prm = build_workload("tank_n4").params
    rest = lambda x, y: fields.uniform(x, y, rho=1.0, p=prm.Rgas)
    return run_config(ssd, stream, "tank_n4", steps, warmup, rest, "uniform fluid at rest (Sec. 4)")


def run_vortex(ssd, stream, t_end=0.25):
    """The vortex configuration (Sec. 4.1): the strength-5 isentropic vortex
    convected through the rotating disk of the 6,016-cell mesh, N = 4 and 5,
    to t_end.  Per N: FP32 and FP64 throughput (CUDA events on the solver's
    stream), the density L2 error against the exact translated vortex at
    t_end, the FP32-vs-FP64 state difference, and the FP64 error and order
    from the same run on the h/2 mesh (24,064 cells)."""
    import torch
    from ssd_inputs.workloads import vortex_family
    vortex = lambda x, y: fields.isentropic_vortex(x, y)

    def run(N, scale, prec):
        mesh, prm, dt = vortex_family(N, scale)
        n = int(math.ceil(t_end / dt))
        dt = t_end / n
        s = ssd.Solver(mesh, N - 1, prm, precision=prec, stream=stream.cuda_stream)
        q0 = s.state_from(vortex)
        s.sd_set_state(q0)
        s.sd_step(dt, 5)
        s.sd_sync()
        s.sd_set_state(q0)
        s.sd_set_time(0.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        s.sd_step(dt, n)
        b.record(stream)
        b.synchronize()
        s.sd_sync()
        ms = a.elapsed_time(b)
        t = s.sd_get_time()
        Q = s.sd_get_state()
        xy = s.sd_sp_coords(t)
        ex = fields.isentropic_vortex(xy[..., 0], xy[..., 1], t=t, period=(-10.0, 20.0))
        err = float(np.sqrt(np.mean((Q[:, 0] - ex[..., 0]) ** 2)))
        res = {"value": s.n_dofs * n / (ms * 1e-3), "unit": "DOF-updates/s", "ms_per_step": ms / n, "steps": n,
               "elements": s.E, "l2_error_rho": err}
        s.close()
        return res, Q

    out = {"workload": "vortex_n4 / vortex_n5", "t_end": t_end,
           "description": "isentropic vortex (strength 5) on periodic [-10,10]^2, rotating disk r<=3 at "
                          "omega=pi/4, 6,016 quads"}
    for N in (4, 5):
        r32, q32 = run(N, 1, ssd.SD_PREC_FP32)
        r64, q64 = run(N, 1, ssd.SD_PREC_FP64)
        fine, _ = run(N, 2, ssd.SD_PREC_FP64)
        out[f"N{N}"] = {"fp32": r32, "fp64": r64,
                        "fp32_rel_l2_vs_fp64": float(np.sqrt(np.sum((q32 - q64) ** 2) / np.sum(q64 ** 2))),
                        "fp32_speedup": r32["value"] / r64["value"],
                        "fp64_h2": {"elements": fine["elements"], "l2_error_rho": fine["l2_error_rho"],
                                    "order": math.log2(r64["l2_error_rho"] / fine["l2_error_rho"])}}
    return out


def run_twin(ssd, stream, steps, warmup):
    """Two counter-rotating rotors (123,450 cells, N = 6, Euler; two rotating
    zones, each with its own sliding interface) with the strength-5 vortex
    between them."""
    return run_config(ssd, stream, "twin_rotor_n6", steps, warmup, lambda x, y: fields.isentropic_vortex(x, y),
                      "strength-5 vortex at the origin, between the two disks")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rotor_n6")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "fp32s", "tf32"])
    ap.add_argument("--fp64-steps", type=int, default=100)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-steps", type=int, default=40)
    ap.add_argument("--no-cpu", action="store_true")
    # the batched form is held off the GPU by default (0 cases): a 64-case run
    # of it stopped on a device error whose cause is not yet found
    ap.add_argument("--batch-cases", type=int, default=0)
    ap.add_argument("--batch-steps", type=int, default=50)
    ap.add_argument("--batch-max-cells", type=int, default=50000)
    ap.add_argument("--ellipse-steps", type=int, default=200)
    ap.add_argument("--tank-steps", type=int, default=200)
    ap.add_argument("--couette-steps", type=int, default=200)
    ap.add_argument("--twin-steps", type=int, default=200)
    ap.add_argument("--vortex-t", type=float, default=0.25, help="vortex-configuration leg end time (0: skip)")
    ap.add_argument("--fp32s-steps", type=int, default=-1, help="FP32-state leg steps (-1: same as --steps)")
    ap.add_argument("--tf32-steps", type=int, default=-1, help="3xTF32 tensor-core leg steps (-1: same as --steps)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    import paper_1503_02198_gb300 as ssd

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    ssd.build()

    w = build_workload(args.workload)
    N, dt = w.N, w.cfl_dt
    prec = {"fp32": ssd.SD_PREC_FP32, "fp64": ssd.SD_PREC_FP64, "fp32s": ssd.SD_PREC_FP32S,
            "tf32": ssd.SD_PREC_FP32_TF32}[args.precision]
    stream = torch.cuda.Stream()
    solver = ssd.Solver(w.mesh, N - 1, w.params, precision=prec, stream=stream.cuda_stream)
    Q0 = solver.state_from(start_field(w))
    solver.sd_set_state(Q0)
    dofs = solver.n_dofs

    def barrier():
        if world > 1:
            dist.barrier()

    # warm-up
    solver.sd_step(dt, args.warmup)
    solver.sd_sync()
    barrier()
    torch.cuda.synchronize()
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        gpu_id = str(local)
    sampler = ClockSampler(gpu_id)
    sampler.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    solver.sd_step(dt, args.steps)
    e1.record(stream)
    e1.synchronize()
    clocks = sampler.stop()
    solver.sd_sync()
    barrier()
    torch.cuda.synchronize()
    ms, work = aggregate_ranks(e0.elapsed_time(e1), dofs * args.steps)
    value = work / (ms * 1e-3)

    # accuracy at the final time: density L2 error against the exact vortex
    # (periodic vortex / rotor workloads)
    t_end = solver.sd_get_time()
    Q = solver.sd_get_state()
    l2_rho = None
    if w.name.startswith(("rotor", "vortex")):
        xy = solver.sd_sp_coords(t_end)
        lo, hi = float(w.mesh["xy"][:, 0].min()), float(w.mesh["xy"][:, 0].max())
        exact = np.moveaxis(fields.isentropic_vortex(xy[..., 0], xy[..., 1], t=t_end, period=(lo, hi - lo)), -1, 1)
        l2_rho = float(np.sqrt(np.mean((Q[:, 0] - exact[:, 0]) ** 2)))

    # FP64 path on the same workload: throughput and FP32-vs-FP64 difference
    fp64 = None
    if prec == ssd.SD_PREC_FP32 and args.fp64_steps > 0:
        s64 = ssd.Solver(w.mesh, N - 1, w.params, precision=ssd.SD_PREC_FP64, stream=stream.cuda_stream)
        s64.sd_set_state(Q0)
        s64.sd_step(dt, args.warmup)
        s64.sd_sync()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        s64.sd_step(dt, args.fp64_steps)
        b.record(stream)
        b.synchronize()
        s64.sd_sync()
        ms64 = a.elapsed_time(b)
        # the FP64 state after the FP32 run's steps (warm-up + timed), from the same start
        s64.sd_set_state(Q0)
        s64.sd_set_time(0.0)
        s64.sd_step(dt, args.warmup + args.steps)
        s64.sd_sync()
        Q64 = s64.sd_get_state()
        rel = float(np.sqrt(np.sum((Q - Q64) ** 2) / np.sum(Q64 ** 2)))
        fp64 = {"value": dofs * args.fp64_steps / (ms64 * 1e-3), "ms_per_step": ms64 / args.fp64_steps,
                "fp32_rel_l2_vs_fp64": rel, "fp32_speedup": (dofs * args.steps / (ms * 1e-3)) /
                (dofs * args.fp64_steps / (ms64 * 1e-3))}
        peak64 = s64.sd_fma_peak(ssd.SD_PREC_FP64)
        fp64["fma_peak_tflops"] = peak64
        # the FP64 volume kernel against the FP64 pipe (its bound: GB300's FP64
        # rate is 1/64 of FP32) and against HBM
        prof64 = s64.sd_profile_step(dt, reps=3)
        fl64 = volume_flops_per_element(N) * s64.E
        ach64 = fl64 / (prof64["volume"] * 1e-3) / 1e12
        vb64 = volume_bytes_per_element(N, 8, 8) * s64.E
        pk_hbm, _ = _peaks()
        fp64["kernel_ms"] = prof64
        fp64["interface_fraction"] = interface_fraction(prof64)
        fp64["roofline"] = {"bound": "alu", "pipe": "fp64", "achieved": ach64, "peak": peak64, "unit": "TFLOP/s",
                            "frac": ach64 / peak64, "kernel": "k_volume",
                            "peak_source": "measured FP64 FMA throughput of this GPU (sd_fma_peak)",
                            "algorithmic_flops_per_launch": fl64,
                            "flops_per_element": volume_flops_per_element(N),
                            "hbm_achieved_gbs": vb64 / (prof64["volume"] * 1e-3) / 1e9,
                            "hbm_frac": vb64 / (prof64["volume"] * 1e-3) / 1e9 / pk_hbm}
        s64.close()

    # FP32 state storage on the same workload: throughput, volume-kernel
    # roofline and state difference from the FP64 path after the same steps
    fp32s = None
    if args.fp32s_steps < 0:
        args.fp32s_steps = args.steps
    if prec == ssd.SD_PREC_FP32 and args.fp32s_steps > 0:
        s3 = ssd.Solver(w.mesh, N - 1, w.params, precision=ssd.SD_PREC_FP32S, stream=stream.cuda_stream)
        s3.sd_set_state(Q0)
        s3.sd_step(dt, args.warmup)
        s3.sd_sync()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        s3.sd_step(dt, args.fp32s_steps)
        b.record(stream)
        b.synchronize()
        s3.sd_sync()
        ms3 = a.elapsed_time(b)
        fp32s = {"value": dofs * args.fp32s_steps / (ms3 * 1e-3), "unit": "DOF-updates/s",
                 "ms_per_step": ms3 / args.fp32s_steps, "steps": args.fp32s_steps, "state_bytes_per_value": 4}
        if fp64 is not None and args.fp32s_steps == args.steps:
            Q3 = s3.sd_get_state()
            fp32s["rel_l2_vs_fp64"] = float(np.sqrt(np.sum((Q3 - Q64) ** 2) / np.sum(Q64 ** 2)))
        prof3 = s3.sd_profile_step(dt, reps=5)
        vb3 = volume_bytes_per_element(N, 4, 4) * s3.E
        ach3 = vb3 / (prof3["volume"] * 1e-3) / 1e9
        pk, _ = _peaks()
        fp32s["kernel_ms"] = prof3
        fp32s["roofline"] = {"bound": "hbm", "achieved": ach3, "peak": pk, "unit": "GB/s", "frac": ach3 / pk,
                             "kernel": "k_volume", "algorithmic_bytes_per_launch": vb3}
        s3.close()

    # the FP32 form with the volume contractions on the tensor cores (3xTF32):
    # throughput, volume-kernel time, difference from the FP64 path
    tf32 = None
    if args.tf32_steps < 0:
        args.tf32_steps = args.steps
    if prec == ssd.SD_PREC_FP32 and args.tf32_steps > 0:
        st = ssd.Solver(w.mesh, N - 1, w.params, precision=ssd.SD_PREC_FP32_TF32, stream=stream.cuda_stream)
        st.sd_set_state(Q0)
        st.sd_step(dt, args.warmup)
        st.sd_sync()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st.sd_step(dt, args.tf32_steps)
        b.record(stream)
        b.synchronize()
        st.sd_sync()
        mst = a.elapsed_time(b)
        tf32 = {"value": dofs * args.tf32_steps / (mst * 1e-3), "unit": "DOF-updates/s",
                "ms_per_step": mst / args.tf32_steps, "steps": args.tf32_steps,
                "contractions": "interpolation and divergence as 3xTF32 mma.sync m16n8k8 (tensor pipe)"}
        if fp64 is not None and args.tf32_steps == args.steps:
            Qt = st.sd_get_state()
            tf32["rel_l2_vs_fp64"] = float(np.sqrt(np.sum((Qt - Q64) ** 2) / np.sum(Q64 ** 2)))
            tf32["rel_l2_vs_fp32_ffma"] = float(np.sqrt(np.sum((Qt - Q) ** 2) / np.sum(Q ** 2)))
        tf32["kernel_ms"] = st.sd_profile_step(dt, reps=5)
        st.close()

    # per-kernel timing (CUDA events on the handle's stream) -> roofline of the volume kernel
    prof = solver.sd_profile_step(dt, reps=5)
    w_c = 8 if prec == ssd.SD_PREC_FP64 else 4
    E = solver.E
    vol_bytes = volume_bytes_per_element(N, w_c, 4 if prec == ssd.SD_PREC_FP32S else 8) * E
    peak, peak_src = _peaks()
    achieved = vol_bytes / (prof["volume"] * 1e-3) / 1e9
    traffic = profiled_traffic() if (args.workload == "rotor_n6" and prec == ssd.SD_PREC_FP32) else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic,
                "traffic_source": ("stored ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of this "
                                   "kernel source, not a measurement of this run") if traffic else None,
                "kernel": "k_volume", "peak_source": peak_src + " hbm_gbs (burst)",
                "algorithmic_bytes_per_launch": vol_bytes}
    try:
        fp32_peak = solver.sd_fma_peak(ssd.SD_PREC_FP32)
    except Exception:
        fp32_peak = None

    # end to end through the public API with host buffers: H2D state, one step, D2H state
    pin_in = torch.empty(solver.shape, dtype=torch.float64, pin_memory=True)
    pin_out = torch.empty(solver.shape, dtype=torch.float64, pin_memory=True)
    pin_in.copy_(torch.from_numpy(Q))
    solver.sd_set_state(pin_in)
    solver.sd_step(dt, 1)
    solver.sd_get_state(pin_out)
    barrier()
    t_set = t_rest = 0.0
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        ta = time.perf_counter()
        solver.sd_set_state(pin_in)  # returns once the state is on the device
        tb = time.perf_counter()
        solver.sd_step(dt, 1)
        solver.sd_get_state(pin_out)  # waits for the step, then the state is on the host
        t_set += tb - ta
        t_rest += time.perf_counter() - tb
    solver.sd_sync()
    e2e_s, e2e_work = aggregate_ranks(time.perf_counter() - t0, dofs * args.e2e_steps)
    state_bytes = dofs * 8
    e2e = {"value": e2e_work / e2e_s if e2e_s > 0 else 0.0, "unit": "DOF-updates/s",
           "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes}
    if args.e2e_steps > 0:
        # per step: set_state (host -> device, FP64 state), then the step and
        # get_state (device -> host); the host link, not the step, dominates
        n_e = args.e2e_steps
        e2e.update({"set_state_ms": 1e3 * t_set / n_e, "step_and_get_state_ms": 1e3 * t_rest / n_e,
                    "h2d_gbs": state_bytes / (t_set / n_e) / 1e9 if t_set > 0 else None})

    batched = (run_batched(ssd, args.batch_cases, args.batch_steps, args.batch_max_cells)
               if args.batch_cases > 0 else
               {"held": "not run: the batched kernels are held off the GPU until an error seen in a 64-case "
                        "run is explained (the library refuses them unless SSD_BATCH_ENABLE=1)"})
    ellipse = run_ellipse(ssd, stream, args.ellipse_steps, 5) if args.ellipse_steps > 0 else None
    tank = run_tank(ssd, stream, args.tank_steps, 5) if args.tank_steps > 0 else None
    couette = run_couette(ssd, stream, args.couette_steps, 5) if args.couette_steps > 0 else None
    twin = run_twin(ssd, stream, args.twin_steps, 5) if args.twin_steps > 0 else None
    vortex = run_vortex(ssd, stream, args.vortex_t) if args.vortex_t > 0 else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        # the oracle on one core, then the same sample on every host core at once
        rate1, el1, Es, level = cpu_oracle_rate(args.cpu_steps, 0, dt)
        rate, el, nproc = cpu_oracle_rate_all_cores(args.cpu_steps, 1, dt, level, N, w.params)
        cpu = {"value": rate, "unit": "DOF-updates/s", "cores": nproc, "kind": "oracle",
               "sample": f"{args.cpu_steps} SSP-RK3 steps of the same rotor family at {Es} quads, N={N}, on each "
                         f"of {nproc} processes (one per host core; {el:.1f} s)",
               "single_core": {"value": rate1, "cores": 1, "seconds": el1}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "DOF-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == ssd.SD_PREC_FP64 else "f32",
            "data": "synthetic",
            "config": {"workload": w.name, "elements": E, "N": N, "dofs": dofs, "dt": dt,
                       "state_precision": "f32" if prec == ssd.SD_PREC_FP32S else "f64", "l2_flush": "state 284 MB > L2 (inputs larger than L2)",
                       "parallelism": f"replicas x{world}", "description": w.description},
            "l2_error_rho_vs_exact": l2_rho, "t_final": t_end,
            "fp64": fp64,
            "fp32_state": fp32s,
            "tf32x3": tf32,
            "batched": batched,
            "ellipse": ellipse,
            "tank": tank,
            "couette": couette,
            "twin_rotor": twin,
            "vortex": vortex,
            "kernel_ms": prof,
            "interface_fraction": interface_fraction(prof),
            "fp32_fma_peak_tflops": fp32_peak,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks,
            "gpu_launches": launches_per_step(w.mesh, w.params.viscous) * args.steps + 2,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
