"""Benchmark of the fused shallow-water step on one GB300 (or N replicas).

A bench step is one explicit Euler time step of the whole hot path over the
workload's mesh: edge fluxes with hydrostatic reconstruction and HLLC,
boundary fluxes, semi-implicit friction, update and the CFL min-reduction
(one fused kernel launch, replayed from CUDA graphs).

Default workload: the 12,999,168-cell synthetic river reach (20 km x 2 km,
partially dry, Q = 2000 m^3/s inflow, fixed-stage outflow), FP32 state with
FP64 time step.  Its working set (~1 GB) is far larger than L2, so no flush
is needed between steps.  The default run also measures every other
workload (the fully wet river, the FP64 canal, the FP32 and FP64 ensembles,
the adjoint) with short step counts and reports each as a sub-record of the
same line; ``--workload`` runs one workload alone.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead, on the host cores.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# algorithmic bytes per cell-update: state in (3) + state out (3) + z, m,
# 1/|Omega|, inscribed radius (4) + L n of three edges (6) values, plus three
# int32 neighbour indices
ALG_BYTES = {"f32": 16 * 4 + 12, "f64": 16 * 8 + 12}
# FP64 flops (2 x DFMA + DADD + DMUL) per cell that runs the flux path, from
# ncu's instruction counts of the two FP64 step kernels on the 1M-cell
# dry-bed canal divided by the cells that ran the flux path: the cell-centric
# step evaluates every interior flux twice, the edge pass once; quiet cells
# take no flux path and do no FP64 arithmetic
FP64_FLOPS_PER_ACTIVE_CELL = {"cell": 748, "edge": 505}
# GB300 FP64: 2 DFMA per clock per SM, 152 SMs
FP64_DFMA_PER_CLK_SM, N_SM = 2, 152

WORKLOADS = {
    "river13m_fp32": dict(maker="river_13m", precision="f32", steps=1000,
                          desc="synthetic river reach 20 km x 2 km, 12,999,168 triangles, partially dry, "
                               "Q=2000 m3/s inflow, stage outflow, Manning U[0.02,0.06]; FP32 state, FP64 dt"),
    "river13m_wet_fp32": dict(maker="river_13m_wet", precision="f32", steps=1000,
                              desc="synthetic river reach 20 km x 2 km, 12,999,168 triangles, fully wet (depth >= "
                                   "0.5 m), Q=2000 m3/s inflow, stage outflow, Manning U[0.02,0.06]; FP32 state, "
                                   "FP64 dt"),
    "canal1m_fp64": dict(maker="dam_break_dry_1m", precision="f64", steps=2000,
                         desc="dry-bed dam break, canal 200 m x 10 m, 1,000,000 triangles, n=0.03; FP64"),
    "canal1m_fp32": dict(maker="dam_break_dry_1m", precision="f32", steps=2000,
                         desc="dry-bed dam break, canal 200 m x 10 m, 1,000,000 triangles, n=0.03; FP32"),
    "dam4k_fp64": dict(maker="dam_break_4k", precision="f64", steps=500,
                       desc="wet dam break, canal 200 m x 10 m, 4,000 triangles; FP64"),
    "ensemble256_fp32": dict(maker="ensemble", precision="f32", steps=1000,
                             desc="256-member ensemble, canal and river members of 20k-500k triangles "
                                  "(log-uniform), Manning U[0.015,0.08], Q U[500,3000]; FP32 state, FP64 dt"),
    "adjoint1m_fp64": dict(maker="river_adjoint_1m", precision="f64", steps=2000,
                           desc="adjoint of the gauge misfit (64 gauges) after 2000 FP64 steps on the 1,001,728-"
                                "triangle fully wet river, checkpoints every 50 steps, gradient w.r.t. Manning "
                                "and bed"),
    "ensemble256_fp64": dict(maker="ensemble", precision="f64", steps=1000,
                             desc="256-member ensemble, canal and river members of 20k-500k triangles "
                                  "(log-uniform), Manning U[0.015,0.08], Q U[500,3000]; FP64"),
}


MEMBERS = [256, "all", False]   # ensemble workloads: number of members, which of them, batched only


def _peak_clock():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return float(json.load(f).get("sm_max_mhz", 2070.0))
    return 2070.0


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        return self.summary()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for _, line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return None, 0, 1, 0
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    dist.init_process_group("gloo")
    return dist, rank, ws, local


def max_over_ranks(dist, values):
    """Element-wise max of per-rank timings (the slowest rank sets the time)."""
    if not dist:
        return [float(v) for v in values]
    import torch
    tt = torch.tensor([float(v) for v in values], dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return [float(v) for v in tt.tolist()]


def _make_input(name):
    from paper_2010_14416_gb300 import meshgen
    if WORKLOADS[name]["maker"] == "ensemble":
        return meshgen.ensemble_members(MEMBERS[0])
    return getattr(meshgen, WORKLOADS[name]["maker"])()


def cpu_baseline(mi, budget_s=20.0):
    """The FP64 oracle as it stands, on all host cores: whole-mesh steps until
    the time budget is used (at least two)."""
    import oracle
    M = oracle.Mesh(mi.nodes, mi.tris, mi.z, mi.manning)
    for pairs, kind, value in mi.bcs:
        M.set_bc(pairs, kind, value)
    h, hu, hv = mi.h.astype(np.float64), mi.hu.astype(np.float64), mi.hv.astype(np.float64)
    cores = oracle.max_threads()
    steps = 0
    t0 = time.perf_counter()
    while True:
        dt = M.dt(h, hu, hv, 0.9)
        h, hu, hv, _ = M.step(h, hu, hv, dt)
        steps += 1
        el = time.perf_counter() - t0
        if steps >= 2 and el >= budget_s:
            break
    # the same oracle on one core, over a fixed seeded sample of the cells
    n_s = min(1 << 17, mi.n_cells)
    cells = np.sort(np.random.default_rng(0).choice(mi.n_cells, n_s, replace=False))
    oracle.set_threads(1)
    try:
        reps = 0
        t1 = time.perf_counter()
        while True:
            M.step_cells(h, hu, hv, dt, cells)
            reps += 1
            el1 = time.perf_counter() - t1
            if reps >= 2 and el1 >= budget_s / 4:
                break
    finally:
        oracle.set_threads(cores)
    return {"value": mi.n_cells * steps / el, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
            "sample": f"{steps} whole-mesh FP64 oracle steps from the initial state "
                      f"({mi.n_cells:,} cells, {el:.1f} s, OpenMP over cells)",
            "single_core": {"value": n_s * reps / el1, "unit": "cell-updates/s", "cores": 1,
                            "sample": f"{reps} one-step updates of a fixed seeded sample of {n_s:,} cells "
                                      f"({el1:.1f} s)"}}


def run_reference(args, name):
    """--impl reference: the oracle timed on the host cores; each bench step is
    one oracle step over a fixed seeded sample of 2^20 cells of the mesh."""
    dist, rank, ws, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    mi = _make_input(name)
    M = oracle.Mesh(mi.nodes, mi.tris, mi.z, mi.manning)
    for pairs, kind, value in mi.bcs:
        M.set_bc(pairs, kind, value)
    n_s = min(1 << 20, mi.n_cells)
    cells = np.sort(np.random.default_rng(0).choice(mi.n_cells, n_s, replace=False))
    h, hu, hv = mi.h.astype(np.float64), mi.hu.astype(np.float64), mi.hv.astype(np.float64)
    dt = M.dt(h, hu, hv, 0.9)
    for _ in range(args.warmup):
        M.step_cells(h, hu, hv, dt, cells)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        M.step_cells(h, hu, hv, dt, cells)
    el = time.perf_counter() - t0
    cores = oracle.max_threads()
    val = n_s * args.steps / el
    line = {"impl": "reference", "metric": "cell-updates/s", "value": val, "unit": "cell-updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[name]["desc"], "cells": mi.n_cells},
            "cpu_baseline": {"value": val, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step: one FP64 oracle step over a seeded sample of {n_s:,} "
                                       f"of the {mi.n_cells:,} cells"},
            "e2e": {"value": val, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


class GpuContext:
    """Device, stream, rank and library of one bench process."""

    def __init__(self):
        import torch

        from paper_2010_14416_gb300 import build as libbuild
        from paper_2010_14416_gb300 import capi

        self.torch, self.capi = torch, capi
        self.dist, self.rank, self.ws, self.local = _dist()
        torch.cuda.set_device(self.local)
        self.dev = torch.device("cuda", self.local)
        if self.rank == 0:
            libbuild.build()
        if self.dist:
            self.dist.barrier()
        self.stream = torch.cuda.Stream(device=self.dev)
        self.inputs = {}

    def make_input(self, name):
        # workloads sharing a generator share its (seeded, deterministic) input
        maker = WORKLOADS[name]["maker"]
        if maker not in self.inputs:
            self.inputs[maker] = _make_input(name)
        return self.inputs[maker]

    def timed(self, fn):
        """CUDA-event time (ms) of fn() on the bench stream, synchronised on both
        sides after a barrier, with nvidia-smi clocks sampled meanwhile; the
        slowest rank's time."""
        torch = self.torch
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        clocks = ClockSampler(self.local)
        if self.rank == 0:
            clocks.start()
        if self.dist:
            self.dist.barrier()
        torch.cuda.synchronize(self.dev)
        ev0.record(self.stream)
        fn()
        ev1.record(self.stream)
        torch.cuda.synchronize(self.dev)
        ms = ev0.elapsed_time(ev1)
        clk = clocks.stop() if self.rank == 0 else None
        return max_over_ranks(self.dist, [ms])[0], clk


def _warmup_for(steps, warmup, graph_steps=48):
    """Warm-up steps actually run before a timed region of `steps` steps: the
    requested number, raised when the timed call will replay a CUDA graph so
    that the graph is captured before the timed region (captures start at a
    step index that is a multiple of six)."""
    return max(warmup, graph_steps + 6) if steps >= graph_steps else warmup


def _hbm_roofline(wl, n, kernel_ms, active_frac, activity, name, shape, peak, peak_kind, ensemble=False):
    """HBM roofline of an FP32 step: bytes this kernel's data layout must move
    per launch at the measured active fraction (frac), the ncu DRAM bytes of
    the same kernel source and launch shape when a committed record has them
    (traffic_frac), and the dense per-cell model for reference."""
    ab = ALG_BYTES[wl["precision"]]
    rec = 16 if wl["precision"] == "f32" else 32
    # activity kernels read a cell's byte and clear the previous step's byte
    # (the mesh's kernel also reads the latter)
    act_bytes = (2 if ensemble else 3) if activity else 0
    # an active cell reads its state, topology and geometry records and writes
    # its state; a quiet cell (dry, dry neighbours, no inflow/stage edge)
    # needs no geometry, and with activity bytes no topology either, and with
    # the mesh's activity kernel no store when it was quiet in the previous
    # step too (its state is then in place; a quiet cell that is written
    # moves another record, so this is the lower bound of the layout's bytes
    # and the fraction is the conservative one)
    if not activity:
        quiet_bytes = 2 * rec + 16
    else:
        quiet_bytes = (2 * rec if ensemble else rec) + act_bytes
    layout_bytes = n * (active_frac * (4 * rec + 16 + (0 if wl["precision"] == "f32" else 8) + act_bytes) +
                        (1 - active_frac) * quiet_bytes)
    s = kernel_ms * 1e-3
    traffic = _traffic(name, shape)
    dense = ab * n / s / 1e9
    return {"bound": "hbm", "achieved": layout_bytes / s / 1e9, "peak": peak, "unit": "GB/s",
            "frac": layout_bytes / s / 1e9 / peak, "traffic": traffic,
            "traffic_frac": (traffic / s / 1e9 / peak) if traffic else None,
            "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)",
            "bytes_per_launch": layout_bytes, "active_cell_fraction": active_frac,
            "bytes_per_active_cell": 4 * rec + 16 + (0 if wl["precision"] == "f32" else 8) + act_bytes,
            "bytes_per_quiet_cell": quiet_bytes,
            "dense_model_bytes_per_cell": ab, "dense_model_frac": dense / peak,
            "note": "achieved/frac: the bytes this launch's kernel must move at the measured fraction of cells "
                    "that run the flux path (bytes_per_active_cell, bytes_per_quiet_cell; with the mesh's activity "
                    "kernel a cell quiet in the previous step too needs no store, and one that is written moves "
                    "another state record); traffic_frac: ncu "
                    "DRAM bytes per launch of the same kernel source and shape; dense_model_frac: "
                    f"{ab} B for every cell, which a quiet cell (dry among dry neighbours) does not need, so it "
                    "exceeds 1 on a mostly dry mesh"}


def _fp64_roofline(n, kernel_ms, active_frac, edge_pass, hbm):
    """FP64 steps are bound by the FP64 pipe: FP64 flops per cell that ran the
    flux path (ncu counts) against the pipe's rate from its unit count and the
    maximum SM clock."""
    sm_mhz = _peak_clock()
    peak64 = FP64_DFMA_PER_CLK_SM * 2 * N_SM * sm_mhz * 1e6 / 1e12
    per_cell = FP64_FLOPS_PER_ACTIVE_CELL["edge" if edge_pass else "cell"]
    ach64 = per_cell * active_frac * n / (kernel_ms * 1e-3) / 1e12
    return {"bound": "alu", "achieved": ach64, "peak": peak64, "unit": "TFLOP/s", "frac": ach64 / peak64,
            "traffic": None,
            "peak_source": f"nominal, not measured: {FP64_DFMA_PER_CLK_SM} DFMA/clk/SM x 2 flops x {N_SM} SMs "
                           f"x {sm_mhz:.0f} MHz (the FP64 pipe's unit count at the maximum SM clock; "
                           "MEASURED_PEAKS.json has no FP64 figure)",
            "flops_per_active_cell": per_cell, "active_cell_fraction": active_frac,
            "flops_counted": "2 x DFMA + DADD + DMUL per cell that ran the flux path (ncu instruction counts)",
            "hbm": {k: v for k, v in hbm.items() if k not in ("bound", "traffic")}}


def _traffic(name, shape):
    tpath = os.path.join(ROOT, "profiles", f"traffic_{name}.json")
    if not os.path.exists(tpath):
        return None
    with open(tpath) as f:
        tr = json.load(f)
    if tr.get("kernel_hash") != _kernel_hash():
        return None
    for cap in tr.get("captures", []):
        if cap.get("shape") == _shape_key(shape):
            return cap.get("bytes_per_launch")
    return None


def measure_mesh(ctx, name, steps, warmup, shape_spec=None, e2e=True):
    """One mesh workload: W warm-up steps, the library's autotuner (outside
    the timed region; its trials leave the state untouched), K timed steps
    replayed from CUDA graphs, and (e2e) three whole jobs through the C ABI
    from pinned host arrays."""
    torch, capi = ctx.torch, ctx.capi
    wl = WORKLOADS[name]
    prec = capi.SWE_FP32 if wl["precision"] == "f32" else capi.SWE_FP64
    npdt = np.float32 if prec == capi.SWE_FP32 else np.float64
    tdt = torch.float32 if prec == capi.SWE_FP32 else torch.float64
    mi = ctx.make_input(name)
    fixed = _shape_kwargs(shape_spec)
    m = capi.Mesh(mi.nodes, mi.tris, mi.z, mi.manning, precision=prec, device=ctx.local, **fixed)
    for pairs, kind, value in mi.bcs:
        m.set_bc(pairs, kind, value)
    m.set_stream(ctx.stream)
    h0 = torch.tensor(mi.h.astype(npdt), device=ctx.dev)
    hu0 = torch.tensor(mi.hu.astype(npdt), device=ctx.dev)
    hv0 = torch.tensor(mi.hv.astype(npdt), device=ctx.dev)
    torch.cuda.synchronize(ctx.dev)
    m.set_state(h0, hu0, hv0)
    if fixed:
        shape = dict(block_size=fixed["block_size"], min_blocks=fixed["min_blocks"], stages=fixed["stages"],
                     geometry_early=fixed["geometry_early"], activity=fixed["activity"],
                     edge_pass=fixed["edge_pass"], grid=fixed["grid"], cell_pairs=fixed.get("cell_pairs", 0),
                     chunk=0, fixed=True)
    else:
        shape = m.autotune(8)   # on the initial state, which the trials leave untouched
    warm = _warmup_for(steps, warmup)
    m.step(warm, 0.9, sync=True)
    n = mi.n_cells
    active0 = m.info()["n_active"]
    ms, clk = ctx.timed(lambda: m.step(steps, 0.9, sync=False))
    info = m.info()
    active_frac = (info["n_active"] - active0) / float(n * steps)
    m.synchronize()
    peak, peak_kind = _peaks()
    kernel_ms = ms / steps
    roof = _hbm_roofline(wl, n, kernel_ms, active_frac, shape.get("activity"), name, shape, peak, peak_kind)
    if wl["precision"] == "f64":
        roof = _fp64_roofline(n, kernel_ms, active_frac, shape.get("edge_pass"), roof)
    rec = {
        "metric": "cell-updates/s", "value": ctx.ws * n * steps / (ms * 1e-3), "unit": "cell-updates/s",
        "n_gpus": ctx.ws, "steps": steps, "warmup": warm, "ms_per_step": kernel_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": wl["precision"], "data": "synthetic",
        "config": {"workload": wl["desc"], "cells": n, "parallelism": f"replicas{ctx.ws}",
                   "l2": "working set ~%.2f GB > 129 MB L2, no flush needed" % (
                       (2 * 4 + 8) * n * (4 if wl["precision"] == "f32" else 8) / 1e9 + 16 * n / 1e9),
                   "steps_before_timed": warm, "simulated_time_s": info["t"], "reorder": "hilbert",
                   "graph_steps": 48, "launch_shape": _shape_key(shape), "autotune": shape},
        "roofline": roof,
        "gpu_launches": steps * (2 if shape.get("edge_pass") else 1),
        "clocks": clk,
    }
    m.close()
    if not e2e:
        return rec, mi
    # ---- end to end through the C ABI with pinned host buffers ----
    hp = [torch.from_numpy(a.astype(npdt)).pin_memory() for a in (mi.h, mi.hu, mi.hv)]
    out = [torch.empty(n, dtype=tdt).pin_memory() for _ in range(3)]
    # a mesh with the timed run's launch shape (tuned once above, as a user
    # would tune once and create later meshes with the chosen shape)
    keys = ("block_size", "min_blocks", "stages", "geometry_early", "activity", "edge_pass", "grid", "cell_pairs")
    m2 = capi.Mesh(mi.nodes, mi.tris, mi.z, mi.manning, precision=prec, device=ctx.local,
                   **{k: int(shape[k]) for k in keys})
    for pairs, kind, value in mi.bcs:
        m2.set_bc(pairs, kind, value)
    m2.set_stream(ctx.stream)
    m2.set_state(*hp)
    m2.step(warm, 0.9)   # the same warm-up: any step graph is captured before the timed jobs
    m2.get_state(out)
    for _ in range(2):   # two untimed jobs: first-use costs of the copies stay out of the timed ones
        m2.set_state(*hp)
        m2.step(steps, 0.9, sync=False)
        m2.get_state(out)
    if ctx.dist:
        ctx.dist.barrier()
    torch.cuda.synchronize(ctx.dev)
    jobs = []
    for _ in range(3):   # three identical jobs, each timed whole; the median is reported
        t0 = time.perf_counter()
        m2.set_state(*hp)
        m2.step(steps, 0.9, sync=False)
        m2.get_state(out)
        jobs.append(time.perf_counter() - t0)
    m2.close()
    e2e_s = max_over_ranks(ctx.dist, [sorted(jobs)[1]])[0]
    rec["e2e"] = {"value": ctx.ws * n * steps / e2e_s, "unit": "cell-updates/s",
                  "h2d_bytes_per_step": 3 * n * np.dtype(npdt).itemsize / steps,
                  "d2h_bytes_per_step": 3 * n * np.dtype(npdt).itemsize / steps, "jobs_s": jobs,
                  "note": "one job: swe_set_state from pinned host arrays, swe_step(steps), swe_get_state to "
                          "pinned host arrays, timed whole; median of three jobs; bytes averaged per step; a "
                          "second mesh created with the device run's launch shape"}
    return rec, mi


def measure_ensemble(ctx, name, steps, warmup, ens_shape=None):
    """All members in one CUDA-graph launch per call, against the plain
    solver launched member after member on the same stream (first with the
    library's default launch shapes, then with every member autotuned)."""
    torch, capi = ctx.torch, ctx.capi
    wl = WORKLOADS[name]
    prec = capi.SWE_FP32 if wl["precision"] == "f32" else capi.SWE_FP64
    npdt = np.float32 if prec == capi.SWE_FP32 else np.float64
    mis = ctx.make_input(name)
    if MEMBERS[1] != "all":   # the canal (even) or river (odd) members alone, for profiling
        mis = [mi for mi in mis if (mi.meta["member"] % 2 == 1) == (MEMBERS[1] == "river")]
    meshes = []
    for mi in mis:
        m = capi.Mesh(mi.nodes, mi.tris, mi.z, mi.manning, precision=prec, device=ctx.local)
        for pairs, kind, value in mi.bcs:
            m.set_bc(pairs, kind, value)
        m.set_stream(ctx.stream)
        m.set_state(mi.h.astype(npdt), mi.hu.astype(npdt), mi.hv.astype(npdt))
        meshes.append(m)
    n = sum(mi.n_cells for mi in mis)
    ens = capi.Ensemble(meshes)
    ens.set_stream(ctx.stream)
    if ens_shape:
        v = [int(x) for x in ens_shape.split(",")]
        keys = ("block_size", "min_blocks", "stages", "geometry_early", "activity", "edge_pass", "dynamic", "chunk",
                "grid", "cell_pairs", "queue")
        if len(v) not in (len(keys) - 2, len(keys) - 1, len(keys)):
            raise SystemExit("--ens-shape needs " + ",".join(keys[:-2]) + "[,cell_pairs[,queue]]")
        shape = dict(zip(keys, v))
        ens.set_shape(**shape)
        shape["fixed"] = True
    else:
        shape = ens.autotune(4)   # on the initial states, which the trials leave untouched
    # warm-up: the timed call's graph is captured (for its step phase mod 6)
    # before the timed region, which then starts at the same phase
    warm = max(warmup, 6)
    warm += (-warm) % 6
    ens.step(warm)
    ens.step(steps)
    realign = (-steps) % 6
    if realign:
        ens.step(realign)
    warm_total = warm + steps + realign
    active0 = ens.info(0)["n_active"]
    ms, clk = ctx.timed(lambda: ens.step(steps, sync=False))
    active_frac = (ens.info(0)["n_active"] - active0) / float(n * steps)
    member_shapes = []
    if MEMBERS[2]:   # profiling the batched kernel alone: no per-member launches
        ms_default = ms_plain = float("nan")
    else:
        # per-member launches of the plain solver, the same number of steps
        for m in meshes:
            m.step(48)
        ms_default, _ = ctx.timed(lambda: [m.step(steps, 0.9, sync=False) for m in meshes])
        for m in meshes:
            m.step(96)
            member_shapes.append(m.autotune(4))
            m.step(48)
        ms_plain, _ = ctx.timed(lambda: [m.step(steps, 0.9, sync=False) for m in meshes])
    peak, peak_kind = _peaks()
    kernel_ms = ms / steps
    roof = _hbm_roofline(wl, n, kernel_ms, active_frac, shape.get("activity"), name, shape, peak, peak_kind,
                         ensemble=True)
    roof["traffic"], roof["traffic_frac"] = None, None
    if wl["precision"] == "f64":
        roof = _fp64_roofline(n, kernel_ms, active_frac, shape.get("edge_pass"), roof)
    rec = {
        "metric": "cell-updates/s", "value": ctx.ws * n * steps / (ms * 1e-3), "unit": "cell-updates/s",
        "n_gpus": ctx.ws, "steps": steps, "warmup": warm_total, "ms_per_step": kernel_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": wl["precision"],
        "data": "synthetic",
        "config": {"workload": wl["desc"] + ("" if MEMBERS[1] == "all" else f" (the {MEMBERS[1]} members only)"),
                   "cells": n, "members": len(mis), "parallelism": f"replicas{ctx.ws}",
                   "l2": "working set > 129 MB L2, no flush needed", "steps_before_timed": warm_total,
                   "launch_shape": _shape_key(shape), "autotune": shape,
                   "member_shapes": sorted({tuple(_shape_key(t)[:6]) + ((1,) if t.get("cell_pairs") else ())
                                            for t in member_shapes})},
        "roofline": roof,
        "per_member_launches": {"value": ctx.ws * n * steps / (ms_plain * 1e-3), "unit": "cell-updates/s",
                                "ms_per_step": ms_plain / steps,
                                "note": "the plain solver on each member in turn, each member autotuned"},
        "speedup_vs_per_member": ms_plain / ms,
        "per_member_launches_default_shapes": {"value": ctx.ws * n * steps / (ms_default * 1e-3),
                                               "unit": "cell-updates/s", "ms_per_step": ms_default / steps,
                                               "speedup": ms_default / ms},
        # the edge pass and the split step launch two kernels per step
        "gpu_launches": steps * (2 if shape.get("edge_pass") or shape.get("cell_pairs") else 1),
        "clocks": clk,
    }
    if MEMBERS[2]:
        for k in ("per_member_launches", "speedup_vs_per_member", "per_member_launches_default_shapes"):
            rec[k] = None
    ens.close()
    for m in meshes:
        m.close()
    return rec


def measure_adjoint(ctx, name, steps, warmup, shape_spec=None):
    """Forward run plus reverse sweep of the discrete adjoint; a bench step is
    one time step of the forward and its reverse (recompute + two adjoint
    kernels)."""
    torch, capi = ctx.torch, ctx.capi
    from paper_2010_14416_gb300 import meshgen
    mi = ctx.make_input(name)
    n = mi.n_cells
    gauges = meshgen.gauge_cells(n, 64, seed=1)
    xi = meshgen.perturbation(n, 101)
    fixed = _shape_kwargs(shape_spec)

    def mesh(z, man):
        m = capi.Mesh(mi.nodes, mi.tris, z, man, precision=capi.SWE_FP64, device=ctx.local, **fixed)
        for pairs, kind, value in mi.bcs:
            m.set_bc(pairs, kind, value)
        m.set_stream(ctx.stream)
        m.set_state(mi.h, mi.hu, mi.hv)
        return m

    # seeded target: the same run with perturbed Manning and bed
    tm = mesh(mi.z + 0.05 * xi, mi.manning * (1 + 0.1 * xi))
    tm.step(steps, 0.9)
    target = tm.get_state()[0][gauges]
    tm.close()
    m = mesh(mi.z, mi.manning)
    gm = torch.empty(n, dtype=torch.float64, device=ctx.dev)
    gz = torch.empty(n, dtype=torch.float64, device=ctx.dev)
    # launch shape of the forward and recomputed steps, chosen by the autotuner
    shape = dict(fixed, chunk=0, fixed=True) if fixed else m.autotune(4)
    warm = max(warmup, 3)
    m.adjoint(warm, gauges, target, checkpoint_every=50, out=(gm, gz))
    m.set_state(mi.h, mi.hu, mi.hv)
    res = {}
    ms, clk = ctx.timed(lambda: res.update(r=m.adjoint(steps, gauges, target, checkpoint_every=50, out=(gm, gz))))
    loss = res["r"][0]
    # the forward alone, the same steps from the same state, for the ratio
    m.set_state(mi.h, mi.hu, mi.hv)
    m.step(_warmup_for(steps, 0), 0.9)
    m.set_state(mi.h, mi.hu, mi.hv)
    ms_fwd, _ = ctx.timed(lambda: m.step(steps, 0.9, sync=False))
    rec = {
        "metric": "cell-updates/s", "value": ctx.ws * n * steps / (ms * 1e-3), "unit": "cell-updates/s",
        "n_gpus": ctx.ws, "steps": steps, "warmup": warm, "ms_per_step": ms / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[name]["desc"], "cells": n, "parallelism": f"replicas{ctx.ws}",
                   "checkpoint_every": 50, "gauges": 64, "autotune": shape,
                   "steps_before_timed": warm, "note": "the warm-up is an adjoint call of `warmup` steps"},
        "loss": loss,
        "grad_norms": {"manning": float(gm.norm()), "bathy": float(gz.norm())},
        "forward_only": {"value": n * steps / (ms_fwd * 1e-3), "ms_per_step": ms_fwd / steps},
        "adjoint_over_forward": ms / ms_fwd,
        "roofline": {"bound": "alu", "note": "FP64 arithmetic on forward-mode duals and hand-written "
                                             "transposes: the adjoint kernels and the forward steps are bound "
                                             "by the FP64 pipe"},
        # per step: the forward step and its recomputation (two kernels each with the
        # edge pass), then the two adjoint kernels
        "gpu_launches": steps * (2 * (2 if shape.get("edge_pass") else 1) + 2),
        "clocks": clk,
    }
    m.close()
    return rec


def _measure(ctx, name, steps, warmup, args, e2e):
    if WORKLOADS[name]["maker"] == "ensemble":
        return measure_ensemble(ctx, name, steps, warmup, args.ens_shape), None
    if name.startswith("adjoint"):
        return measure_adjoint(ctx, name, steps, warmup, args.shape), None
    return measure_mesh(ctx, name, steps, warmup, args.shape, e2e=e2e)


# the other workloads, reported beside the headline in the default run with
# step counts that keep the whole command within a few minutes
SUBRECORDS = {
    "river13m_wet_fp32": dict(steps=200, warmup=6),
    "canal1m_fp64": dict(steps=200, warmup=6),
    "ensemble256_fp32": dict(steps=96, warmup=6),
    "ensemble256_fp64": dict(steps=24, warmup=6),
    "adjoint1m_fp64": dict(steps=200, warmup=3),
}


def _compact(rec):
    keep = ("value", "unit", "ms_per_step", "steps", "warmup", "dtype", "roofline", "speedup_vs_per_member",
            "per_member_launches", "per_member_launches_default_shapes", "adjoint_over_forward", "forward_only",
            "grad_norms", "loss", "gpu_launches", "clocks")
    out = {k: rec[k] for k in keep if k in rec}
    cfg = rec.get("config", {})
    out["config"] = {k: cfg[k] for k in ("workload", "cells", "members", "launch_shape", "steps_before_timed",
                                         "checkpoint_every", "gauges") if k in cfg}
    return out


def run_gpu(args, name, subrecords):
    ctx = GpuContext()
    rec, mi = _measure(ctx, name, args.steps, args.warmup, args, e2e=True)
    if mi is not None and ctx.rank == 0 and ctx.ws == 1 and not args.no_cpu_baseline:
        rec["cpu_baseline"] = cpu_baseline(mi, args.cpu_budget)
    if subrecords:
        rec["subrecords"] = {}
        for sub, sp in SUBRECORDS.items():
            if sub == name:
                continue
            r, _ = _measure(ctx, sub, sp["steps"], sp["warmup"], args, e2e=False)
            rec["subrecords"][sub] = _compact(r)
    if ctx.rank == 0:
        print(json.dumps(rec), flush=True)
    if ctx.dist:
        ctx.dist.barrier()
        ctx.dist.destroy_process_group()
    return 0


def _shape_kwargs(spec):
    """Mesh keyword arguments of a --shape string (empty: autotune)."""
    if not spec:
        return {}
    v = [int(x) for x in spec.split(",")]
    if len(v) not in (7, 8):
        raise SystemExit("--shape needs block,min_blocks,stages,geometry_early,activity,edge_pass,grid[,cell_pairs]")
    keys = ("block_size", "min_blocks", "stages", "geometry_early", "activity", "edge_pass", "grid", "cell_pairs")
    return dict(zip(keys, v))


def _shape_key(t):
    """(block, min_blocks, stages, geometry_early, activity, edge_pass, grid[, chunk, dynamic][, 1 for the
    cell-pair kernel]) of an autotuner choice."""
    k = [t["block_size"], t["min_blocks"], t["stages"], t["geometry_early"], t["activity"], t["edge_pass"],
         t["grid"]]
    pairs = [1] if t.get("cell_pairs") else []
    if t.get("chunk"):
        return k + [t["chunk"], t.get("dynamic", 0)] + pairs
    return k + pairs


def _kernel_hash():
    import hashlib
    hsh = hashlib.sha1()
    for f in ("swe_kernels.cuh", "swe_launch.cuh", "swe_f32.cuh"):
        with open(os.path.join(ROOT, "paper_2010_14416_gb300", "csrc", f), "rb") as fh:
            hsh.update(fh.read())
    return hsh.hexdigest()[:12]


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=12)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=None,
                    help="one workload alone (default: the 13M river, with every other workload as a sub-record)")
    ap.add_argument("--no-subrecords", action="store_true",
                    help="the default run without the other workloads' sub-records")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--members", type=int, default=256, help="ensemble workloads: number of members")
    ap.add_argument("--member-kind", choices=["all", "canal", "river"], default="all",
                    help="ensemble workloads: all members, or only the canal (even) or river (odd) ones")
    ap.add_argument("--batched-only", action="store_true",
                    help="ensemble workloads: time the batched step alone, without the per-member launches "
                         "(for profiling)")
    ap.add_argument("--ens-shape", default=None,
                    help="ensemble workloads: block,min_blocks,stages,geometry_early,activity,edge_pass,dynamic,chunk,grid"
                         "[,cell_pairs[,queue]] "
                         "-- use this launch shape instead of autotuning (for profiling)")
    ap.add_argument("--shape", default=None,
                    help="mesh workloads: block,min_blocks,stages,geometry_early,activity,edge_pass,grid -- use "
                         "this launch shape instead of autotuning (for profiling the shape a tuned run chose)")
    args = ap.parse_args()
    explicit = args.workload is not None
    name = args.workload or "river13m_fp32"
    if args.steps is None:
        args.steps = WORKLOADS[name]["steps"]
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args, name)
    MEMBERS[0] = args.members
    MEMBERS[1] = args.member_kind
    MEMBERS[2] = args.batched_only
    subrecords = not explicit and not args.no_subrecords
    return run_gpu(args, name, subrecords)


if __name__ == "__main__":
    sys.exit(main())
