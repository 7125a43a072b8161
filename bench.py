"""Throughput benchmark of the compact 8th-order GKS on GB300 (FP64 cell-updates/s).

A step is one full two-stage fourth-order time step of the whole grid (CFL time step, both
stages of reconstruction + gas-kinetic flux + Gauss-theorem update).  The default run prints one
JSON line with three measurements:

  value    the plain sweep of the 2D isentropic vortex on a 2048^2 periodic grid (vortex strength 5
           on free stream (1,1,1,1), [0,10]^2, CFL 0.5), K steps, state (3 x 12 planes, 1.2 GB)
           resident in HBM and larger than L2; with its roofline, per-kernel times, e2e through the
           C ABI from pinned host buffers and the oracle's CPU rate
  batched  256 uneven periodic grids (acoustic pulses, N log-uniform in [64, 512], seed 1570): K
           steps of the batched persistent launch (cgks_batch_step, autotuned) against one grid per
           launch, overall and per size class
  served   a prefix of the seeded Poisson request stream (seed 2001, grids 128^2..2048^2,
           100..2000 steps, pulse / vortex / Mach 1.05..1.5 shock-vortex) at the stated grid sizes
           and step counts through the continuous-batching server, saturated (all requests at once)
           (least remaining work first, and every solve in every round) and capacity-matched
           (arrivals time-scaled to ~70 % of the saturated capacity), against the same requests
           solved one after another; p50/p99 latency

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cgks|reference] [--workload NAME]

--no-batched / --no-served drop those records.  Other workloads (plain sweeps unless noted):
vortex256/512/1024, shockvortex1024x512 (--order 6 runs the compact 6th-order variant of the
reconstruction), batched256 and acoustic1d (2048 copies of the 1D acoustic-wave test, 12-48 cells
each) as batched-vs-plain lines, served (the served record alone).

--impl reference times the CPU oracle (test infrastructure, plain FP64 C) on a bounded sample of
the same workload on the host cores.  Prints one JSON line (rank 0).
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
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

L2_BYTES = 129e6   # GB300 L2 capacity
METRIC = "FP64 cell-updates/s on 1 GB300 (plain 2048^2 sweep); served-batched vs plain; p50/p99 solve latency"
UNIT = "cell-updates/s"

# Algorithmic FP64 operations per cell and stage (FMA = 2) on the 256^2 vortex, where every kernel does
# exactly the method's work (no halo recomputation, every face once): two face-row records (1,888
# each: linear P7 + WENO-Z pair of 4 variables), two face segments (3,076.44 in stage 1, 2,878.44 in
# stage 2: two Gauss points each) and the update (80 / 121).  The kernels issue their adds and
# multiplies as DFMAs, so the operations are counted by ncu on a build with plain adds and
# multiplies; each per-unit figure is the smallest count of the formulations measured (the current
# code spends 1,916 per record and 3,076.44 / 2,878.44 per segment).
# The compact 6th-order variant (--order 6) changes only the record kernel's linear reconstruction:
# 1,840 per face row with WENO-Z.
RECORD_FLOP_PER_CELL = {8: 3776.0, 6: 3680.0}
FLUX_FLOP_PER_CELL = {1: 6152.88, 2: 5756.88}
UPDATE_FLOP_PER_CELL = {1: 80.0, 2: 121.0}
FLOP_PER_CELL = {s: RECORD_FLOP_PER_CELL[8] + FLUX_FLOP_PER_CELL[s] + UPDATE_FLOP_PER_CELL[s] for s in (1, 2)}
# The same per-cell counts taken from the kernels' formulas rather than from an instruction stream:
# a host build of the kernels' device arithmetic with a counting FP64 type, run over one step of the
# 2048^2 bench grid (python -m paper_2001_01570_gb300.opcount 2048), counting add/sub/mul 1, fma 2 and
# every divide, square root, reciprocal, exponential and erfc as 1 however the GPU expands it.
OPCOUNT_FLOP_PER_CELL = {"records": 3733.73, "flux": {1: 5398.63, 2: 5050.46}, "update": {1: 80.0, 2: 71.0}}
TRAFFIC_TILE = "8x16"     # the tile shape the DRAM bytes below were captured on
# DRAM bytes (read + write) per cell of one stage-1 flux-kernel launch with 8x16 tiles: ncu
# dram__bytes_{read,write}.sum of the current kernel on the 1024^2 vortex (records and state larger
# than L2), 478.90 + 244.60 MB, divided by the cells; the 2048^2 bench grid moves the same bytes per
# cell (its launch is too large to capture under the profiling size rule).
FLUX_DRAM_BYTES_PER_CELL = {1: (478.897664e6 + 244.597504e6) / 1048576}
# algorithmic bytes per cell of the flux kernel: the two face rows' records (2 x 28 doubles) read and
# the two faces' results written (stage 1: 16 doubles each, stage 2: 8)
FLUX_ALGO_BYTES_PER_CELL = {1: 448 + 256, 2: 448 + 128}
# FP64 peak of this GB300: DFMA with register operands issues 1.99 per SM and cycle (measured by
# paper_2001_01570_gb300.diag, FMA = 2 flops; the nominal 1.25 TFLOP/s at 2070 MHz on 152 SMs is
# 1.99 too).  The peak is taken at the median SM clock sampled during the timed region
# (1.252 TFLOP/s at 2070 MHz).
FP64_DFMA_PER_SM_CYCLE = 1.99
DEFAULT_SM_MHZ = 2070.0


def fp64_peak_tflops(nsm, sm_mhz):
    return 2.0 * FP64_DFMA_PER_SM_CYCLE * nsm * sm_mhz * 1e6 / 1e12


def workloads():
    from paper_2001_01570_gb300 import workloads as wl
    return {
        "vortex2048": lambda: wl.isentropic_vortex(2048),
        "vortex512": lambda: wl.isentropic_vortex(512),
        "vortex1024": lambda: wl.isentropic_vortex(1024),
        "vortex256": lambda: wl.isentropic_vortex(256),
        "shockvortex1024x512": lambda: wl.shock_vortex(1024, 512),
    }


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "samples": len(sm), "reasons": sorted(reasons)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "cgks":
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if args.impl == "cgks" else "gloo")
    return world, rank, local


def barrier_max(world, value):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_sample(seconds_target=12.0, n=96, threads=None, order=8):
    """Time the CPU oracle (as it stands) on a bounded sample of the vortex workload: the same
    initial condition on an n x n grid (cost per cell-update is independent of grid size)."""
    import oracle as O
    from paper_2001_01570_gb300 import workloads as wl
    spec, W = wl.isentropic_vortex(n)
    spec.order = order
    P = O.make_problem(**spec.as_kwargs())
    cores = threads or os.cpu_count()
    os.environ["OMP_NUM_THREADS"] = str(cores)
    O.run(P, W, 1, threads=cores)                       # warm-up (compile/load)
    steps, t0 = 0, time.perf_counter()
    Wc = W
    while True:
        Wc, _, _, _ = O.run(P, Wc, 1, threads=cores)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds_target:
            break
    rate = n * n * steps / el
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"isentropic vortex {n}x{n} periodic{'' if order == 8 else ', 6th-order variant'}, "
                      f"{steps} steps ({el:.1f} s), OpenMP over rows"}


def run_reference(args, world, rank):
    if rank != 0:
        return
    cb = oracle_sample(seconds_target=max(5.0, min(20.0, 2.0 * args.steps)), order=args.order)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload} (oracle on a bounded sample)"},
            "cpu_baseline": cb, "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_cgks(args, world, rank, local):
    import torch
    from paper_2001_01570_gb300 import build as libbuild
    from paper_2001_01570_gb300 import cgks

    libbuild.build()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    spec, W = workloads()[args.workload]()
    spec.order = args.order
    cells = spec.cells
    solver = cgks.Solver(cgks.problem_from_spec(spec), stream=stream.cuda_stream)
    if args.tile:
        cgks.cgks_set_tile_shape(solver.handle, args.tile)
    solver.set_state(W)

    # warm-up (also fills the per-kernel shared-memory configuration)
    solver.step(args.warmup)
    torch.cuda.synchronize()

    # ---------------- device-resident throughput: K steps, events on the solver's stream
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        start.record(stream)
        cgks.cgks_step(solver.handle, args.steps)
        stop.record(stream)
        torch.cuda.synchronize()
    launches = cgks.cgks_last_launch_count()
    ms = start.elapsed_time(stop)
    ms = barrier_max(world, ms)
    value = world * cells * args.steps / (ms * 1e-3)
    clocks = clk.summary()

    # ---------------- per-kernel durations (events around every launch) for the roofline
    prof_steps = max(2, min(args.steps, 5))
    stage_ms = cgks.cgks_step_profiled(solver.handle, prof_steps)
    tile = args.tile or cgks.cgks_tile_shape(solver.handle)
    # stage_ms: begin, stage-1 records, flux, update, stage-2 records, flux, update, end
    flux_ms, rec_ms, upd_ms = stage_ms[2], stage_ms[1], stage_ms[3]
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    peak_mhz = clocks["sm_mhz"] if clocks else DEFAULT_SM_MHZ
    peak = fp64_peak_tflops(nsm, peak_mhz)
    achieved = FLUX_FLOP_PER_CELL[1] * cells / (flux_ms * 1e-3) / 1e12
    rec_flop = RECORD_FLOP_PER_CELL[args.order]
    stage1_flop = None if rec_flop is None else rec_flop + FLUX_FLOP_PER_CELL[1] + UPDATE_FLOP_PER_CELL[1]
    stage1 = None if stage1_flop is None else stage1_flop * cells / ((flux_ms + rec_ms + upd_ms) * 1e-3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": FLUX_DRAM_BYTES_PER_CELL[1] * cells if tile == TRAFFIC_TILE else None,
                "algorithmic_bytes": FLUX_ALGO_BYTES_PER_CELL[1] * cells,
                "algorithmic_flop_per_cell": FLUX_FLOP_PER_CELL[1],
                "kernel": f"stage_kernel<{tile},1>", "kernel_ms": flux_ms,
                "stage1_records_plus_flux": {"kernels": "records_kernel<1,0> + stage_kernel<%s,1> + update_kernel<1>" % tile,
                                             "ms": flux_ms + rec_ms + upd_ms, "achieved": stage1,
                                             "frac": None if stage1 is None else stage1 / peak,
                                             "algorithmic_flop_per_cell": stage1_flop,
                                             "state_algorithmic_bytes": 288 * cells},
                "peak_source": "measured FP64 DFMA rate (register operands, FMA = 2): %.2f per SM and cycle x %d SMs "
                               "x %.0f MHz (median SM clock in the timed region), of measured"
                               % (FP64_DFMA_PER_SM_CYCLE, nsm, peak_mhz)}
    # the same kernels against the operation count of their formulas (exp, erfc, reciprocal,
    # divide, square root one operation each): the convention of the algorithmic FP64 count
    oc_flux = OPCOUNT_FLOP_PER_CELL["flux"][1]
    oc_stage1 = OPCOUNT_FLOP_PER_CELL["records"] + oc_flux + OPCOUNT_FLOP_PER_CELL["update"][1]
    oc_ach = oc_flux * cells / (flux_ms * 1e-3) / 1e12
    oc_stage1_ach = oc_stage1 * cells / ((flux_ms + rec_ms + upd_ms) * 1e-3) / 1e12
    roofline["formula_count"] = {
        "convention": "add/sub/mul 1, fma 2, div/sqrt/rcp/exp/erfc 1 each (host count of the kernels' formulas, "
                      "python -m paper_2001_01570_gb300.opcount 2048)",
        "algorithmic_flop_per_cell": oc_flux, "achieved": oc_ach, "frac": oc_ach / peak,
        "stage1_algorithmic_flop_per_cell": oc_stage1, "stage1_achieved": oc_stage1_ach,
        "stage1_frac": oc_stage1_ach / peak}

    # ---------------- the fused step (both stages of a step in one launch, W* in shared memory)
    # on the same grid from the same initial state
    fused = None
    if spec.dim == 2:
        fsteps = max(2, min(args.steps, 10))
        solver.set_state(W)
        cgks.cgks_step_fused(solver.handle, 2)
        torch.cuda.synchronize()
        with ClockSampler(local) as fclk:
            start.record(stream)
            cgks.cgks_step_fused(solver.handle, fsteps)
            stop.record(stream)
            torch.cuda.synchronize()
        flaunch = cgks.cgks_last_launch_count()
        fms = barrier_max(world, start.elapsed_time(stop))
        fused = {"kernel": "fused_step_kernel<16,8> (one launch per step between the step-control kernels)",
                 "steps": fsteps, "ms_per_step": fms / fsteps, "value": world * cells * fsteps / (fms * 1e-3),
                 "vs_three_kernel_step": (ms / args.steps) / (fms / fsteps), "gpu_launches": flaunch,
                 "clocks": fclk.summary()}

    # ---------------- end to end through the C ABI with host buffers
    host_in = torch.from_numpy(np.ascontiguousarray(W)).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    e2e_reps = 1
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_reps):
        cgks.cgks_set_state(solver.handle, host_in.numpy())
        cgks.cgks_step(solver.handle, args.steps)
        cgks.cgks_get_state(solver.handle, host_out.numpy())
    el = time.perf_counter() - t0
    el = barrier_max(world, el)
    e2e_value = world * cells * args.steps * e2e_reps / el
    nbytes = host_in.numel() * 8

    solver.close()
    if rank != 0:
        return None
    cpu = None if args.no_cpu_baseline or world > 1 else oracle_sample(order=args.order)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload + ("" if args.order == 8 else " (compact 6th-order variant)"),
                   "order": args.order, "cells": cells, "grid": [spec.nx, spec.ny],
                   "cfl": spec.cfl,
                   "l2": ("inputs larger than L2 (3 x 12 planes resident, %.2f GB)" % (36 * cells * 8 / 1e9)
                          if 36 * cells * 8 > L2_BYTES else
                          "state (3 x 12 planes, %.3f GB) fits in L2 and is not flushed between steps" % (36 * cells * 8 / 1e9)),
                   "parallelism": "one grid per GPU (independent replicas)" if world > 1 else "single GPU"},
        "roofline": roofline,
        "stage_ms": {"begin": stage_ms[0], "records1": stage_ms[1], "flux1": stage_ms[2], "update1": stage_ms[3],
                     "records2": stage_ms[4], "flux2": stage_ms[5], "update2": stage_ms[6], "end": stage_ms[7]},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nbytes / args.steps,
                "d2h_bytes_per_step": nbytes / args.steps,
                "note": "per repetition: H2D of the 12 state planes from pinned host memory, K steps, D2H of the state"},
        "gpu_launches": launches,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "fused_step": fused,
    }
    return line


def _pulse_ic(p):
    from paper_2001_01570_gb300 import workloads as wl
    spec, W = wl.acoustic_pulse(p["N"], p["A"], p["b"], p["cx"], p["cy"])
    return spec, W


def _acoustic_ic(p):
    from paper_2001_01570_gb300 import workloads as wl
    return wl.acoustic_wave_1d(p["N"], eps_tau=0.0)


def _request_ic(req):
    from paper_2001_01570_gb300 import workloads as wl
    return wl.request_problem(req)


def _parallel_ics(fn, items):
    """Initial conditions in a spawn pool (fresh interpreters: safe after the first CUDA call)."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(min(len(items), os.cpu_count() or 4)) as pool:
        return pool.map(fn, items)


TUNE_STEPS = 12   # steps the batched autotuner times its candidates on (4 tile shapes, then 2 more
                  # cells-per-thread counts of the update kernel, one untimed and one timed step each)


def measure_batched(args, local, ics, steps, classes=None):
    """One grid per launch (cgks_step per grid, each timed with CUDA events) against the batched
    persistent launch over all grids (cgks_batch_step, warmed up through the autotuner), both for
    `steps` steps from the same state; `classes` maps a label to the indices of a size class, each
    also batched on its own."""
    import torch
    from paper_2001_01570_gb300 import cgks
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    solvers = []
    for spec, W in ics:
        s = cgks.Solver(cgks.problem_from_spec(spec), stream=stream.cuda_stream)
        s.set_state(W)
        solvers.append(s)
    cells = [spec.cells for spec, _ in ics]
    handles = [s.handle for s in solvers]
    for s in solvers:
        s.step(args.warmup)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in solvers]
    launches_plain = 0
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk_plain:
        start.record(stream)
        for s, (a, b) in zip(solvers, ev):
            a.record(stream)
            cgks.cgks_step(s.handle, steps)
            b.record(stream)
            launches_plain += cgks.cgks_last_launch_count()
        stop.record(stream)
        torch.cuda.synchronize()
    ms_plain = start.elapsed_time(stop)
    per_grid_ms = [a.elapsed_time(b) for a, b in ev]

    def batched(idx):
        hs = [handles[k] for k in idx]
        cgks.cgks_batch_step(hs, max(args.warmup, TUNE_STEPS))
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            start.record(stream)
            cgks.cgks_batch_step(hs, steps)
            stop.record(stream)
            torch.cuda.synchronize()
        shape, cpt = cgks.cgks_batch_tile_shape(hs), cgks.cgks_batch_update_cpt(hs)
        return (start.elapsed_time(stop), cgks.cgks_last_launch_count(), clk.summary(),
                cgks.TILE_SHAPES[shape] if shape >= 0 else None, cpt)

    ms_batch, launches, clocks, shape, cpt = batched(list(range(len(solvers))))
    total = sum(cells) * steps
    rec = {"grids": len(solvers), "cells": sum(cells), "steps": steps,
           "value": total / (ms_batch * 1e-3), "ms_per_step": ms_batch / steps, "gpu_launches": launches,
           "tile_shape": shape, "update_cells_per_thread": cpt, "clocks": clocks,
           "plain": {"value": total / (ms_plain * 1e-3), "ms_per_step": ms_plain / steps,
                     "gpu_launches": launches_plain, "clocks": clk_plain.summary()}}
    rec["batched_vs_plain"] = rec["value"] / rec["plain"]["value"]
    if classes:
        rec["size_classes"] = {}
        for label, idx in classes.items():
            if not idx:
                continue
            work = sum(cells[k] for k in idx) * steps
            ms_p = sum(per_grid_ms[k] for k in idx)
            ms_b, _, _, shp, cp = batched(idx)
            rec["size_classes"][label] = {"grids": len(idx), "plain": work / (ms_p * 1e-3),
                                          "batched": work / (ms_b * 1e-3), "batched_vs_plain": ms_p / ms_b,
                                          "tile_shape": shp, "update_cells_per_thread": cp}
    for s in solvers:
        s.close()
    return rec


def batched_record(args, local):
    """Config 4: the 256 uneven grids, seed 1570, `--steps` steps."""
    from paper_2001_01570_gb300 import workloads as wl
    params = wl.batched_pulses(seed=1570, count=args.grids)
    ics = _parallel_ics(_pulse_ic, params)
    N = [p["N"] for p in params]
    classes = {"64-128": [k for k, n in enumerate(N) if n < 128],
               "128-256": [k for k, n in enumerate(N) if 128 <= n < 256],
               "256-512": [k for k, n in enumerate(N) if n >= 256]}
    rec = measure_batched(args, local, ics, args.batched_steps or args.steps, classes)
    rec["workload"] = (f"batched{args.grids}: periodic acoustic pulses, N log-uniform in [64, 512], A log-uniform "
                       "in [1e-5, 1e-3], half-width 3..10 cells, seed 1570")
    rec["l2"] = "state of all grids (%.2f GB) larger than L2" % (36 * rec["cells"] * 8 / 1e9)
    return rec


def _serve_pass(cgks, local, reqs, ics, arrival_scale, args, order=None):
    """Submit the requests at their stream arrival times x arrival_scale (0: all at once) and wait
    for every result; the server's statistics."""
    order = cgks.CGKS_SERVE_LEAST_WORK_FIRST if order is None else order
    srv = cgks.cgks_serve_start(hbm_budget_bytes=120e9, max_active=args.max_active,
                                steps_per_round=args.steps_per_round,
                                tile_shape=cgks.TILE_SHAPES.index(args.tile) if args.tile else -1, order=order)
    ids = []
    t0 = time.perf_counter()
    try:
        with ClockSampler(local) as clk:
            for r, (spec, W) in zip(reqs, ics):
                delay = (r["arrival"] - reqs[0]["arrival"]) * arrival_scale - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
                ids.append(cgks.cgks_serve_submit(srv, cgks.problem_from_spec(spec), W, r["steps"]))
            for rid, (spec, W) in zip(ids, ics):
                out = np.empty_like(W)
                cgks.cgks_serve_wait(srv, rid, 3600.0, out)
            stats = cgks.cgks_serve_stats(srv)
    finally:
        cgks.cgks_serve_stop(srv)
    keep = ("cell_updates_per_s", "p50_s", "p99_s", "mean_s", "wall_s", "busy_s", "gpu_s", "round_overhead",
            "rounds", "completed", "failed", "hbm_peak", "tile_shape", "update_cpt", "graph_captures")
    out = {k: stats[k] for k in keep}
    out["value"] = out.pop("cell_updates_per_s")
    out["tile_shape"] = cgks.TILE_SHAPES[out["tile_shape"]] if out["tile_shape"] >= 0 else None
    out["order"] = "least remaining work first (4e6 cells per round)" if order == cgks.CGKS_SERVE_LEAST_WORK_FIRST \
        else "every admitted solve in every round"
    out["clocks"] = clk.summary()
    return out


def served_record(args, local, ablation=False):
    """Config 5: a prefix of the seeded request stream at the stated sizes and step counts.
    ablation: also the saturated run with every admitted solve in every round (the default run
    leaves it out to stay within a few minutes)."""
    import torch
    from paper_2001_01570_gb300 import cgks
    from paper_2001_01570_gb300 import workloads as wl
    reqs = wl.served_requests(seed=2001)[: args.requests]
    ics = _parallel_ics(_request_ic, reqs)
    torch.cuda.set_device(local)
    work = sum(spec.cells * r["steps"] for r, (spec, _) in zip(reqs, ics))
    # one request after another, each on its own solver: allocation and copies timed apart from the steps
    alloc_copy = steps_s = 0.0
    t0 = time.perf_counter()
    with ClockSampler(local) as clk_plain:
        for r, (spec, W) in zip(reqs, ics):
            ta = time.perf_counter()
            s = cgks.Solver(cgks.problem_from_spec(spec))
            s.set_state(W)
            tb = time.perf_counter()
            s.step(r["steps"])
            tc = time.perf_counter()
            s.get_state()
            s.close()
            td = time.perf_counter()
            alloc_copy += (tb - ta) + (td - tc)
            steps_s += tc - tb
    plain_s = time.perf_counter() - t0
    plain = {"value": work / plain_s, "wall_s": plain_s, "steps_s": steps_s, "alloc_copy_s": alloc_copy,
             "steps_only_value": work / steps_s, "clocks": clk_plain.summary()}
    saturated = _serve_pass(cgks, local, reqs, ics, 0.0, args)
    saturated_all = _serve_pass(cgks, local, reqs, ics, 0.0, args, order=cgks.CGKS_SERVE_ALL_ACTIVE) \
        if ablation else None
    span = reqs[-1]["arrival"] - reqs[0]["arrival"]
    # arrivals stretched so that the offered load is 70 % of the saturated capacity
    scale = saturated["wall_s"] / (0.7 * span) if span > 0 else 1.0
    matched = _serve_pass(cgks, local, reqs, ics, scale, args)
    matched["arrival_scale"] = scale
    matched["offered_load_vs_capacity"] = 0.7
    kinds = {}
    for r in reqs:
        kinds[r["kind"]] = kinds.get(r["kind"], 0) + 1
    return {"workload": f"served: the first {len(reqs)} requests of the seeded stream (seed 2001, Poisson 50 req/s, "
                        "N log-uniform 128..2048, steps log-uniform 100..2000, pulse/vortex/shock-vortex, "
                        "Mach 1.05..1.5) at their stated N and step counts, 120 GB budget",
            "requests": len(reqs), "kinds": kinds, "cell_updates": work,
            "grids": [[spec.nx, spec.ny, r["steps"]] for r, (spec, _) in zip(reqs, ics)],
            "max_active": args.max_active, "steps_per_round": args.steps_per_round,
            "plain": plain, "saturated": saturated,
            **({"saturated_every_solve_every_round": saturated_all} if ablation else {}),
            "capacity_matched": matched,
            "served_vs_plain": saturated["value"] / plain["value"],
            "served_vs_plain_steps_only": saturated["value"] / plain["steps_only_value"]}


def run_batched_line(args, world, rank, local):
    """--workload batched256 / acoustic1d: the batched record as a line of its own."""
    from paper_2001_01570_gb300 import build as libbuild
    from paper_2001_01570_gb300 import workloads as wl
    libbuild.build()
    if args.workload == "acoustic1d":
        count = args.grids if args.grids_set else 2048
        params = wl.batched_acoustic_1d(seed=618, count=count)
        ics = _parallel_ics(_acoustic_ic, params)
        rec = measure_batched(args, local, ics, args.steps)
        rec["workload"] = f"acoustic1d: {count} 1D acoustic-wave grids, N log-uniform in [12, 48], seed 618; eps_tau = 0"
    else:
        rec = batched_record(args, local)
    if rank == 0:
        line = {"metric": "FP64 cell-updates/s, batched persistent launch vs one grid per launch",
                "value": rec["value"], "unit": UNIT, "n_gpus": world, "steps": rec["steps"], "warmup": args.warmup,
                "ms_per_step": rec["ms_per_step"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": rec["workload"]}, "batched": rec,
                "gpu_launches": rec["gpu_launches"], "clocks": rec["clocks"]}
        print(json.dumps(line), flush=True)


def run_served_line(args, world, rank, local):
    from paper_2001_01570_gb300 import build as libbuild
    libbuild.build()
    rec = served_record(args, local, ablation=True)
    if rank == 0:
        line = {"metric": "FP64 cell-updates/s, served continuous batching vs one request after another; p50/p99",
                "value": rec["saturated"]["value"], "unit": UNIT, "n_gpus": world, "steps": None, "warmup": 0,
                "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic", "config": {"workload": rec["workload"]}, "served": rec,
                "clocks": rec["saturated"]["clocks"]}
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cgks", choices=["cgks", "reference"])
    ap.add_argument("--workload", default="vortex2048")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="default run: leave out the batched record")
    ap.add_argument("--no-served", action="store_true", help="default run: leave out the served record")
    ap.add_argument("--tile", default=None, help="tile shape of the plain path (e.g. 16x7, 24x8)")
    ap.add_argument("--order", type=int, default=8, choices=[8, 6],
                    help="plain sweeps: 8 = the paper's scheme, 6 = its compact 6th-order variant")
    ap.add_argument("--grids", type=int, default=None)
    ap.add_argument("--batched-steps", type=int, default=None, help="steps of the batched record (default --steps)")
    ap.add_argument("--requests", type=int, default=12, help="served record: requests of the stream's prefix")
    ap.add_argument("--max-active", type=int, default=64)
    ap.add_argument("--steps-per-round", type=int, default=8)
    args = ap.parse_args()
    args.grids_set = args.grids is not None
    if args.grids is None:
        args.grids = 256
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload.startswith("batched") or args.workload == "acoustic1d":
        run_batched_line(args, world, rank, local)
    elif args.workload == "served":
        run_served_line(args, world, rank, local)
    else:
        line = run_cgks(args, world, rank, local)
        # the batched and served records are single-GPU measurements (under torchrun every rank
        # would run its own copy): the default run adds them at N = 1
        default = args.workload == "vortex2048" and args.order == 8 and not args.tile and world == 1
        batched = None if (args.no_batched or not default) else batched_record(args, local)
        served = None if (args.no_served or not default) else served_record(args, local)
        if rank == 0:
            if batched is not None:
                line["batched"] = batched
            if served is not None:
                line["served"] = served
            print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
