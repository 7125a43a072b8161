"""Parity at the full sizes of the stated workloads, in the launch configuration bench.py times.

The oracle cannot rerun these in a test, so tests/golden/make_golden.py (which calls only oracle/)
stored, for each case, the final time and step count, the per-plane max |value| over the whole grid
and all 12 planes at 1500 seeded cells.  The GPU runs the same seeded inputs for the same number of
steps; the sampled cells must agree to 1e-11 relative (per conserved variable, normalised by the
scale of tests/parity_util.plane_scales) and 1e-9 for the gradient planes."""
import multiprocessing as mp
import os

import numpy as np
import pytest

from conftest import GOLDEN
from parity_util import check
from paper_2001_01570_gb300 import cgks, workloads as wl

pytestmark = pytest.mark.gpu

TOL, GRAD_TOL = 1e-11, 1e-9


def _golden(name):
    path = os.path.join(GOLDEN, f"oracle_{name}.npz")
    if not os.path.exists(path):
        pytest.skip(f"golden file {path} not generated")
    return np.load(path)


def _compare(out, g, spec, name=None):
    planes = out.reshape(out.shape[0], -1)[:, g["idx"]]
    scaled, _ = check(name, planes, g["values"], dx=spec.dx, dy=spec.dy, gamma=spec.gamma, tol=TOL,
                      grad_tol=GRAD_TOL, maxabs=g["maxabs"])
    return scaled


def _run(spec, W, nsteps):
    s = cgks.Solver(cgks.problem_from_spec(spec))
    s.set_state(W)
    s.step(nsteps)
    out, t, steps = s.get_state()
    s.close()
    return out, t, steps


def test_vortex_512_200_steps():
    g = _golden("vortex512_200")
    spec, W = wl.isentropic_vortex(512)
    out, t, steps = _run(spec, W, 200)
    assert steps == int(g["steps"]) and abs(t - float(g["t"])) <= 1e-13 * float(g["t"])
    _compare(out, g, spec)


def test_vortex_2048_bench_grid_2_steps():
    """The bench's own grid and launch configuration (default tile shape, plain steps)."""
    g = _golden("vortex2048_2")
    spec, W = wl.isentropic_vortex(2048)
    out, t, steps = _run(spec, W, 2)
    assert steps == int(g["steps"]) == 2 and abs(t - float(g["t"])) <= 1e-13 * float(g["t"])
    _compare(out, g, spec)


def test_vortex_2048_sixth_order_variant_1_step():
    g = _golden("vortex2048o6_1")
    spec, W = wl.isentropic_vortex(2048)
    spec.order = 6
    out, t, steps = _run(spec, W, 1)
    assert steps == int(g["steps"]) == 1 and abs(t - float(g["t"])) <= 1e-13 * float(g["t"])
    _compare(out, g, spec)


def test_shock_vortex_1024x512_400_steps():
    g = _golden("shockvortex1024x512_400")
    spec, W = wl.shock_vortex(1024, 512)
    out, t, steps = _run(spec, W, 400)
    assert steps == int(g["steps"]) and abs(t - float(g["t"])) <= 1e-12 * float(g["t"])
    _compare(out, g, spec)


def _pulse_ic(p):
    return wl.acoustic_pulse(p["N"], p["A"], p["b"], p["cx"], p["cy"])


def _pulse_sample(params):
    """The grids of the 256-grid batch with stored oracle values: the 8 smallest and 16 across the
    size quantiles (65^2 .. 501^2), tests/golden/make_golden.py pulses / pulses16."""
    smallest = sorted(range(len(params)), key=lambda k: params[k]["N"])[:8]
    order = sorted(range(len(params)), key=lambda k: params[k]["N"])
    ranks = np.linspace(0, len(params) - 1, 16).round().astype(int)
    return sorted(set(smallest) | {order[r] for r in ranks})


def _batched_all():
    """tests/golden/make_golden.py batched256: 128 seeded cells of every grid of the batch that the
    oracle has run (smallest first), one file."""
    path = os.path.join(GOLDEN, "oracle_batched256_100.npz")
    if not os.path.exists(path):
        return {}
    g = np.load(path)
    return {int(k): {"idx": g["idx"][j], "values": g["values"][j], "maxabs": g["maxabs"][j], "t": g["t"][j],
                     "steps": g["steps"][j]} for j, k in enumerate(g["grid"])}


def test_batched_256_grids_100_steps():
    """All 256 grids of the batched workload (seed 1570) in one cgks_batch_step call of 100 steps;
    compared with the oracle: 1500 cells of the smallest eight and of sixteen across the size
    quantiles up to the largest, 128 cells of every grid of the one-file golden; every grid's
    step count and time checked."""
    params = wl.batched_pulses()
    order = _pulse_sample(params)
    goldens = {k: _golden(f"pulse{k:03d}_100") for k in order}
    every = _batched_all()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 4)) as pool:
        ics = pool.map(_pulse_ic, params)
    solvers = []
    for spec, W in ics:
        s = cgks.Solver(cgks.problem_from_spec(spec))
        s.set_state(W)
        solvers.append(s)
    try:
        cgks.cgks_batch_step([s.handle for s in solvers], 100)
        for k in order:
            out, t, steps = solvers[k].get_state()
            assert steps == int(goldens[k]["steps"]) == 100
            assert abs(t - float(goldens[k]["t"])) <= 1e-13 * float(goldens[k]["t"])
            _compare(out, goldens[k], ics[k][0], name=f"batched256 grid {k} ({params[k]['N']}^2, "
                                                      f"A={params[k]['A']:.1e})")
        for k, g in every.items():
            out, t, steps = solvers[k].get_state()
            assert steps == int(g["steps"]) == 100
            assert abs(t - float(g["t"])) <= 1e-13 * float(g["t"])
            _compare(out, g, ics[k][0], name=f"batched256 grid {k} ({params[k]['N']}^2, A={params[k]['A']:.1e}, "
                                             "128 cells)")
        for s in solvers:
            assert s.get_state()[2] == 100
    finally:
        for s in solvers:
            s.close()
