"""Batched stepping (one persistent launch per stage over the tiles of many grids, replayed as a
CUDA graph) gives bit-identical results to stepping each grid alone, and error handling keeps the
last valid state."""
import numpy as np
import pytest

from paper_2001_01570_gb300 import cgks, workloads as wl

pytestmark = pytest.mark.gpu


def test_batched_equals_alone_bitwise():
    cases = [wl.acoustic_pulse(37, 1e-3, 4.0, 10.0, 20.0), wl.isentropic_vortex(24),
             wl.shock_vortex(nx=50, ny=26, mach=1.2), wl.acoustic_pulse(64, 1e-5, 8.0, 3.0, 60.0)]
    alone = []
    for spec, W in cases:
        s = cgks.Solver(cgks.problem_from_spec(spec))
        s.set_state(W)
        s.step(4)
        alone.append(s.get_state())
        s.close()
    solvers = []
    for spec, W in cases:
        s = cgks.Solver(cgks.problem_from_spec(spec))
        s.set_state(W)
        solvers.append(s)
    cgks.cgks_batch_step([s.handle for s in solvers], 4)
    assert cgks.cgks_last_launch_count() >= 16
    for s, (ref, t, steps) in zip(solvers, alone):
        out, tb, sb = s.get_state()
        assert sb == steps == 4 and tb == t
        assert np.array_equal(out, ref)
        s.close()


def test_nonphysical_state_is_reported_and_last_state_kept():
    spec, W = wl.acoustic_pulse(32, 1e-3, 4.0, 16.0, 16.0)
    s = cgks.Solver(cgks.problem_from_spec(spec))
    s.set_state(W)
    s.step(2)
    good, t_good, steps_good = s.get_state()
    # a cell with negative pressure: the kernels flag it, no step is taken
    bad = good.copy()
    bad[3, 5, 7] = 0.1 * bad[3, 5, 7] - 10.0
    s.set_state(bad)
    with pytest.raises(cgks.CgksError) as ei:
        s.step(3)
    assert ei.value.status == cgks.CGKS_E_NONPHYSICAL
    buf = np.empty(s.shape)
    with pytest.raises(cgks.CgksError):
        cgks.cgks_get_state(s.handle, buf)
    assert np.array_equal(buf, bad)       # the last valid state is the one that was set
    # the solver is usable again after a new state
    s.set_state(good, t_good)
    s.step(1)
    s.close()


@pytest.mark.parametrize("shape", [s for s in cgks.TILE_SHAPES if s != "64x1"])
def test_tile_shape_does_not_change_results(shape):
    """Every 2D tile shape (two CTAs per SM where they fit, one otherwise) gives the default
    shape's results bit for bit."""
    spec, W = wl.shock_vortex(nx=61, ny=37, mach=1.25)
    ref = cgks.Solver(cgks.problem_from_spec(spec))
    ref.set_state(W)
    ref.step(3)
    a, _, _ = ref.get_state()
    ref.close()
    s = cgks.Solver(cgks.problem_from_spec(spec))
    cgks.cgks_set_tile_shape(s.handle, shape)
    s.set_state(W)
    s.step(3)
    b, _, _ = s.get_state()
    s.close()
    assert np.array_equal(a, b)


def test_batched_1d_acoustic_grids_equal_alone_bitwise():
    params = wl.batched_acoustic_1d(count=40)
    cases = [wl.acoustic_wave_1d(p["N"], eps_tau=0.0) for p in params]
    alone = []
    for spec, W in cases:
        s = cgks.Solver(cgks.problem_from_spec(spec))
        s.set_state(W)
        s.step(25)
        alone.append(s.get_state())
        s.close()
    solvers = []
    for spec, W in cases:
        s = cgks.Solver(cgks.problem_from_spec(spec))
        s.set_state(W)
        solvers.append(s)
    cgks.cgks_batch_step([s.handle for s in solvers], 25)
    for s, (ref, t, steps) in zip(solvers, alone):
        out, tb, sb = s.get_state()
        assert sb == steps == 25 and tb == t
        assert np.array_equal(out, ref)
        s.close()


def test_batched_mixed_options_equal_alone_bitwise():
    """One batch mixing conservative and characteristic reconstruction (two record-kernel queues),
    the 8th-order scheme and its 6th-order variant, a viscous grid and the shock reflection's
    per-side inflow states."""
    a = wl.shock_vortex(nx=40, ny=22, mach=1.3)
    b = wl.shock_vortex(nx=33, ny=17, mach=1.2)
    b[0].recon_vars = 1
    c = wl.shear_wave(32, 1e-3, 0.01, kind="shear")
    d = wl.shock_reflection(40, 10)
    d[0].recon_vars = 1
    e = wl.shock_vortex(nx=36, ny=20, mach=1.25)
    e[0].order = 6
    f = wl.shock_reflection(36, 9)
    f[0].recon_vars, f[0].order = 1, 6
    cases = [a, b, c, d, e, f]
    alone = []
    for spec, W in cases:
        s = cgks.Solver(cgks.problem_from_spec(spec))
        s.set_state(W)
        s.step(5)
        alone.append(s.get_state())
        s.close()
    solvers = []
    for spec, W in cases:
        s = cgks.Solver(cgks.problem_from_spec(spec))
        s.set_state(W)
        solvers.append(s)
    cgks.cgks_batch_step([s.handle for s in solvers], 5)
    for s, (ref, t, steps) in zip(solvers, alone):
        out, tb, sb = s.get_state()
        assert sb == steps == 5 and tb == t
        assert np.array_equal(out, ref)
        s.close()


def test_autotuner_picks_a_shape_and_cells_per_thread_without_changing_results():
    """The batched autotuner times four tile shapes and then the update kernel at 2 and 4 cells per
    thread (12 steps); its choice is reported, and the results equal the solves alone whichever
    candidate ran which step."""
    cases = [wl.acoustic_pulse(70, 1e-3, 5.0, 20.0, 40.0), wl.isentropic_vortex(45),
             wl.shock_vortex(nx=52, ny=26, mach=1.45)]
    nsteps = 15
    alone = []
    for spec, W in cases:
        s = cgks.Solver(cgks.problem_from_spec(spec))
        s.set_state(W)
        s.step(nsteps)
        alone.append(s.get_state())
        s.close()
    solvers = []
    for spec, W in cases:
        s = cgks.Solver(cgks.problem_from_spec(spec))
        s.set_state(W)
        solvers.append(s)
    handles = [s.handle for s in solvers]
    cgks.cgks_batch_step(handles, 5)
    assert cgks.cgks_batch_tile_shape(handles) == -1           # still timing candidates
    cgks.cgks_batch_step(handles, nsteps - 5)
    assert cgks.TILE_SHAPES[cgks.cgks_batch_tile_shape(handles)] in ("8x16", "14x8", "16x8", "16x16")
    assert cgks.cgks_batch_update_cpt(handles) in (1, 2, 4)
    for s, (ref, t, steps) in zip(solvers, alone):
        out, tb, sb = s.get_state()
        assert sb == steps == nsteps and tb == t
        assert np.array_equal(out, ref)
        s.close()
