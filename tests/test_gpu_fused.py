"""The fused step (cgks_step_fused: both stages of each step in one kernel launch, W* in shared
memory) against the three-kernel step (cgks_step): the same bits on every boundary type, ragged
and tiny grids, both reconstruction orders, characteristic variables, a viscous flow and a clipped
last step; the same error on a state that turns non-physical inside a step; and, through the
three-kernel step's stored oracle values, parity with the oracle on the 512^2 vortex after 200
fused steps."""
import os

import numpy as np
import pytest

from conftest import GOLDEN
from parity_util import check
from paper_2001_01570_gb300 import cgks, workloads as wl

pytestmark = pytest.mark.gpu


def _run(spec, W, nsteps, fused, t_end=0.0):
    s = cgks.Solver(cgks.problem_from_spec(spec))
    s.set_state(W)
    s.step(nsteps, t_end=t_end, fused=fused)
    out, t, steps = s.get_state()
    s.close()
    return out, t, steps


def _vortex(nx, ny):
    L = 10.0
    spec = wl.ProblemSpec(dim=2, nx=nx, ny=ny, x0=0.0, x1=L, y0=0.0, y1=L * ny / nx)
    W = wl.cell_state_2d(wl._vortex_fun(0.5 * L, 0.5 * L * ny / nx, L, 5.0, 1.4), nx, ny, 0.0, L, 0.0,
                         L * ny / nx, 1.4)
    return spec, W


CASES = {
    "vortex 256^2": (lambda: wl.isentropic_vortex(256), 12, {}),
    "vortex 131x77 (ragged tiles)": (lambda: _vortex(131, 77), 10, {}),
    "vortex 5x3 (smaller than a tile and a stencil)": (lambda: _vortex(5, 3), 6, {}),
    "vortex 16x8 (one tile, the region wraps onto itself)": (lambda: _vortex(16, 8), 6, {}),
    "shock-vortex 200x100 (inflow, outflow, walls)": (lambda: wl.shock_vortex(200, 100), 20, {}),
    "shock-vortex 37x19 Mach 1.5": (lambda: wl.shock_vortex(37, 19, mach=1.5), 12, {}),
    "shock reflection 120x30 Mach 2.9": (lambda: wl.shock_reflection(120, 30), 15, {}),
    "pulse 97^2 A=1e-5": (lambda: wl.acoustic_pulse(97, 1e-5, 4.0, 30.0, 61.0), 10, {}),
    "vortex 96^2 sixth-order variant": (lambda: wl.isentropic_vortex(96), 8, {"order": 6}),
    "shock-vortex 64x32 characteristic variables": (lambda: wl.shock_vortex(64, 32), 8, {"recon_vars": 1}),
    "shear wave 48^2 viscous": (lambda: wl.shear_wave(48), 8, {}),
}


@pytest.mark.parametrize("name", list(CASES))
def test_fused_step_gives_the_same_bits(name):
    make, nsteps, extra = CASES[name]
    spec, W = make()
    for k, v in extra.items():
        setattr(spec, k, v)
    a, ta, sa = _run(spec, W, nsteps, fused=False)
    b, tb, sb = _run(spec, W, nsteps, fused=True)
    assert sa == sb == nsteps and ta == tb
    assert np.array_equal(a, b), f"{name}: max difference {np.abs(a - b).max():.3e}"


def test_fused_step_clips_the_last_step_like_the_three_kernel_step():
    spec, W = wl.shock_vortex(48, 24, mach=1.3)
    a, ta, sa = _run(spec, W, 1000, fused=False, t_end=3e-3)
    b, tb, sb = _run(spec, W, 1000, fused=True, t_end=3e-3)
    assert ta == tb == 3e-3 and sa == sb and 0 < sa < 1000
    assert np.array_equal(a, b)


def test_fused_step_reports_a_state_that_turns_nonphysical():
    """A huge density gradient in one cell: the cell averages are valid (the state is accepted),
    but the reconstructed face states are not; both arrangements stop with CGKS_E_NONPHYSICAL and
    keep the state that was set."""
    spec, W = wl.acoustic_pulse(40, 1e-3, 4.0, 20.0, 20.0)
    W = W.copy()
    W[4, 17, 23] = 1e7
    for fused in (False, True):
        s = cgks.Solver(cgks.problem_from_spec(spec))
        s.set_state(W)
        with pytest.raises(cgks.CgksError) as ei:
            s.step(3, fused=fused)
        assert ei.value.status == cgks.CGKS_E_NONPHYSICAL
        buf = np.empty(s.shape)
        with pytest.raises(cgks.CgksError):
            cgks.cgks_get_state(s.handle, buf)
        assert np.array_equal(buf, W)
        s.close()


def test_fused_step_rejects_1d():
    spec, W = wl.density_wave_1d(32)
    s = cgks.Solver(cgks.problem_from_spec(spec))
    s.set_state(W)
    with pytest.raises(cgks.CgksError) as ei:
        s.step(1, fused=True)
    assert ei.value.status == cgks.CGKS_E_INVAL
    s.close()


def test_fused_vortex_512_200_steps_against_the_oracle():
    path = os.path.join(GOLDEN, "oracle_vortex512_200.npz")
    if not os.path.exists(path):
        pytest.skip("golden file not generated")
    g = np.load(path)
    spec, W = wl.isentropic_vortex(512)
    out, t, steps = _run(spec, W, 200, fused=True)
    assert steps == int(g["steps"]) and abs(t - float(g["t"])) <= 1e-13 * float(g["t"])
    planes = out.reshape(out.shape[0], -1)[:, g["idx"]]
    check("fused vortex512 200 steps", planes, g["values"], dx=spec.dx, dy=spec.dy, gamma=spec.gamma, tol=1e-11,
          grad_tol=1e-9, maxabs=g["maxabs"])
