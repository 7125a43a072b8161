"""Edge cases of the CUDA path against the oracle: grids smaller than a tile in both directions
(every tile ragged), grids smaller than the reconstruction stencil (periodic wrap over the same
cells several times, reflecting walls on two cells), 1D grids of one to three cells, zero steps,
and stepping on once t_end has been reached."""
import numpy as np
import pytest

from parity_util import check, run_gpu, run_oracle
from paper_2001_01570_gb300 import cgks, workloads as wl

pytestmark = pytest.mark.gpu


def _vortex(nx, ny):
    L = 10.0
    spec = wl.ProblemSpec(dim=2, nx=nx, ny=ny, x0=0.0, x1=L, y0=0.0, y1=L * ny / nx)
    W = wl.cell_state_2d(wl._vortex_fun(0.5 * L, 0.5 * L * ny / nx, L, 5.0, 1.4), nx, ny, 0.0, L, 0.0,
                         L * ny / nx, 1.4)
    return spec, W


@pytest.mark.parametrize("nx,ny", [(8, 8), (9, 7), (13, 5), (3, 5), (1, 6), (6, 1), (2, 2)])
def test_tiny_periodic_grids(nx, ny):
    spec, W = _vortex(nx, ny)
    g, tg, sg = run_gpu(spec, W, 4)
    o, to, so = run_oracle(spec, W, 4)
    assert sg == so == 4 and tg == pytest.approx(to, rel=1e-14)
    check(None, g, o, dx=spec.dx, dy=spec.dy)


@pytest.mark.parametrize("nx,ny", [(9, 7), (4, 2), (2, 3)])
def test_tiny_grids_with_every_boundary_type(nx, ny):
    spec, W = wl.shock_vortex(nx=nx, ny=ny, mach=1.2)
    g, _, sg = run_gpu(spec, W, 3)
    o, _, so = run_oracle(spec, W, 3)
    assert sg == so == 3
    check(None, g, o, dx=spec.dx, dy=spec.dy)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_1d_grids_of_one_to_three_cells(n):
    spec, W = wl.density_wave_1d(n, eps=0.2, cfl=0.3)
    g, tg, sg = run_gpu(spec, W, 5)
    o, to, so = run_oracle(spec, W, 5)
    assert sg == so == 5 and tg == pytest.approx(to, rel=1e-14)
    check(None, g, o, dx=spec.dx)


def test_zero_steps_and_steps_after_t_end():
    spec, W = wl.shock_vortex(nx=30, ny=16, mach=1.3)
    s = cgks.Solver(cgks.problem_from_spec(spec))
    s.set_state(W)
    s.step(0)
    out, t, steps = s.get_state()
    assert steps == 0 and t == 0.0 and np.array_equal(out, W)
    t1 = s.step(1000, t_end=2e-3)
    out1, t, steps1 = s.get_state()
    assert t1 == t == 2e-3 and 0 < steps1 < 1000
    s.step(5, t_end=2e-3)                       # t_end reached: no further step
    out2, t2, steps2 = s.get_state()
    assert steps2 == steps1 and t2 == t and np.array_equal(out2, out1)
    s.close()
