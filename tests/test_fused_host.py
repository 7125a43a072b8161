"""The fused step's tile layout, run on the host (paper_2001_01570_gb300/opcount.py host_step: the
kernels' own device arithmetic compiled for the CPU, cgks_fused.cuh's six phases run by one caller
thread): one step gives the same bits as the three-kernel arrangement of the same arithmetic on
every boundary type, ragged and tiny grids, both orders, characteristic variables and a viscous
flow.  The GPU test (test_gpu_fused.py) checks the kernel itself."""
import numpy as np
import pytest

from paper_2001_01570_gb300 import opcount, workloads as wl


def _vortex(nx, ny):
    L = 10.0
    spec = wl.ProblemSpec(dim=2, nx=nx, ny=ny, x0=0.0, x1=L, y0=0.0, y1=L * ny / nx)
    W = wl.cell_state_2d(wl._vortex_fun(0.5 * L, 0.5 * L * ny / nx, L, 5.0, 1.4), nx, ny, 0.0, L, 0.0,
                         L * ny / nx, 1.4)
    return spec, W


CASES = {
    "vortex 40^2": (lambda: wl.isentropic_vortex(40), {}),
    "vortex 37x23": (lambda: _vortex(37, 23), {}),
    "vortex 5x3": (lambda: _vortex(5, 3), {}),
    "vortex 16x8": (lambda: _vortex(16, 8), {}),
    "shock-vortex 61x29": (lambda: wl.shock_vortex(61, 29), {}),
    "shock-vortex 9x7 Mach 1.2": (lambda: wl.shock_vortex(9, 7, mach=1.2), {}),
    "shock reflection 50x13": (lambda: wl.shock_reflection(50, 13), {}),
    "pulse 23^2": (lambda: wl.acoustic_pulse(23, 1e-3, 3.0, 7.0, 15.0), {}),
    "vortex 40^2 sixth-order variant": (lambda: wl.isentropic_vortex(40), {"order": 6}),
    "shock-vortex 40x20 characteristic, sixth order": (lambda: wl.shock_vortex(40, 20),
                                                         {"recon_vars": 1, "order": 6}),
    "shear wave 24^2 viscous": (lambda: wl.shear_wave(24), {}),
}


@pytest.mark.parametrize("name", list(CASES))
def test_fused_tile_layout_gives_the_same_bits_on_the_host(name):
    make, extra = CASES[name]
    spec, W = make()
    for k, v in extra.items():
        setattr(spec, k, v)
    a, b = W, W
    for _ in range(2):
        a = opcount.host_step(spec, a, fused=False)
        b = opcount.host_step(spec, b, fused=True)
    assert not np.array_equal(a, W)
    assert np.array_equal(a, b), f"{name}: max difference {np.abs(a - b).max():.3e}"


def test_host_step_rejects_1d():
    spec, W = wl.density_wave_1d(16)
    with pytest.raises(RuntimeError):
        opcount.host_step(spec, W, fused=True)
