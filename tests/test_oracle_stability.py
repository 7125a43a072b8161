"""Linear stability of the 2D reading of the tangential reconstruction.

The paper leaves the 2D procedure to a missing figure.  A reading that takes the tangential slope
at a face from the cell-averaged tangential gradients is linearly unstable under advection (the
one-step amplification on a uniform diagonal stream at CFL 0.5 is about 1.15); the reading used
here (tangential profiles fitted to the face line averages of the neighbouring rows) is not.
Pinned here: the spectral radius of the one-step Jacobian of the oracle on small periodic grids,
and a long run of an under-resolved vortex that used to blow up.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2001_01570_gb300 import workloads as wl


def _spectral_radius(n, U, V, cfl, eps_tau=0.01, h=1e-6):
    g, rho, p = 1.4, 1.0, 1.0
    W = np.zeros((12, n, n))
    W[0], W[1], W[2] = rho, rho * U, rho * V
    W[3] = p / (g - 1) + 0.5 * rho * (U * U + V * V)
    dt = cfl / (max(abs(U), abs(V)) + math.sqrt(g * p / rho))
    P = O.make_problem(dim=2, nx=n, ny=n, dx=1.0, dy=1.0, cfl=cfl, eps_tau=eps_tau)
    O.set_threads(1)          # 64-cell grids: threads only add overhead
    N = W.size
    J = np.zeros((N, N))
    for k in range(N):
        e = np.zeros(N)
        e[k] = h
        Wp = O.run_fixed_dt(P, W + e.reshape(W.shape), 1, dt)
        Wm = O.run_fixed_dt(P, W - e.reshape(W.shape), 1, dt)
        J[:, k] = (Wp - Wm).ravel() / (2 * h)
    O.set_threads(os.cpu_count() or 1)
    return np.abs(np.linalg.eigvals(J)).max()


@pytest.mark.parametrize("U,V,bound", [(0.0, 0.0, 1.0 + 1e-6), (1.0, 0.0, 1.006), (1.0, 1.0, 1.01)])
def test_one_step_spectral_radius(U, V, bound):
    assert _spectral_radius(8, U, V, 0.5) <= bound


def test_underresolved_vortex_long_run_stays_bounded():
    spec, W = wl.isentropic_vortex(32)
    P = O.make_problem(**spec.as_kwargs())
    Wn, t, steps, _ = O.run(P, W, 600)
    _, ex = wl.isentropic_vortex(32, t=t)
    assert steps == 600 and np.abs(Wn[0] - ex[0]).max() < 0.05
