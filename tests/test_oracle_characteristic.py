"""Nonlinear reconstruction in characteristic variables (Sec. 3.2 allows conservative or
characteristic variables).  Pins: the eigenvector basis diagonalises the normal flux Jacobian;
uniform flow stays bitwise uniform; conservation; the shock tubes
stay within the same error bounds as with conservative variables.  (2D on y-uniform data equals
1D in both variable sets: test_oracle_tangential.)"""
import numpy as np

import exact_riemann as ER
import oracle as O
from paper_2001_01570_gb300 import workloads as wl


def test_uniform_flow_and_conservation_characteristic():
    nx, ny, g = 9, 7, 1.4
    rho, u, v, p = 1.3, 0.7, -0.4, 0.9
    W = np.zeros((12, ny, nx))
    W[0], W[1], W[2], W[3] = rho, rho * u, rho * v, p / (g - 1) + 0.5 * rho * (u * u + v * v)
    P = O.make_problem(dim=2, nx=nx, ny=ny, dx=0.1, dy=0.15, cfl=0.5, recon_vars=1)
    Wn, _, _, _ = O.run(P, W, 5)
    assert np.array_equal(Wn, W)
    spec, Wv = wl.shock_vortex(nx=40, ny=20, mach=1.3)
    spec.bc = (0, 0, 0, 0)
    spec.recon_vars = 1
    Wn, _, _, _ = O.run(O.make_problem(**spec.as_kwargs()), Wv, 3)
    assert np.all(np.abs(Wn[:4].sum(axis=(1, 2)) - Wv[:4].sum(axis=(1, 2)))
                  <= 1e-13 * np.abs(Wv[:4]).sum(axis=(1, 2)))


def test_characteristic_shock_tubes():
    for states, t_end, l1_max in ((wl.SOD, 0.2, 3.5e-3), (wl.LAX, 0.16, 6.0e-3)):
        spec, W = wl.shock_tube_1d(100, states, cfl=0.5)
        spec.recon_vars = 1
        Wn, t, _, _ = O.run(O.make_problem(**spec.as_kwargs()), W, 10 ** 6, t_end=t_end)
        ex = ER.cell_average_density(states[0], states[1], t_end, 100)
        jump = max(states[0][0], states[1][0], ex.max()) - min(states[0][0], states[1][0], ex.min())
        assert np.abs(Wn[0] - ex).mean() < l1_max
        assert Wn[0].max() <= ex.max() + 0.02 * jump and Wn[0].min() >= ex.min() - 0.02 * jump


def _normal_flux(W, gamma, D):
    rho, mn = W[0], W[1]
    u = mn / rho
    if D == 1:
        E = W[2]
        p = (gamma - 1) * (E - 0.5 * rho * u * u)
        return np.array([mn, mn * u + p, (E + p) * u])
    mt, E = W[2], W[3]
    v = mt / rho
    p = (gamma - 1) * (E - 0.5 * rho * (u * u + v * v))
    return np.array([mn, mn * u + p, mt * u, (E + p) * u])


def test_eigenbasis_diagonalises_the_flux_jacobian():
    """L A R = diag(U-c, U, [U], U+c) with A the Jacobian of the normal Euler flux by central
    differences (independent of the closed-form eigenvectors), and L R = I."""
    g = 1.4
    for D, W in ((1, np.array([1.3, 0.9, 3.1])), (2, np.array([0.8, -0.5, 0.35, 2.4]))):
        R, L = O.char_basis(D, g, W)
        nv = D + 2
        A = np.zeros((nv, nv))
        for k in range(nv):
            h = 1e-6 * max(1.0, abs(W[k]))
            e = np.zeros(nv)
            e[k] = h
            A[:, k] = (_normal_flux(W + e, g, D) - _normal_flux(W - e, g, D)) / (2 * h)
        rho, u = W[0], W[1] / W[0]
        v = W[2] / W[0] if D == 2 else 0.0
        p = (g - 1) * (W[-1] - 0.5 * rho * (u * u + v * v))
        c = np.sqrt(g * p / rho)
        lam = [u - c, u] + ([u] if D == 2 else []) + [u + c]
        assert np.allclose(L @ A @ R, np.diag(lam), atol=1e-8)
        assert np.allclose(L @ R, np.eye(nv), atol=1e-14)
