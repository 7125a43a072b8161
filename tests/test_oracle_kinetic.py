"""Pins of the oracle's gas-kinetic part (Sec. 2.1-2.2) against quadrature, symbolic algebra and
limits the mathematics fixes.

- Maxwellian moments: whole-line moments against Gauss-Hermite quadrature of the Maxwellian with
  K literal internal Gaussian coordinates; half-line moments against adaptive quadrature
- the psi-weighted moment assembly <u^a v^b psi (c . psi)> against the same quadrature
- Euler time derivatives (Cauchy-Kowalevski jets) against sympy differentiation of the Euler
  equations on random quadratic fields
- the interface evaluation in its limits: tau = 0 gives the Euler flux F(W0) and its exact time
  derivative; identical left/right/equilibrium states make the half-line sums equal the whole-line
  moments and the non-equilibrium interface part vanish (the kinetic W_t equals the Euler W_t)
"""
import itertools
import math

import numpy as np
import pytest
import sympy as sp
from scipy import integrate

import oracle as O

GAMMA = 1.4


def _maxwellian_expect(D, U, V, lam, K, func, npts=8):
    """E[func(u, v, xi2)] under the normalised Maxwellian, by tensor Gauss-Hermite quadrature over
    u, v and K internal Gaussian coordinates (K must be an integer here)."""
    z, w = np.polynomial.hermite.hermgauss(npts)
    w = w / math.sqrt(math.pi)
    s = 1.0 / math.sqrt(lam)
    ndim = D + int(K)
    total = 0.0
    for idx in itertools.product(range(npts), repeat=ndim):
        wt = np.prod([w[i] for i in idx])
        u = U + s * z[idx[0]]
        v = V + s * z[idx[1]] if D == 2 else 0.0
        xi2 = sum((s * z[i]) ** 2 for i in idx[D:])
        total += wt * func(u, v, xi2)
    return total


def _psi(D, u, v, xi2):
    if D == 2:
        return np.array([1.0, u, v, 0.5 * (u * u + v * v + xi2)])
    return np.array([1.0, u, 0.5 * (u * u + xi2)])


def test_whole_line_moments_gauss_hermite():
    z, w = np.polynomial.hermite.hermgauss(20)
    for U, lam in ((0.3, 0.7), (-1.7, 2.5), (2.2, 0.35)):
        mu = O.moments_u(U, lam, 0)
        for n in range(9):
            ref = np.sum(w * (U + z / math.sqrt(lam)) ** n) / math.sqrt(math.pi)
            assert abs(mu[n] - ref) <= 1e-12 * max(1.0, abs(ref))


@pytest.mark.parametrize("half", [1, -1])
def test_half_line_moments_quadrature(half):
    for U, lam in ((0.3, 0.7), (-1.7, 2.5), (2.2, 0.35), (0.0, 1.0)):
        mu = O.moments_u(U, lam, half)
        for n in range(9):
            f = lambda u: u ** n * math.sqrt(lam / math.pi) * math.exp(-lam * (u - U) ** 2)
            lo, hi = (0.0, np.inf) if half > 0 else (-np.inf, 0.0)
            ref, _ = integrate.quad(f, lo, hi, epsabs=1e-14, epsrel=1e-13, limit=200)
            assert abs(mu[n] - ref) <= 1e-10 * max(1.0, abs(ref)), (n, mu[n], ref)
        full = O.moments_u(U, lam, 0)
        other = O.moments_u(U, lam, -half)
        assert np.allclose(mu + other, full, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("D", [1, 2])
def test_psi_moment_assembly(D):
    K = (3 - GAMMA) / (GAMMA - 1) if D == 1 else (4 - 2 * GAMMA) / (GAMMA - 1)
    assert abs(K - round(K)) < 1e-12
    K = float(round(K))
    rng = np.random.default_rng(3 + D)
    U, V, lam = 0.4, (-0.6 if D == 2 else 0.0), 1.3
    cases = [(0, 0), (1, 0), (2, 0)] + ([(0, 1), (1, 1)] if D == 2 else [])
    for a0, b0 in cases:
        cf = rng.normal(size=D + 2)
        got = O.mom_psi_poly(D, U, V, lam, K, 0, a0, b0, cf)
        ref = _maxwellian_expect(D, U, V, lam, K,
                                 lambda u, v, x2: u ** a0 * v ** b0 * _psi(D, u, v, x2) * np.dot(cf, _psi(D, u, v, x2)),
                                 npts=6)
        assert np.allclose(got, ref, rtol=1e-11, atol=1e-11), (a0, b0, got, ref)
        got0 = O.mom_psi_poly(D, U, V, lam, K, 0, a0, b0, None)
        ref0 = _maxwellian_expect(D, U, V, lam, K, lambda u, v, x2: u ** a0 * v ** b0 * _psi(D, u, v, x2), npts=6)
        assert np.allclose(got0, ref0, rtol=1e-11, atol=1e-11)


def _euler_symbolic(D):
    x, y = sp.symbols("x y")
    syms = sp.symbols("r m n E")[: D + 1] if D == 1 else sp.symbols("r m n E")
    if D == 1:
        r, m, E = sp.symbols("r m E")
        U = m / r
        p = (GAMMA - 1) * (E - m * U / 2)
        F = [m, m * U + p, U * (E + p)]
        return (r, m, E), F, None
    r, m, n, E = syms
    U, V = m / r, n / r
    p = (GAMMA - 1) * (E - (m * U + n * V) / 2)
    F = [m, m * U + p, m * V, U * (E + p)]
    G = [n, n * U, n * V + p, V * (E + p)]
    return (r, m, n, E), F, G


@pytest.mark.parametrize("D", [1, 2])
def test_euler_time_derivatives_match_symbolic(D):
    x, y = sp.symbols("x y")
    Wsym, F, G = _euler_symbolic(D)
    nv = D + 2
    rng = np.random.default_rng(20 + D)
    for trial in range(3):
        base = {1: [1.1, 0.4, 2.6], 2: [1.1, 0.4, -0.3, 2.6]}[D]
        W0 = np.array(base) + 0.05 * rng.normal(size=nv)
        Wx, Wy, Wxx, Wxy, Wyy = (0.3 * rng.normal(size=nv) for _ in range(5))
        if D == 1:
            Wy[:] = Wxy[:] = Wyy[:] = 0.0
        fields = [sp.Float(W0[k]) + sp.Float(Wx[k]) * x + sp.Float(Wy[k]) * y
                  + sp.Float(Wxx[k]) * x ** 2 / 2 + sp.Float(Wxy[k]) * x * y + sp.Float(Wyy[k]) * y ** 2 / 2
                  for k in range(nv)]
        sub = dict(zip(Wsym, fields))
        Fx = [f.subs(sub) for f in F]
        Wt = [-sp.diff(Fx[k], x) - (sp.diff(G[k].subs(sub), y) if D == 2 else 0) for k in range(nv)]
        JF = sp.Matrix(F).jacobian(sp.Matrix(Wsym))
        Ft = (JF.subs(sub) * sp.Matrix(Wt))
        if D == 2:
            JG = sp.Matrix(G).jacobian(sp.Matrix(Wsym))
            Gt = (JG.subs(sub) * sp.Matrix(Wt))
        Wtt = [-sp.diff(Ft[k], x) - (sp.diff(Gt[k], y) if D == 2 else 0) for k in range(nv)]
        at0 = {x: 0, y: 0}
        ref_t = np.array([float(e.subs(at0)) for e in Wt])
        ref_tt = np.array([float(e.subs(at0)) for e in Wtt])
        got_t, got_tt = O.euler_time_derivs(D, GAMMA, W0, Wx, Wy, Wxx, Wxy, Wyy)
        assert np.allclose(got_t, ref_t, rtol=1e-12, atol=1e-12)
        assert np.allclose(got_tt, ref_tt, rtol=1e-11, atol=1e-11)


def _euler_flux(D, W):
    if D == 1:
        r, m, E = W
        U = m / r
        p = (GAMMA - 1) * (E - 0.5 * m * U)
        return np.array([m, m * U + p, U * (E + p)])
    r, m, n, E = W
    U, V = m / r, n / r
    p = (GAMMA - 1) * (E - 0.5 * (m * U + n * V))
    return np.array([m, m * U + p, m * V, U * (E + p)])


@pytest.mark.parametrize("D", [1, 2])
def test_gks_point_euler_limit(D):
    """tau = 0 (eps_tau = 0, equal pressures): flux average is F(W0) and its slope is dF/dW . W_t."""
    nv = D + 2
    P = O.make_problem(dim=D, nx=4, ny=4, dx=1, dy=1, eps_tau=0.0)
    rng = np.random.default_rng(30 + D)
    W0 = np.array([1.2, 0.5, 2.9]) if D == 1 else np.array([1.2, 0.5, -0.2, 2.9])
    Wn, Wt_sp = 0.2 * rng.normal(size=nv), (0.2 * rng.normal(size=nv) if D == 2 else np.zeros(nv))
    dt = 0.01
    fields = dict(W0=W0, W0n=Wn, W0t=Wt_sp, Wl=W0, Wr=W0, Wln=Wn, Wrn=Wn, Wlt=Wt_sp, Wrt=Wt_sp)
    out = O.gks_point(P, D, dt, **fields)
    assert out["tau"] == 0.0
    Fb = (4 * out["S2"] - out["S1"]) / dt
    Ft = 4 * (out["S1"] - 2 * out["S2"]) / dt ** 2
    assert np.allclose(Fb, _euler_flux(D, W0), rtol=1e-13, atol=1e-13)
    # dF/dW . W_t by central differences of the closed-form flux (W_t from the Euler equations)
    h = 1e-6
    ref = (_euler_flux(D, W0 + h * out["Wt"]) - _euler_flux(D, W0 - h * out["Wt"])) / (2 * h)
    assert np.allclose(Ft, ref, rtol=1e-7, atol=1e-8)
    # and W_t itself is -dF/dx - dG/dy
    Fx = (_euler_flux(D, W0 + h * Wn) - _euler_flux(D, W0 - h * Wn)) / (2 * h)
    Gy = np.zeros(nv)
    if D == 2:
        def G(W):
            r, m, n, E = W
            U, V = m / r, n / r
            p = (GAMMA - 1) * (E - 0.5 * (m * U + n * V))
            return np.array([n, n * U, n * V + p, V * (E + p)])
        Gy = (G(W0 + h * Wt_sp) - G(W0 - h * Wt_sp)) / (2 * h)
    assert np.allclose(out["Wt"], -Fx - Gy, rtol=1e-7, atol=1e-8)


@pytest.mark.parametrize("D", [1, 2])
def test_gks_point_equal_states(D):
    """Left, right and equilibrium states identical, tau > 0: the half-line sums reproduce the
    whole-line moments, so S(Delta) = Delta F0 + Delta^2/2 F_t - tau Delta (T2 + T1), and the
    non-equilibrium part of the interface state is zero (kinetic W_t = Euler W_t)."""
    nv = D + 2
    P = O.make_problem(dim=D, nx=4, ny=4, dx=1, dy=1, eps_tau=0.3)
    rng = np.random.default_rng(40 + D)
    W0 = np.array([0.9, -0.3, 2.1]) if D == 1 else np.array([0.9, -0.3, 0.4, 2.1])
    Wn, Wt_sp = 0.3 * rng.normal(size=nv), (0.3 * rng.normal(size=nv) if D == 2 else np.zeros(nv))
    dt = 0.02
    out = O.gks_point(P, D, dt, W0=W0, W0n=Wn, W0t=Wt_sp, Wl=W0, Wr=W0, Wln=Wn, Wrn=Wn, Wlt=Wt_sp, Wrt=Wt_sp)
    tau = out["tau"]
    assert abs(tau - 0.3 * dt) < 1e-18
    ref0 = O.make_problem(dim=D, nx=4, ny=4, dx=1, dy=1, eps_tau=0.0)
    o0 = O.gks_point(ref0, D, dt, W0=W0, W0n=Wn, W0t=Wt_sp, Wl=W0, Wr=W0, Wln=Wn, Wrn=Wn, Wlt=Wt_sp, Wrt=Wt_sp)
    # tau enters only through -tau Delta (T2 + T1): S(dt) - S0(dt) = 2 (S(dt/2) - S0(dt/2))
    d1 = out["S1"] - o0["S1"]
    d2 = out["S2"] - o0["S2"]
    assert np.allclose(d1, 2 * d2, rtol=1e-9, atol=1e-13)
    assert np.abs(out["NEh"]).max() < 1e-13 and np.abs(out["NEf"]).max() < 1e-13


def test_gks_point_mirror_symmetry():
    """Reflecting x -> -x maps the interface problem onto itself with left and right exchanged:
    mass and energy fluxes change sign, the normal momentum flux does not."""
    D = 2
    P = O.make_problem(dim=D, nx=4, ny=4, dx=1, dy=1, eps_tau=0.01)
    rng = np.random.default_rng(50)
    Wl = np.array([1.0, 0.3, 0.1, 2.5]); Wr = np.array([0.8, 0.1, -0.2, 2.0]); W0 = 0.5 * (Wl + Wr)
    g = {k: 0.2 * rng.normal(size=4) for k in ("W0n", "W0t", "W0nn", "W0nt", "W0tt", "Wln", "Wlt", "Wrn", "Wrt")}
    dt = 0.01
    a = O.gks_point(P, D, dt, W0=W0, Wl=Wl, Wr=Wr, **g)
    S = np.array([1.0, -1.0, 1.0, 1.0])       # x-mirror acts on (rho, rhoU, rhoV, rhoE) by sign of rhoU
    m = lambda v: S * v
    b = O.gks_point(P, D, dt, W0=m(W0), Wl=m(Wr), Wr=m(Wl),
                    W0n=-m(g["W0n"]), W0t=m(g["W0t"]), W0nn=m(g["W0nn"]), W0nt=-m(g["W0nt"]), W0tt=m(g["W0tt"]),
                    Wln=-m(g["Wrn"]), Wlt=m(g["Wrt"]), Wrn=-m(g["Wln"]), Wrt=m(g["Wlt"]))
    flux_sign = np.array([-1.0, 1.0, -1.0, -1.0])
    assert np.allclose(b["S1"], flux_sign * a["S1"], rtol=1e-12, atol=1e-14)
    assert np.allclose(b["S2"], flux_sign * a["S2"], rtol=1e-12, atol=1e-14)
    assert np.allclose(b["NEf"], m(a["NEf"]), rtol=1e-12, atol=1e-14)


def test_collision_time_pressure_jump_limits():
    """Sec. 4's collision time at an interface: equal left/right pressures leave only eps*dt (the
    smooth-flow value); the enhancement is symmetric in the two sides, grows with |p_l - p_r| and
    tends to (eps + C) dt as one pressure dominates; with mu > 0 the first part is mu/p of the
    equilibrium state, whatever the jump."""
    D, dt, eps, C = 1, 0.01, 0.01, 1.0
    P = O.make_problem(dim=D, nx=4, ny=1, dx=1, dy=1, eps_tau=eps, c_tau=C)

    def tau_of(pl, pr, problem=P, p0=None):
        Wl = np.array([1.0, 0.0, pl / (GAMMA - 1.0)])
        Wr = np.array([1.0, 0.0, pr / (GAMMA - 1.0)])
        W0 = 0.5 * (Wl + Wr) if p0 is None else np.array([1.0, 0.0, p0 / (GAMMA - 1.0)])
        return O.gks_point(problem, D, dt, W0=W0, Wl=Wl, Wr=Wr)["tau"]

    assert tau_of(0.7, 0.7) == eps * dt
    jumps = [tau_of(1.0, pr) for pr in (1.0, 0.9, 0.5, 0.1, 1e-3, 1e-9)]
    assert all(b > a for a, b in zip(jumps, jumps[1:])), jumps
    assert tau_of(1.0, 0.3) == tau_of(0.3, 1.0)
    # p_r / p_l = 1e-9: the limit (eps + C) dt is approached as 2 C (p_r / p_l) dt
    assert 0.0 < (eps + C) * dt - jumps[-1] < 2.5e-9 * C * dt
    # without the jump term (C = 0) the pressure ratio is irrelevant
    P0 = O.make_problem(dim=D, nx=4, ny=1, dx=1, dy=1, eps_tau=eps, c_tau=0.0)
    assert tau_of(1.0, 1e-3, P0) == eps * dt
    # viscous: mu / p of the equilibrium state, the jump term added on top
    mu = 2e-3
    Pv = O.make_problem(dim=D, nx=4, ny=1, dx=1, dy=1, eps_tau=eps, c_tau=0.0, mu=mu)
    assert abs(tau_of(1.0, 1.0, Pv, p0=0.8) - mu / 0.8) < 1e-15
    Pvc = O.make_problem(dim=D, nx=4, ny=1, dx=1, dy=1, eps_tau=eps, c_tau=C, mu=mu)
    assert tau_of(1.0, 0.5, Pvc, p0=0.8) > tau_of(1.0, 0.5, Pv, p0=0.8)
