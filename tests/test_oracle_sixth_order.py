"""Pins of the oracle's compact 6th-order variant (named in Sec. 3.2, formulas not printed).

Reading: the linear reconstruction is the degree-5 polynomial fixed by the four cell averages of
the compact stencil and the cell-averaged slopes of the two cells next to the face; the nonlinear
reconstruction keeps the paper's candidates q_0..q_6 (Eq. sub-stencil) with the linear weights
that recombine them into that polynomial's interface value.

- the linear reconstruction reproduces every polynomial of degree <= 5 (value, first and second
  derivative at the interface) and fails for degree 6
- the oracle's weights, applied to the paper's printed candidate values, give the interface value
  of the degree-5 fit solved here symbolically from its definition; they are positive, sum to 1 and
  have the mirror structure of the printed d^8
- on smooth data WENO-Z with these weights approaches the degree-5 value at 8th order (the fit
  itself is 6th order), and across a jump the stencils that cross it lose their weight
- the whole scheme (S2O4 with dt = 0.5 dx^2, the Table 1 protocol of Sec. 4.1) converges at
  order 6 on the density wave, and the 2D scheme on y-independent data reproduces the 1D one
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import sympy as sp

import oracle as O
from conftest import GOLDEN
from paper_2001_01570_gb300 import workloads as wl
from test_oracle_recon import _poly_data


@pytest.mark.parametrize("deg", list(range(0, 6)))
def test_linear_recon6_exact_up_to_degree_5(deg):
    rng = np.random.default_rng(600 + deg)
    for _ in range(3):
        coeffs = [Fraction(int(v), 7) for v in rng.integers(-9, 10, size=deg + 1)]
        if coeffs[-1] == 0:
            coeffs[-1] = Fraction(1)
        h = sp.Rational(int(rng.integers(1, 9)), 10)
        xi0 = sp.Rational(int(rng.integers(-5, 6)), 4)
        Q, hQp, exact = _poly_data(coeffs, h, xi0)
        out = O.linear_recon(Q, hQp, order=6)
        scale = max(1.0, max(abs(v) for v in Q + hQp))
        assert np.allclose(out, exact, rtol=0, atol=1e-12 * scale), (deg, out, exact)


def test_linear_recon6_not_exact_at_degree_6():
    Q, hQp, exact = _poly_data([0] * 6 + [1], sp.Rational(1, 2), sp.Integer(0))
    out = O.linear_recon(Q, hQp, order=6)
    assert abs(out[0] - exact[0]) > 1e-8


def test_linear_recon6_ignores_the_outer_slopes():
    rng = np.random.default_rng(61)
    Q, hQp = rng.normal(size=4), rng.normal(size=4)
    a = O.linear_recon(Q, hQp, order=6)
    hQp2 = hQp.copy()
    hQp2[[0, 3]] = rng.normal(size=2)
    assert np.array_equal(a, O.linear_recon(Q, hQp2, order=6))


def _degree5_value_map():
    """Interface value of the degree-5 fit as exact rational weights of
    (Q_{i-1}, Q_i, Q_{i+1}, Q_{i+2}, hQ'_{i-1}, hQ'_i, hQ'_{i+1}, hQ'_{i+2})."""
    xi = sp.Symbol("xi")
    data = sp.symbols("a b c d A B C D")
    cs = sp.symbols("c0:6")
    q = sum(cs[m] * xi ** m for m in range(6))
    half = sp.Rational(1, 2)
    eqs = [sp.Eq(sp.integrate(q, (xi, k - half, k + half)), data[k + 1]) for k in (-1, 0, 1, 2)]
    eqs += [sp.Eq(q.subs(xi, k + half) - q.subs(xi, k - half), data[4 + k + 1]) for k in (0, 1)]
    val = sp.expand(q.subs(sp.solve(eqs, cs, dict=True)[0]).subs(xi, half))
    return [sp.Rational(val.coeff(v)) for v in data]


def test_weights_recombine_printed_candidates_into_the_degree5_fit():
    with open(os.path.join(GOLDEN, "sub_stencil.json")) as f:
        g = json.load(f)
    d = O.linear_weights(6)
    dq = [Fraction(v).limit_denominator(1000) for v in d]
    assert all(abs(float(a) - b) < 1e-16 for a, b in zip(dq, d))
    assert all(w > 0 for w in dq) and sum(dq) == 1
    # mirror structure of the printed d^8: q0 + q1 mirror q2, q3 ~ q4, q5 ~ q6
    assert dq[0] + dq[1] == dq[2] and dq[3] == dq[4] and dq[5] == dq[6]
    assert dq[0] / dq[1] == Fraction(3, 5)
    combo = [sum(dq[k] * Fraction(g["q"][str(k)]["num"][m], g["q"][str(k)]["den"]) for k in range(7))
             for m in range(8)]
    target = _degree5_value_map()
    assert [sp.Rational(c.numerator, c.denominator) for c in combo] == target
    # and the oracle's own candidate values recombine into its degree-5 fit on random data
    rng = np.random.default_rng(62)
    for _ in range(20):
        s = rng.normal(size=8)
        _, _, diag = O.weno_left(s, diag=True, order=6)
        assert abs(float(np.dot(d, diag["q"])) - O.linear_recon(s[:4], s[4:], order=6)[0]) < 1e-13


def _smooth_stencil(fun, h, x0=0.3):
    gx, gw = np.polynomial.legendre.leggauss(8)
    xs = x0 + h * np.array([-1, 0, 1, 2])
    Q = [0.5 * np.sum(gw * fun(xc + 0.5 * h * gx)) for xc in xs]
    hQ = [fun(xc + 0.5 * h) - fun(xc - 0.5 * h) for xc in xs]
    return np.array(Q + hQ)


def test_weno6_smooth_order():
    """On smooth data the nonlinear value approaches the degree-5 fit faster than the fit
    approaches the function (|v - P5| ~ h^8 against |P5 - f| ~ h^6), so the variant keeps its
    order; with a jump the stencils across it lose their weight as with d^8."""
    dev, err = [], []
    for h in (0.2, 0.1, 0.05):
        s = _smooth_stencil(np.exp, h)
        v, _ = O.weno_left(s, order=6)
        lin = O.linear_recon(s[:4], s[4:], order=6)[0]
        dev.append(abs(v - lin))
        err.append(abs(lin - math.exp(0.3 + 0.5 * h)))
    dev_orders = [math.log2(dev[k] / dev[k + 1]) for k in range(2)]
    err_orders = [math.log2(err[k] / err[k + 1]) for k in range(2)]
    assert min(dev_orders) > 7.0, (dev, dev_orders)
    assert min(err_orders) > 5.8 and max(err_orders) < 6.3, (err, err_orders)
    v, _, diag = O.weno_left(np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0]), diag=True, order=6)
    assert abs(v - 1.0) < 1e-6 and diag["delta"][[2, 4, 6]].max() < 1e-6


def test_scheme_order6_small_dt():
    """Table 1 protocol (dt = 0.5 dx^2, eps_tau = 0) on the density wave to t = 2: the time error
    O(dt^4) = O(dx^8) is below the spatial one, so the variant shows its spatial order."""
    got = {6: [], 8: []}
    for order in (6, 8):
        for N in (10, 20, 40):
            spec, W = wl.density_wave_1d(N, eps=0.2, eps_tau=0.0)
            spec.order = order
            P = O.make_problem(**spec.as_kwargs())
            dx = 2.0 / N
            dt = 0.5 * dx * dx
            nst = int(round(2.0 / dt))
            Wn = O.run_fixed_dt(P, W, nst, dt)
            got[order].append(np.abs(Wn[0] - wl.density_wave_1d_exact(N, nst * dt, eps=0.2)[0]).mean())
    o6 = [math.log2(got[6][k] / got[6][k + 1]) for k in range(2)]
    o8 = [math.log2(got[8][k] / got[8][k + 1]) for k in range(2)]
    assert min(o6) > 5.8 and max(o6) < 6.5, (got[6], o6)
    assert min(o8) > 7.8, (got[8], o8)
    assert all(a > b for a, b in zip(got[6], got[8]))


def test_order6_2d_reproduces_1d_on_y_uniform_data():
    spec, W1 = wl.density_wave_1d(24, eps=0.2)
    spec.order = 6
    P1 = O.make_problem(**spec.as_kwargs())
    kw = spec.as_kwargs()
    kw.update(dim=2, ny=3, dy=0.5)
    P2 = O.make_problem(**kw)
    W2 = np.repeat(wl.state_1d_as_2d(W1), 3, axis=1)
    a, _, _, _ = O.run(P1, W1, 10)
    b, _, _, _ = O.run(P2, W2, 10)
    for r in range(3):
        b1 = np.array([b[0, r], b[1, r], b[3, r], b[4, r], b[5, r], b[7, r]])
        rel = np.abs(a - b1).max(axis=1) / np.abs(a).max(axis=1).clip(1e-300)
        assert rel[:3].max() < 1e-13 and rel[3:].max() < 1e-11
    # and the variant is a different scheme from the 8th-order one
    spec.order = 8
    c, _, _, _ = O.run(O.make_problem(**spec.as_kwargs()), W1, 10)
    assert np.abs(a[0] - c[0]).max() > 1e-10
