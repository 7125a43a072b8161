"""Pins of the oracle's reconstruction (Sec. 3.2 and 3.3) against the paper and the mathematics.

- the linear compact reconstruction reproduces every polynomial of degree <= 7 (value, first and
  second derivative at the interface) and fails for degree 8: this is what "8th order" means
- each candidate polynomial, built by the oracle from its sub-stencil definition, has the point
  value printed in Eq. (sub-stencil); with the printed linear weights d_k the candidates recombine
  into the printed P7 value exactly
- smoothness indicators agree with an exact symbolic integration of the definition
- WENO-Z behaviour: linear weights recovered on smooth data, Z_ref = O(h^3) relative to beta,
  the stencils that cross a jump lose their weight, mirror symmetry of left/right states
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest
import sympy as sp

import oracle as O
from conftest import GOLDEN


def _poly_data(coeffs, h, xi0):
    """Exact (rational) stencil data of f(x) = sum c_n x^n on cells centred at xi0 + k*h,
    k = -1..2, with the interface at xi0 + h/2.  Returns floats (Q, hQ') and exact interface
    value, h f', h^2 f''."""
    x = sp.Symbol("x")
    f = sum(sp.Rational(c) * x ** n for n, c in enumerate(coeffs))
    F = sp.integrate(f, x)
    Q, hQp = [], []
    for k in (-1, 0, 1, 2):
        a = xi0 + (k - sp.Rational(1, 2)) * h
        b = xi0 + (k + sp.Rational(1, 2)) * h
        Q.append((F.subs(x, b) - F.subs(x, a)) / h)
        hQp.append(f.subs(x, b) - f.subs(x, a))
    xf = xi0 + h / 2
    exact = (f.subs(x, xf), h * sp.diff(f, x).subs(x, xf), h ** 2 * sp.diff(f, x, 2).subs(x, xf))
    return [float(v) for v in Q], [float(v) for v in hQp], [float(v) for v in exact]


@pytest.mark.parametrize("deg", list(range(0, 8)))
def test_linear_recon_exact_up_to_degree_7(deg):
    rng = np.random.default_rng(100 + deg)
    for _ in range(3):
        coeffs = [Fraction(int(v), 7) for v in rng.integers(-9, 10, size=deg + 1)]
        if coeffs[-1] == 0:
            coeffs[-1] = Fraction(1)
        h = sp.Rational(int(rng.integers(1, 9)), 10)
        xi0 = sp.Rational(int(rng.integers(-5, 6)), 4)
        Q, hQp, exact = _poly_data(coeffs, h, xi0)
        out = O.linear_recon(Q, hQp)
        scale = max(1.0, max(abs(v) for v in Q + hQp))
        assert np.allclose(out, exact, rtol=0, atol=1e-12 * scale), (deg, out, exact)


def test_linear_recon_not_exact_at_degree_8():
    coeffs = [0] * 8 + [1]
    Q, hQp, exact = _poly_data(coeffs, sp.Rational(1, 2), sp.Integer(0))
    out = O.linear_recon(Q, hQp)
    assert abs(out[0] - exact[0]) > 1e-8


def _golden():
    with open(os.path.join(GOLDEN, "sub_stencil.json")) as f:
        return json.load(f)


def test_candidate_point_values_match_printed_formulas():
    g = _golden()
    half_powers = np.array([0.5 ** m for m in range(5)])
    for k in range(7):
        C = O.poly_coef_matrix(k)                # (5, 8) monomial coefficient map
        value_map = half_powers @ C              # q_k(1/2) as a map of the data
        printed = np.array(g["q"][str(k)]["num"], dtype=float) / g["q"][str(k)]["den"]
        assert np.allclose(value_map, printed, atol=1e-14), (k, value_map, printed)


def test_linear_weights_recover_p7():
    g = _golden()
    d = np.array([a / b for a, b in g["d"]])
    assert abs(d.sum() - 1.0) < 1e-15
    combo = sum(d[k] * np.array(g["q"][str(k)]["num"], dtype=float) / g["q"][str(k)]["den"] for k in range(7))
    p7 = np.array(g["p7"]["num"], dtype=float) / g["p7"]["den"]
    assert np.allclose(combo, p7, atol=1e-15)
    # and the oracle's WENO with linear weights forced gives the P7 value on random data
    rng = np.random.default_rng(7)
    for _ in range(20):
        s = rng.normal(size=8)
        _, _, diag = O.weno_left(s, diag=True)
        lin_val = float(np.dot(d, diag["q"]))
        Qv, hv = s[:4], s[4:]
        assert abs(lin_val - O.linear_recon(Qv, hv)[0]) < 1e-13


def _sympy_candidates():
    """Candidate polynomials from their definitions, solved exactly with sympy."""
    xi = sp.Symbol("xi")
    a, b, c, d, A, B, C, D = sp.symbols("a b c d A B C D")
    avg = {-1: a, 0: b, 1: c, 2: d}
    slope = {-1: A, 0: B, 1: C, 2: D}
    defs = {
        0: (2, [("avg", -1), ("avg", 0), ("slope", -1)]),
        1: (2, [("avg", -1), ("avg", 0), ("avg", 1)]),
        2: (3, [("avg", 0), ("avg", 1), ("avg", 2), ("slope", 2)]),
        3: (2, [("avg", -1), ("avg", 0), ("avg", 1)]),
        4: (2, [("avg", 0), ("avg", 1), ("avg", 2)]),
        5: (4, [("avg", -1), ("avg", 0), ("avg", 1), ("slope", -1), ("slope", 0)]),
        6: (4, [("avg", 0), ("avg", 1), ("avg", 2), ("slope", 1), ("slope", 2)]),
        "1t": (3, [("avg", -1), ("avg", 0), ("avg", 1), ("slope", -1)]),
    }
    out = {}
    for key, (deg, cons) in defs.items():
        cs = sp.symbols(f"c0:{deg + 1}")
        q = sum(cs[m] * xi ** m for m in range(deg + 1))
        eqs = []
        for kind, k in cons:
            lo, hi = k - sp.Rational(1, 2), k + sp.Rational(1, 2)
            if kind == "avg":
                eqs.append(sp.Eq(sp.integrate(q, (xi, lo, hi)), avg[k]))
            else:
                eqs.append(sp.Eq(q.subs(xi, hi) - q.subs(xi, lo), slope[k]))
        sol = sp.solve(eqs, cs, dict=True)[0]
        qs = sp.expand(q.subs(sol))
        beta = sum(sp.integrate(sp.diff(qs, xi, r) ** 2, (xi, -sp.Rational(1, 2), sp.Rational(1, 2)))
                   for r in range(1, deg + 1))
        out[key] = dict(q=qs, value=sp.expand(qs.subs(xi, sp.Rational(1, 2))),
                        slope=sp.expand(sp.diff(qs, xi).subs(xi, sp.Rational(1, 2))), beta=sp.expand(beta))
    return out, (a, b, c, d, A, B, C, D)


def test_indicators_slopes_match_symbolic_definition():
    cands, syms = _sympy_candidates()
    rng = np.random.default_rng(11)
    for _ in range(10):
        s = rng.normal(size=8)
        subs = dict(zip(syms, s))
        _, _, diag = O.weno_left(s, diag=True)
        for k in range(7):
            key = "1t" if k == 1 else k
            beta_ref = float(cands[key]["beta"].subs(subs))
            assert abs(diag["beta"][k] - beta_ref) <= 1e-12 * max(1.0, abs(beta_ref)), (k, diag["beta"][k], beta_ref)
            val_ref = float(cands[k]["value"].subs(subs))
            slope_ref = float(cands[k]["slope"].subs(subs))
            assert abs(diag["q"][k] - val_ref) < 1e-12
            assert abs(diag["qs"][k] - slope_ref) < 1e-12


def _smooth_stencil(fun, dfun, h, x0=0.3):
    """Cell averages (6-pt Gauss) and h * cell-averaged slopes of a smooth function."""
    gx, gw = np.polynomial.legendre.leggauss(8)
    Q, hQ = [], []
    for k in (-1, 0, 1, 2):
        xc = x0 + k * h
        Q.append(0.5 * np.sum(gw * fun(xc + 0.5 * h * gx)))
        hQ.append(fun(xc + 0.5 * h) - fun(xc - 0.5 * h))
    return np.array(Q + hQ)


def test_weno_smooth_limit_and_zref_order():
    ratios, dev = [], []
    for h in (0.2, 0.1, 0.05, 0.025):
        s = _smooth_stencil(np.sin, np.cos, h)
        _, _, diag = O.weno_left(s, eps=1e-40, diag=True)
        beta = diag["beta"]
        Z = abs(3 * (beta[0] - beta[4]) + (beta[4] - beta[3]))
        ratios.append(Z / beta.min())
        d = np.array([3, 5, 8, 7, 7, 34, 34]) / 98.0
        dev.append(np.abs(diag["delta"] - d).max())
    orders = np.log2(np.array(ratios[:-1]) / np.array(ratios[1:]))
    assert orders.min() > 2.8, orders            # Z_ref / beta = O(h^3)
    assert dev[-1] < dev[0] and dev[-1] < 1e-3


def test_weno_discards_stencils_across_a_jump():
    # jump between cells i+1 and i+2: candidates using Q_{i+2} must lose their weight
    s = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0])
    v, sl, diag = O.weno_left(s, diag=True)
    assert abs(v - 1.0) < 1e-6
    assert diag["delta"][[2, 4, 6]].max() < 1e-6


def test_right_state_is_mirror_of_left():
    rng = np.random.default_rng(5)
    for _ in range(10):
        s = rng.normal(size=8)
        m = np.array([s[3], s[2], s[1], s[0], -s[7], -s[6], -s[5], -s[4]])
        vr, sr = O.weno_right(s)
        vl, sl = O.weno_left(m)
        assert vr == vl and sr == -sl
    # data symmetric about the interface: left and right values coincide, slopes are opposite
    s = np.array([0.3, 1.2, 1.2, 0.3, 0.4, -0.2, 0.2, -0.4])
    vl, sl = O.weno_left(s)
    vr, sr = O.weno_right(s)
    assert abs(vl - vr) < 1e-14 and abs(sl + sr) < 1e-14
