"""2D reading: nonlinear point values along a face (WENO-Z over the line averages of neighbouring
face rows).  Pins: the linear weights at the two Gauss points equal the closed forms derived by
hand from the segment-mean polynomials; with the nonlinearity switched off the value is the
full-stencil polynomial; polynomial data of the candidates' degree are reproduced exactly; the
value stays on the smooth side of a jump; mirror symmetry; and a strong normal shock on a 2D grid
(which the linear quartic turns negative at the faces parallel to it) runs."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2001_01570_gb300 import workloads as wl

G = 1.0 / (2.0 * math.sqrt(3.0))


def _segment_means(coeffs, offsets):
    """means of sum_m c_m eta^m over unit segments centred at the offsets"""
    out = []
    for o in offsets:
        lo, hi = o - 0.5, o + 0.5
        out.append(sum(c * (hi ** (m + 1) - lo ** (m + 1)) / (m + 1) for m, c in enumerate(coeffs)))
    return np.array(out)


def test_linear_weights_closed_form_at_gauss_points():
    # linear data: every candidate is the same line, all beta equal, Z = 0, so omega = d
    v5 = _segment_means([0.3, 1.7], range(-2, 3))
    _, _, om = O.tang_weno(v5, +G)
    d_plus = [7 / 36 - math.sqrt(3) / 1080, 11 / 18, 7 / 36 + math.sqrt(3) / 1080]
    assert np.allclose(om, d_plus, rtol=0, atol=1e-14)
    _, _, om = O.tang_weno(v5, -G)
    assert np.allclose(om, d_plus[::-1], rtol=0, atol=1e-14)
    v3 = np.array([1.0, 1.5, 2.0])          # equal jumps: beta_0 = beta_1
    for eta in (G, -G):
        _, _, om = O.tang_weno(v3, eta)
        assert np.allclose(om, [0.5, 0.5], rtol=0, atol=1e-15)


def test_linear_limit_is_the_full_stencil_polynomial():
    rng = np.random.default_rng(7)
    for _ in range(20):
        v5, v3 = rng.normal(size=5), rng.normal(size=3)
        for eta in (G, -G, 0.37):
            # eps -> infinity switches the nonlinearity off (alpha_k -> d_k)
            val, _, _ = O.tang_weno(v5, eta, eps=1e300)
            A = np.array([[((o + 0.5) ** (m + 1) - (o - 0.5) ** (m + 1)) / (m + 1) for m in range(5)]
                          for o in range(-2, 3)])
            c = np.linalg.solve(A, v5)
            assert abs(val - sum(c[m] * eta ** m for m in range(5))) < 1e-13
        for eta in (G, -G):
            val, _, _ = O.tang_weno(v3, eta, eps=1e300)
            # the quadratic through three segment means: v0 + eta (v+ - v-)/2 + (v- - 2 v0 + v+)/2 (eta^2 - 1/12)
            q = v3[1] + eta * (v3[2] - v3[0]) / 2 + (v3[0] - 2 * v3[1] + v3[2]) / 2 * (eta * eta - 1 / 12)
            assert abs(val - q) < 1e-14


def test_candidate_degree_polynomials_are_exact():
    rng = np.random.default_rng(11)
    for _ in range(10):
        c2 = rng.normal(size=3)
        v5 = _segment_means(c2, range(-2, 3))
        for eta in (G, -G):
            val, dval, _ = O.tang_weno(v5, eta)
            assert abs(val - (c2[0] + c2[1] * eta + c2[2] * eta * eta)) < 1e-13
            assert abs(dval - (c2[1] + 2 * c2[2] * eta)) < 1e-12
        c1 = rng.normal(size=2)
        v3 = _segment_means(c1, range(-1, 2))
        for eta in (G, -G):
            val, dval, _ = O.tang_weno(v3, eta)
            assert abs(val - (c1[0] + c1[1] * eta)) < 1e-14 and abs(dval - c1[1]) < 1e-14


def test_jump_value_stays_on_the_smooth_side_and_mirror_symmetry():
    # the linear quartic gives -0.025 at +G for these means; the nonlinear value is ~0.125
    v5 = np.array([1.0, 1.0, 0.125, 0.125, 0.125])
    for eta in (G, -G):
        val, _, _ = O.tang_weno(v5, eta)
        assert abs(val - 0.125) < 1e-5
    v3 = np.array([1.0, 0.1, 0.1])
    for eta in (G, -G):
        val, _, _ = O.tang_weno(v3, eta)
        assert abs(val - 0.1) < 1e-5
    rng = np.random.default_rng(3)
    for n in (5, 3):
        v = rng.normal(size=n)
        a, da, _ = O.tang_weno(v, G)
        b, db, _ = O.tang_weno(v[::-1].copy(), -G)
        assert abs(a - b) < 1e-14 and abs(da + db) < 1e-13


@pytest.mark.parametrize("recon_vars", [0, 1])
def test_strong_normal_shock_on_a_2d_grid(recon_vars):
    """Sod along x, uniform in y: 2D steps agree with the 1D scheme (K differs but the kinetic
    model is the same: the y-velocity plays one internal degree of freedom)."""
    spec, W1 = wl.shock_tube_1d(40, wl.SOD, cfl=0.5)
    spec.recon_vars = recon_vars
    a, _, _, _ = O.run(O.make_problem(**spec.as_kwargs()), W1, 12)
    kw = spec.as_kwargs()
    kw.update(dim=2, ny=4, dy=1.0)
    W2 = np.repeat(wl.state_1d_as_2d(W1), 4, axis=1)
    b, _, _, _ = O.run(O.make_problem(**kw), W2, 12)
    assert np.all(b[:, 1:] == b[:, :1])                                # rows stay identical
    # no y-momentum and no y-gradients up to the rounding of the fitted tangential derivatives
    b1 = np.array([b[0, 0], b[1, 0], b[3, 0], b[4, 0], b[5, 0], b[7, 0]])
    rel = np.abs(a - b1).max(axis=1) / np.abs(a).max(axis=1)
    assert rel[:3].max() < 1e-12
    assert np.abs(b[2]).max() <= 1e-15 * np.abs(b[1]).max()
    assert np.abs(b[8:]).max() <= 1e-15 * np.abs(b[4:8]).max()


@pytest.mark.parametrize("n", [5, 3])
def test_segment_profiles_exact_for_polynomials(n):
    """The linear tangential profile through n unit-segment means is the degree-(n-1) polynomial
    with those means: for every polynomial of degree <= n - 1 it returns the value and the first
    and second derivatives exactly, at any eta on the central segment; degree n is not reproduced."""
    rng = np.random.default_rng(70 + n)
    offs = np.arange(n) - n // 2

    def means(coef):
        # exact mean of sum_m coef[m] eta^m over [o - 1/2, o + 1/2]
        return np.array([sum(c * ((o + 0.5) ** (m + 1) - (o - 0.5) ** (m + 1)) / (m + 1)
                             for m, c in enumerate(coef)) for o in offs])

    for deg in range(n):
        for _ in range(3):
            coef = rng.normal(size=deg + 1)
            for eta in (-0.5, -0.2886751345948129, 0.0, 0.31, 0.5):
                got = O.seg_profile(means(coef), eta)
                want = [sum(c * eta ** m for m, c in enumerate(coef)),
                        sum(m * c * eta ** (m - 1) for m, c in enumerate(coef) if m >= 1),
                        sum(m * (m - 1) * c * eta ** (m - 2) for m, c in enumerate(coef) if m >= 2)]
                assert np.allclose(got, want, rtol=0, atol=1e-12), (n, deg, eta, got, want)
    coef = np.zeros(n + 1)
    coef[n] = 1.0
    got = O.seg_profile(means(coef), 0.3)
    assert abs(got[0] - 0.3 ** n) > 1e-4 or abs(got[2] - n * (n - 1) * 0.3 ** (n - 2)) > 1e-4


def test_strong_normal_shock_along_y_on_a_2d_grid():
    """Sod along y, uniform in x, outflow at both y ends: the 2D steps agree with the 1D scheme, the
    y-outflow ghosts behaving as the 1D ones do."""
    spec, W1 = wl.shock_tube_1d(40, wl.SOD, cfl=0.5)
    a, _, _, _ = O.run(O.make_problem(**spec.as_kwargs()), W1, 12)
    kw = spec.as_kwargs()
    kw.update(dim=2, nx=4, ny=40, dx=1.0, dy=spec.dx, bc=(0, 0, spec.bc[0], spec.bc[1]))
    W2 = np.zeros((12, 40, 4))
    for k_1d, k_2d in ((0, 0), (1, 2), (2, 3)):
        W2[k_2d] = W1[k_1d][:, None]
        W2[8 + k_2d] = W1[3 + k_1d][:, None]
    b, _, _, _ = O.run(O.make_problem(**kw), W2, 12)
    assert np.all(b[:, :, 1:] == b[:, :, :1])                          # columns stay identical
    b1 = np.array([b[0, :, 0], b[2, :, 0], b[3, :, 0], b[8, :, 0], b[10, :, 0], b[11, :, 0]])
    rel = np.abs(a - b1).max(axis=1) / np.abs(a).max(axis=1)
    assert rel[:3].max() < 1e-12 and rel[3:].max() < 1e-10
