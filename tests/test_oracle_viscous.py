"""Viscous collision time tau = mu/p + C|dp|/(sum p) dt (Sec. 4): the kinetic flux then carries the
Navier-Stokes stresses and Fourier heat flux of the BGK model (Prandtl number 1).  Pins: a shear
wave v = A sin(2 pi x) decays like exp(-nu k^2 t) and an entropy wave (density at constant
pressure) like exp(-alpha k^2 t) with alpha = kappa/(rho c_p) = nu; conservation is kept."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2001_01570_gb300 import workloads as wl


def _decay_ratio(kind, n, mu, t_end=0.5):
    spec, W = wl.shear_wave(n, amp=1e-4, mu=mu, kind=kind)
    P = O.make_problem(**spec.as_kwargs())
    xc = (np.arange(n) + 0.5) / n
    basis = np.sin(2.0 * math.pi * xc)[None, :]
    plane = 2 if kind == "shear" else 0

    def amp(Wc):
        f = Wc[plane] - (0.0 if kind == "shear" else Wc[plane].mean())
        return (f * basis).mean() / (basis * basis).mean()

    Wn, t, steps, _ = O.run(P, W, 10 ** 6, t_end=t_end)
    assert t == t_end
    rate = -math.log(amp(Wn) / amp(W)) / t
    tot0, tot1 = W[:4].sum(axis=(1, 2)), Wn[:4].sum(axis=(1, 2))
    assert np.all(np.abs(tot1 - tot0) <= 1e-13 * np.abs(W[:4]).sum(axis=(1, 2)) + 1e-15)
    return rate / (mu * (2.0 * math.pi) ** 2)


@pytest.mark.parametrize("n,mu", [(32, 0.002), (32, 0.01), (64, 0.01)])
def test_shear_wave_decays_at_nu_k2(n, mu):
    assert abs(_decay_ratio("shear", n, mu) - 1.0) < 0.01


def test_entropy_wave_decays_at_alpha_k2():
    # Pr = 1: alpha = nu.  The kinetic flux adds O(tau/dt) corrections to the heat flux; with
    # dt ~ 5 tau the rate is within a few percent
    assert abs(_decay_ratio("entropy", 32, 0.002) - 1.0) < 0.05


def test_viscous_cfl_term():
    spec, W = wl.shear_wave(64, amp=1e-4, mu=0.01)
    P = O.make_problem(**spec.as_kwargs())
    dt = O.cfl_dt(P, W)
    c = 1.0                     # rho = 1, p = 1/gamma; |v| <= 1e-4
    assert abs(dt / (0.5 / 64 / (c + 2 * 0.01 * 64)) - 1.0) < 2e-4
    # each direction's diffusion term on its own spacing: with dy = 4 dx the x bound decides,
    # with dx = 4 dy the y bound, and in 1D the x bound alone
    h = 1.0 / 64
    for dx, dy in ((h, 4 * h), (4 * h, h)):
        kw = spec.as_kwargs()
        kw.update(dx=dx, dy=dy)
        want = 0.5 * min(dx / (c + 2 * 0.01 / dx), dy / (c + 2 * 0.01 / dy))
        assert abs(O.cfl_dt(O.make_problem(**kw), W) / want - 1.0) < 2e-4
    spec1, W1 = wl.density_wave_1d(32, eps=0.0)
    spec1.mu = 0.01
    P1 = O.make_problem(**spec1.as_kwargs())
    u, a = W1[1, 0] / W1[0, 0], math.sqrt(1.4 * 1.0 / W1[0, 0])
    want = P1.cfl * P1.dx / (abs(u) + a + 2 * 0.01 / P1.dx)
    assert abs(O.cfl_dt(P1, W1) / want - 1.0) < 1e-12
