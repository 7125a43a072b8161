"""Sec. 4's 1D acoustic wave (periodic [0, 1/3], eps = 1e-5, omega = 6 pi, CFL 0.2): after 10 and
100 domain lengths of travel the oracle matches linear acoustics (tests/acoustic_exact.py) on the
coarse meshes the paper uses.  Run with eps_tau = 0 (the accuracy reading): with the paper's 0.01
the collision time adds a viscosity tau p = 0.01 dt p that damps the wave by several per cent."""
import math

import numpy as np
import pytest

import acoustic_exact as AE
import oracle as O
from paper_2001_01570_gb300 import workloads as wl

EPS, RHO_INF = 1e-5, 1.1771
A_INF = math.sqrt(1.4 * 101325.0 / RHO_INF)


def _errors(n, t_end, eps_tau=0.0):
    spec, W = wl.acoustic_wave_1d(n, eps_tau=eps_tau)
    Wn, t, _, _ = O.run(O.make_problem(**spec.as_kwargs()), W, 10 ** 7, t_end=t_end)
    assert t == t_end
    ex = wl.cell_state_1d(lambda x: AE.acoustic_wave_exact(x, t_end), n, 0.0, 1.0 / 3.0, 1.4)
    e_rho = np.abs(Wn[0] - ex[0]).max() / (EPS * RHO_INF)
    e_u = np.abs(Wn[1] / Wn[0] - ex[1] / ex[0]).max() / (EPS * A_INF)
    return e_rho, e_u


@pytest.mark.parametrize("n,t_end,bound", [(12, 0.01, 0.01), (16, 0.01, 0.003), (16, 0.1, 0.03)])
def test_acoustic_wave_coarse_meshes(n, t_end, bound):
    e_rho, e_u = _errors(n, t_end)
    assert e_rho < bound and e_u < bound


def test_collision_time_damps_the_wave():
    e0, _ = _errors(16, 0.01, 0.0)
    e1, _ = _errors(16, 0.01, 0.01)
    assert e1 > 10 * e0
