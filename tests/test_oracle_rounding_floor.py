"""How closely two correct FP64 evaluations of the scheme can agree on a weak acoustic pulse.

The oracle is run on a pulse of the batched workload's weakest amplitude (A = 1e-5 on a fluid at
rest, 64^2, periodic) and again on the same data transposed (x <-> y, momenta and gradient planes
exchanged): the same arithmetic on the same values, with sums taken in another order.  The two
agree in density and energy to a few ulp of their maxima and in momentum to a few ulp of rho c,
the scale of the pressure fluxes the momentum is the difference of -- but only to ~1e-9 of the
momentum's own maximum (~2e-6).  So 1e-11 of max |momentum| is below the rounding floor of FP64
for this flow: the parity tests measure momentum against max(max |m|, rho c) at 1e-11 and
against max |m| at 1e-8 (tests/parity_util.py)."""
import numpy as np
import pytest

import oracle as O
from parity_util import MOMENTUM_STRICT_TOL, TOL, plane_scales
from paper_2001_01570_gb300 import workloads as wl


def _transpose(W):
    W = np.transpose(W, (0, 2, 1)).copy()
    W[[1, 2]] = W[[2, 1]]
    W[[5, 6]] = W[[6, 5]]
    W[[9, 10]] = W[[10, 9]]
    W[4:8], W[8:12] = W[8:12].copy(), W[4:8].copy()
    return W


@pytest.mark.parametrize("A,lo", [(1e-5, 1e-11), (1e-3, 0.0)])
def test_momentum_rounding_floor_of_a_weak_pulse(A, lo):
    spec, W = wl.acoustic_pulse(64, A, 5.0, 20.3, 37.8)
    nsteps = 60
    a = O.run(O.make_problem(**spec.as_kwargs()), W, nsteps)[0]
    kw = spec.as_kwargs()
    kw["nx"], kw["ny"], kw["dx"], kw["dy"] = kw["ny"], kw["nx"], kw["dy"], kw["dx"]
    b = _transpose(O.run(O.make_problem(**kw), _transpose(W), nsteps)[0])
    diff = np.abs(a - b).reshape(12, -1).max(axis=1)
    m = np.abs(a).reshape(12, -1).max(axis=1)
    scaled = diff / plane_scales(m, 2, spec.dx, spec.dy)
    strict = diff / m
    assert diff.max() > 0.0                                   # the two evaluations do round differently
    assert scaled[:4].max() <= 1e-2 * TOL                      # agree on the rounding scale
    assert strict[[0, 3]].max() <= 1e-2 * TOL                  # density and energy: also on their own
    assert lo <= strict[1:3].max() <= 0.25 * MOMENTUM_STRICT_TOL   # momentum: floor above 1e-11 at A = 1e-5
