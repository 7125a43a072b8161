"""Regular shock reflection (Sec. 4's 2D shock test: Mach 2.9, 29-degree incident shock, reflecting
wall, inflow on the left and top with different states): the oracle reaches the exact steady
states of the three regions (oblique-shock relations, tests/shock_reflection_exact.py) and puts the
reflection point where the incident shock meets the wall."""
import math

import numpy as np

import oracle as O
import shock_reflection_exact as EX
from paper_2001_01570_gb300 import workloads as wl


def test_textbook_region_states():
    (r1, p1), (r2, p2), (r3, p3) = EX.regions()
    assert abs(r2 - 1.69997) < 1e-5 and abs(p2 - 1.52819) < 1e-5
    assert abs(r3 - 2.68723) < 1e-4 and abs(p3 - 2.93398) < 1e-4
    post = wl.oblique_shock_state(2.9, 29.0)
    assert abs(post[0] - r2) < 1e-12 and abs(post[3] - p2) < 1e-12


def test_shock_reflection_steady_state():
    g = 1.4
    spec, W = wl.shock_reflection(40, 10)
    Wn, t, steps, _ = O.run(O.make_problem(**spec.as_kwargs()), W, 10 ** 6, t_end=5.0)
    assert t == 5.0
    rho = Wn[0]
    p = (g - 1.0) * (Wn[3] - 0.5 * (Wn[1] ** 2 + Wn[2] ** 2) / rho)
    assert rho.min() > 0.0 and p.min() > 0.0
    (r1, p1), (r2, p2), (r3, p3) = EX.regions()
    x = (np.arange(40) + 0.5) * 0.1
    # behind the reflected shock, next to the wall, downstream end
    assert np.abs(rho[0:2, 34:] / r3 - 1.0).max() < 0.01
    assert np.abs(p[0:2, 34:] / p3 - 1.0).max() < 0.01
    # behind the incident shock, below the top boundary, mid-domain
    assert np.abs(rho[7:10, 12:24] / r2 - 1.0).max() < 0.01
    assert np.abs(p[7:10, 12:24] / p2 - 1.0).max() < 0.01
    # free stream ahead of both shocks
    assert np.abs(rho[0:3, 0:8] / r1 - 1.0).max() < 0.01
    # the density on the wall row crosses the mid value of regions 1 and 3 near the reflection
    # point x = 1 / tan(29 deg) (the reflected shock leans downstream by less than a cell there)
    xr = 1.0 / math.tan(math.radians(29.0))
    first = x[np.argmax(rho[0] > 0.5 * (r1 + r3))]
    assert abs(first - xr) < 0.3
