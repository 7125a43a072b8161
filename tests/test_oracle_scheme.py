"""Pins of the oracle's full time step (Sec. 2.2 S2O4 + Sec. 3.1 Gauss-theorem gradient update)
against the paper's printed accuracy tables, exact solutions and invariants.

- Table 1 (dt = 0.5 dx^2) and Table 3 (CFL 0.8) of Sec. 4.1: errors within a few percent of the
  printed values, design orders 8 and 4
- the 100-cell density wave of the same section at CFL 0.3 returns to its initial state at t = 2
- uniform flow is preserved bit for bit with every boundary type
- mass, momentum and energy are conserved to roundoff with periodic boundaries, and the cell-averaged
  gradients sum to zero (telescoping of the Gauss-theorem update)
- the 2D scheme on y-independent data reproduces the 1D scheme; x/y transposition commutes with a step
- Sod and Lax shock tubes converge to the exact Riemann solution without large overshoots
- the isentropic vortex converges at high order to its translated initial state
- the CFL rule gives the step count quoted in Sec. 4.6 (143 steps to t = 28.45 at CFL 0.3 on 200^2)
"""
import json
import math
import os

import numpy as np
import pytest

import exact_riemann as ER
import oracle as O
from conftest import GOLDEN
from paper_2001_01570_gb300 import workloads as wl


def _table(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _errors(W, ex):
    e = np.abs(W[0] - ex[0])
    return e.mean(), math.sqrt((e ** 2).mean()), e.max()


def test_table1_eighth_order_small_dt():
    tab = _table("table1_compact8.json")
    got = []
    for N, L1, L2, Li in tab["rows"][:3]:
        spec, W = wl.density_wave_1d(N, eps=1e-4, eps_tau=0.0)
        P = O.make_problem(**spec.as_kwargs())
        dx = 2.0 / N
        dt = 0.5 * dx * dx
        nst = int(round(200.0 / dt))
        Wn = O.run_fixed_dt(P, W, nst, dt)
        e1, e2, ei = _errors(Wn, wl.density_wave_1d_exact(N, nst * dt, eps=1e-4))
        got.append((e1, ei))
        assert abs(e1 / L1 - 1) < 0.05 and abs(e2 / L2 - 1) < 0.05 and abs(ei / Li - 1) < 0.05, (N, e1, L1, ei, Li)
    orders = [math.log2(got[k][0] / got[k + 1][0]) for k in range(2)]
    assert min(orders) > 7.5, orders


def test_table3_fourth_order_at_cfl_08():
    tab = _table("table3_compact8_cfl08.json")
    got = []
    for N, L1, L2, Li in tab["rows"][:4]:
        spec, W = wl.density_wave_1d(N, eps=1e-4, eps_tau=0.0, cfl=0.8)
        P = O.make_problem(**spec.as_kwargs())
        Wn, t, steps, _ = O.run(P, W, 10 ** 7, t_end=200.0)
        assert t == 200.0
        e1, e2, ei = _errors(Wn, wl.density_wave_1d_exact(N, t, eps=1e-4))
        got.append(e1)
        assert abs(e1 / L1 - 1) < 0.03 and abs(e2 / L2 - 1) < 0.03 and abs(ei / Li - 1) < 0.03, (N, e1, L1)
    orders = [math.log2(got[k] / got[k + 1]) for k in range(3)]
    assert min(orders) > 3.9, orders


@pytest.mark.parametrize("eps_tau,bound", [(0.0, 1e-9), (0.01, 5e-4)])
def test_density_wave_100_cells(eps_tau, bound):
    spec, W = wl.density_wave_1d(100, eps=0.2, cfl=0.3, eps_tau=eps_tau)
    P = O.make_problem(**spec.as_kwargs())
    Wn, t, steps, _ = O.run(P, W, 10 ** 6, t_end=2.0)
    assert t == 2.0 and 700 < steps < 850
    ex = wl.density_wave_1d_exact(100, 2.0, eps=0.2)
    assert np.abs(Wn[0] - ex[0]).max() < bound
    assert np.allclose(Wn[:3].sum(axis=1), W[:3].sum(axis=1), rtol=1e-14, atol=1e-12)


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (2, 3, 1, 1), (1, 1, 0, 0), (3, 3, 3, 3)])
def test_uniform_flow_preserved_bitwise_2d(bc):
    nx, ny = 9, 7
    g = 1.4
    rho, u, v, p = 1.3, 0.7, -0.4, 0.9
    if bc[0] == 1:
        u = 0.0
    if bc[2] == 1:
        v = 0.0
    W = np.zeros((12, ny, nx))
    W[0], W[1], W[2], W[3] = rho, rho * u, rho * v, p / (g - 1) + 0.5 * rho * (u * u + v * v)
    P = O.make_problem(dim=2, nx=nx, ny=ny, dx=0.1, dy=0.15, cfl=0.5, bc=bc, inflow=(rho, u, v, p))
    Wn, _, _, _ = O.run(P, W, 5)
    assert np.array_equal(Wn, W)


def test_uniform_flow_preserved_bitwise_1d():
    g, rho, u, p = 1.4, 0.8, 1.1, 0.6
    W = np.zeros((6, 11))
    # same evaluation order as the oracle's inflow state, so the ghost state is bitwise equal
    W[0], W[1], W[2] = rho, rho * u, p / (g - 1.0) + 0.5 * rho * u * u
    for bc in ((0, 0, 0, 0), (3, 3, 0, 0), (2, 3, 0, 0)):
        P = O.make_problem(dim=1, nx=11, ny=1, dx=0.1, dy=1.0, cfl=0.5, bc=bc, inflow=(rho, u, 0.0, p))
        Wn, _, _, _ = O.run(P, W, 5)
        assert np.array_equal(Wn, W), bc


def test_conservation_and_gradient_sum_periodic():
    spec, W = wl.isentropic_vortex(24)
    P = O.make_problem(**spec.as_kwargs())
    Wn, _, steps, _ = O.run(P, W, 4)
    tot0, tot1 = W[:4].sum(axis=(1, 2)), Wn[:4].sum(axis=(1, 2))
    assert np.all(np.abs(tot1 - tot0) <= 1e-13 * np.abs(W[:4]).sum(axis=(1, 2)))
    assert np.abs(Wn[4:].sum(axis=(1, 2))).max() < 1e-11


def test_2d_reproduces_1d_on_y_uniform_data():
    spec, W1 = wl.density_wave_1d(24, eps=0.2)
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
    # y-momentum and y-gradients stay at roundoff (the tangential fits sum constants to ~1 ulp)
    assert np.abs(b[2]).max() < 1e-15 and np.abs(b[8:]).max() < 1e-13


def test_transpose_symmetry():
    spec, W = wl.isentropic_vortex(16)
    P = O.make_problem(**spec.as_kwargs())
    # transpose: swap x and y, rhoU <-> rhoV, x-gradients <-> y-gradients
    perm = [0, 2, 1, 3]
    WT = np.empty_like(W)
    for k in range(4):
        WT[k] = W[perm[k]].T
        WT[4 + k] = W[8 + perm[k]].T
        WT[8 + k] = W[4 + perm[k]].T
    a, _, _, _ = O.run(P, W, 3)
    b, _, _, _ = O.run(P, WT, 3)
    for k in range(4):
        for grp_a, grp_b in ((0, 0), (4, 8), (8, 4)):
            x = a[grp_a + perm[k]].T
            y = b[grp_b + k]
            assert np.abs(x - y).max() <= 1e-13 * max(1.0, np.abs(x).max())


@pytest.mark.parametrize("name,states,t_end,n,l1_max,overshoot", [
    ("sod", wl.SOD, 0.2, 100, 3.5e-3, 0.01),
    ("sod", wl.SOD, 0.2, 200, 2.0e-3, 0.01),
    ("lax", wl.LAX, 0.16, 100, 6.0e-3, 0.02),
])
def test_shock_tube_vs_exact_riemann(name, states, t_end, n, l1_max, overshoot):
    spec, W = wl.shock_tube_1d(n, states, cfl=0.5)
    P = O.make_problem(**spec.as_kwargs())
    Wn, t, _, _ = O.run(P, W, 10 ** 6, t_end=t_end)
    ex = ER.cell_average_density(states[0], states[1], t_end, n)
    jump = max(states[0][0], states[1][0], ex.max()) - min(states[0][0], states[1][0], ex.min())
    assert np.abs(Wn[0] - ex).mean() < l1_max
    assert Wn[0].max() <= ex.max() + overshoot * jump
    assert Wn[0].min() >= ex.min() - overshoot * jump


def test_pressure_jump_collision_time_damps_shock_oscillations():
    """Sec. 4 enlarges the collision time where the pressures on the two sides of an interface
    differ, so that at a shock the flux leans on the nonlinear (non-equilibrium) part: on the Sod
    and Lax tubes the solution with the enhancement (C = 1) has less total variation and smaller
    over- and undershoots than the same run with C = 0, at the price of a little smearing."""
    for states, t_end in ((wl.SOD, 0.2), (wl.LAX, 0.16)):
        ex = ER.cell_average_density(states[0], states[1], t_end, 100)
        got = {}
        for c_tau in (1.0, 0.0):
            spec, W = wl.shock_tube_1d(100, states, cfl=0.5)
            spec.c_tau = c_tau
            Wn, _, _, _ = O.run(O.make_problem(**spec.as_kwargs()), W, 10 ** 6, t_end=t_end)
            r = Wn[0]
            got[c_tau] = (np.abs(np.diff(r)).sum(), max(r.max() - ex.max(), 0.0) + max(ex.min() - r.min(), 0.0),
                          np.abs(r - ex).mean())
        assert got[1.0][0] < got[0.0][0], got
        assert got[1.0][1] < got[0.0][1], got
        assert got[1.0][2] > got[0.0][2], got


def test_isentropic_vortex_convergence():
    errs = []
    for n in (20, 40):
        spec, W = wl.isentropic_vortex(n, eps_tau=0.0)
        P = O.make_problem(**spec.as_kwargs())
        dx = 10.0 / n
        T = 0.5
        nst = int(math.ceil(T / (0.1 * dx * dx)))
        Wn = O.run_fixed_dt(P, W, nst, T / nst)
        _, ex = wl.isentropic_vortex(n, t=T)
        errs.append(np.abs(Wn[0] - ex[0]).max())
    assert math.log2(errs[0] / errs[1]) > 3.0, errs


def test_isentropic_vortex_convergence_on_tall_cells():
    """Cells twice as tall as wide (dy = 2 dx), CFL 0.5 to t = 1: the error falls at the scheme's
    fourth temporal order (3.9 and 4.2 between 20, 40 and 80 columns), which needs each direction's
    spacing in the derivatives along and across every face (a tangential slope scaled by the wrong
    spacing leaves an O(dt) time-derivative error and drops the order below 2)."""
    errs = []
    L, T = 10.0, 1.0
    for n in (20, 40, 80):
        m = n // 2
        W = wl.cell_state_2d(wl._vortex_fun(0.5 * L, 0.5 * L, L, 5.0, 1.4), n, m, 0.0, L, 0.0, L, 1.4)
        ex = wl.cell_state_2d(wl._vortex_fun(0.5 * L + T, 0.5 * L + T, L, 5.0, 1.4), n, m, 0.0, L, 0.0, L, 1.4)
        P = O.make_problem(dim=2, nx=n, ny=m, dx=L / n, dy=L / m, eps_tau=0.0, cfl=0.5)
        Wn, t, _, _ = O.run(P, W, 10 ** 6, t_end=T)
        assert t == T
        errs.append(np.abs(Wn[0] - ex[0]).max())
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert min(orders) > 3.5, (errs, orders)


def test_cfl_rule_reproduces_tam_webb_step_count():
    spec, W = wl.tam_webb(200)
    P = O.make_problem(**spec.as_kwargs())
    dt = O.cfl_dt(P, W)
    assert math.ceil(28.45 / dt) == 143
    assert abs(math.ceil(56.9 / dt) - 286) <= 1


def _smooth_periodic_2d(Lx, Ly):
    def fun(x, y):
        a, b = 2 * math.pi * x / Lx, 2 * math.pi * y / Ly
        return (1.0 + 0.2 * np.sin(a) * np.cos(b) + 0.1 * np.cos(2 * b), 0.4 + 0.3 * np.cos(a + b),
                -0.2 + 0.25 * np.sin(b - a), 1.0 + 0.15 * np.sin(a + 2 * b))
    return fun


def test_reflecting_walls_equal_the_mirrored_periodic_domain():
    """A reflecting wall is a mirror (Sec. 4's reflective boundaries): on a domain with walls at
    both ends the solution equals the half of the periodic domain of twice the length whose other
    half holds the mirror image.  Under x -> -x a field f maps to S f(-x) with S flipping the sign
    of the x-momentum, so cell averages and y-gradients map by S and x-gradients by -S (and the
    same with x and y exchanged, and in 1D)."""
    g = 1.4
    nst = 4
    # 1D
    spec, W = wl.density_wave_1d(10, eps=0.2)
    S = np.array([1.0, -1.0, 1.0])
    mirror = np.concatenate([(S[:, None] * W[:3])[:, ::-1], (-S[:, None] * W[3:])[:, ::-1]])
    Wd = np.concatenate([mirror, W], axis=1)
    kw = spec.as_kwargs()
    dt = 0.02
    Pw = O.make_problem(**dict(kw, bc=(O.BC_REFLECT, O.BC_REFLECT, 0, 0)))
    Pp = O.make_problem(**dict(kw, nx=20))
    a = O.run_fixed_dt(Pw, W, nst, dt)
    b = O.run_fixed_dt(Pp, Wd, nst, dt)[:, 10:]
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), np.abs(a - b).max()
    # 2D, walls on x (periodic in y) and walls on y (periodic in x)
    nx, ny, Lx, Ly = 8, 6, 0.8, 0.6
    W2 = wl.cell_state_2d(_smooth_periodic_2d(Lx, Ly), nx, ny, 0.0, Lx, 0.0, Ly, g)
    for axis in (0, 1):
        S = np.array([1.0, -1.0, 1.0, 1.0]) if axis == 0 else np.array([1.0, 1.0, -1.0, 1.0])
        grad_sign = [1.0, -1.0, 1.0] if axis == 0 else [1.0, 1.0, -1.0]   # groups W, W_x, W_y
        flip = (lambda A: A[:, :, ::-1]) if axis == 0 else (lambda A: A[:, ::-1, :])
        mirror = np.concatenate([grad_sign[q] * S[:, None, None] * flip(W2[4 * q:4 * q + 4]) for q in range(3)])
        Wd = np.concatenate([mirror, W2], axis=2 - axis)
        base = dict(dim=2, nx=nx, ny=ny, dx=Lx / nx, dy=Ly / ny, gamma=g, eps_tau=0.01)
        bcw = (O.BC_REFLECT, O.BC_REFLECT, 0, 0) if axis == 0 else (0, 0, O.BC_REFLECT, O.BC_REFLECT)
        Pw = O.make_problem(**dict(base, bc=bcw))
        Pp = O.make_problem(**dict(base, nx=2 * nx if axis == 0 else nx, ny=2 * ny if axis == 1 else ny))
        a = O.run_fixed_dt(Pw, W2, nst, 0.01)
        b = O.run_fixed_dt(Pp, Wd, nst, 0.01)
        b = b[:, :, nx:] if axis == 0 else b[:, ny:, :]
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), (axis, np.abs(a - b).max())


def test_supersonic_inflow_keeps_its_uniform_state():
    """A uniform supersonic stream entering through an inflow side with the same state is an exact
    steady solution, whatever states the other sides' inflow entries hold."""
    g = 1.4
    state = np.array([1.0, 2.5, 0.0, 1.0 / g])     # sound speed 1: Mach 2.5
    other = [3.0, 0.3, -0.2, 2.0]
    for side in range(4):
        q = state.copy()
        axis, sign = side // 2, (1.0 if side % 2 == 0 else -1.0)
        q[1], q[2] = (sign * 2.5, 0.3) if axis == 0 else (0.3, sign * 2.5)
        inflow = [other] * 4
        inflow[side] = list(q)
        bc = [0, 0, 0, 0]
        bc[side], bc[side ^ 1] = O.BC_INFLOW, O.BC_OUTFLOW
        P = O.make_problem(dim=2, nx=8, ny=7, dx=0.1, dy=0.1, gamma=g, bc=bc, inflow=inflow)
        W = np.zeros((12, 7, 8))
        W[0:4] = np.array([q[0], q[0] * q[1], q[0] * q[2], q[3] / (g - 1) + 0.5 * q[0] * (q[1] ** 2 + q[2] ** 2)])[:, None, None]
        out = O.run_fixed_dt(P, W, 3, 0.01)
        assert np.abs(out - W).max() <= 1e-13, (side, np.abs(out - W).max())
    for side in range(2):
        u = 2.5 if side == 0 else -2.5
        inflow = [other] * 4
        inflow[side] = [1.0, u, 0.0, 1.0 / g]
        bc = [O.BC_INFLOW, O.BC_OUTFLOW, 0, 0] if side == 0 else [O.BC_OUTFLOW, O.BC_INFLOW, 0, 0]
        P = O.make_problem(dim=1, nx=9, ny=1, dx=0.1, dy=0.1, gamma=g, bc=bc, inflow=inflow)
        W = np.zeros((6, 9))
        W[0:3] = np.array([1.0, u, 1.0 / (g * (g - 1)) + 0.5 * u * u])[:, None]
        out = O.run_fixed_dt(P, W, 3, 0.01)
        assert np.abs(out - W).max() <= 1e-13, (side, np.abs(out - W).max())


@pytest.mark.parametrize("mu", [0.0, 2e-3])
def test_scale_invariance(mu):
    """The Euler (and Navier-Stokes) equations are unchanged by x -> s x, t -> s t (with mu -> s mu):
    the same cell averages on a grid s times coarser, gradients divided by s, advanced with s dt,
    give the same averages and gradients divided by s.  Every spacing enters the scheme only in such
    ratios, so with s a power of two the results agree to rounding.  A large eps_tau keeps the
    non-equilibrium terms of the interface state in play."""
    s = 4.0
    nx, ny, Lx, Ly = 8, 6, 0.8, 0.9
    W2 = wl.cell_state_2d(_smooth_periodic_2d(Lx, Ly), nx, ny, 0.0, Lx, 0.0, Ly, 1.4)
    Ws = W2.copy()
    Ws[4:] /= s
    base = dict(dim=2, nx=nx, ny=ny, gamma=1.4, eps_tau=0.3)
    a = O.run_fixed_dt(O.make_problem(**base, dx=Lx / nx, dy=Ly / ny, mu=mu), W2, 3, 0.01)
    b = O.run_fixed_dt(O.make_problem(**base, dx=s * Lx / nx, dy=s * Ly / ny, mu=s * mu), Ws, 3, s * 0.01)
    b[4:] *= s
    for q in range(3):
        A, B = a[4 * q:4 * q + 4], b[4 * q:4 * q + 4]
        assert np.abs(A - B).max() <= 1e-12 * np.abs(A).max(), (q, np.abs(A - B).max())
    spec, W1 = wl.density_wave_1d(12, eps=0.2, eps_tau=0.3)
    kw = dict(spec.as_kwargs(), mu=mu)
    W1s = W1.copy()
    W1s[3:] /= s
    a = O.run_fixed_dt(O.make_problem(**kw), W1, 3, 0.02)
    b = O.run_fixed_dt(O.make_problem(**dict(kw, dx=s * kw["dx"], mu=s * mu)), W1s, 3, s * 0.02)
    b[3:] *= s
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()
