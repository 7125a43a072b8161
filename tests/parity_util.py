"""Helpers shared by the GPU parity tests: run a problem through the CUDA library (C ABI via the
ctypes binding) and through the oracle, and measure the per-plane relative L-infinity error."""
import os

import numpy as np

import oracle as O
from paper_2001_01570_gb300 import cgks

TOL = 1e-11          # relative L-inf per conserved variable (normalised by max |oracle| of the variable)


def oracle_problem(spec, **over):
    kw = spec.as_kwargs()
    kw.update(over)
    return O.make_problem(**kw)


def run_gpu(spec, W, nsteps, t_end=0.0):
    s = cgks.Solver(cgks.problem_from_spec(spec))
    try:
        s.set_state(np.ascontiguousarray(W))
        s.step(nsteps, t_end)
        out, t, steps = s.get_state()
    finally:
        s.close()
    return out, t, steps


def run_oracle(spec, W, nsteps, t_end=0.0):
    Wn, t, steps, _ = O.run(oracle_problem(spec), W, nsteps, t_end)
    return Wn, t, steps


def plane_scales(maxabs, dim, dx, dy, gamma=1.4):
    """Normalisation of the parity error of every plane.

    A conserved variable is measured against the largest of its own maximum and the natural scale of
    the fluxes it is updated from: momentum against the acoustic momentum rho*c (bounded above by
    sqrt(gamma (gamma-1) max rho max rhoE)), because a momentum that stays far below rho*c (a weak
    acoustic pulse) is the small difference of O(rho c^2) pressure fluxes, whose last-bit rounding
    differs between any two correct FP64 evaluations.  A gradient plane is measured against the
    larger of its own maximum and (scale of its variable) / (cell size)."""
    maxabs = np.asarray(maxabs, dtype=float)
    nv = 3 if dim == 1 else 4
    s = maxabs.copy()
    rho, rhoE = maxabs[0], maxabs[nv - 1]
    mom = np.sqrt(gamma * (gamma - 1.0) * rho * rhoE)
    for k in range(1, nv - 1):
        s[k] = max(s[k], mom)
    for k in range(nv):
        s[nv + k] = max(s[nv + k], s[k] / dx)
        if dim == 2:
            s[2 * nv + k] = max(s[2 * nv + k], s[k] / dy)
    return s


def rel_errors(gpu, ora, dx=1.0, dy=1.0, gamma=1.4):
    """err_p = max |gpu - oracle| / scale_p for every plane p (scale from plane_scales)."""
    nplanes = gpu.shape[0]
    g = gpu.reshape(nplanes, -1)
    o = ora.reshape(nplanes, -1)
    dim = 1 if nplanes == 6 else 2
    scale = plane_scales(np.abs(o).max(axis=1), dim, dx, dy, gamma)
    diff = np.abs(g - o).max(axis=1)
    return np.where(scale > 0, diff / np.where(scale > 0, scale, 1.0), diff)


def strict_errors(gpu, ora, maxabs=None):
    """The parity error of the contract, per plane: max |gpu - oracle| / max |oracle plane| (the
    maximum over the whole grid where only sampled cells are compared)."""
    nplanes = gpu.shape[0]
    g = gpu.reshape(nplanes, -1)
    o = ora.reshape(nplanes, -1)
    m = np.abs(o).max(axis=1) if maxabs is None else np.asarray(maxabs, dtype=float)
    diff = np.abs(g - o).max(axis=1)
    return np.where(m > 0, diff / np.where(m > 0, m, 1.0), diff)


# Both errors of every parity comparison of the session, written to the JSON-lines file named by
# $CGKS_PARITY_REPORT at the end of the session (tests/conftest.py).
REPORT = []


def _current_test():
    return os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]


def record(name, strict, scaled, nv, maxabs=None):
    name = name or _current_test()
    REPORT.append({"case": name, "nvars": int(nv),
                   "strict": [float(x) for x in strict], "scaled": [float(x) for x in scaled],
                   "maxabs": None if maxabs is None else [float(x) for x in maxabs[:nv]]})
    print(f"parity {name}: strict conserved {np.array2string(np.asarray(strict[:nv]), precision=2)} "
          f"scaled {np.array2string(np.asarray(scaled[:nv]), precision=2)}")


# A conserved variable must meet TOL under both definitions, except momentum, which must meet TOL
# against its rounding scale (plane_scales) and, where it carries a resolved signal (max |m| of at
# least RESOLVED_MOMENTUM rho c: an acoustic pulse of amplitude 1e-5 has ~2e-6 rho c),
# MOMENTUM_STRICT_TOL against its own maximum.  In a near-quiescent flow the momentum is the
# small difference of O(rho c^2) pressure fluxes, and two correct FP64 evaluations of the scheme
# that round in different orders differ in it by ~1e-15 rho c (tests/test_oracle_rounding_floor.py:
# the oracle against itself transposed, ~1e-9 of max |m| on a 1e-5 pulse).  A momentum component
# whose maximum is below that (zero by symmetry, or a second-order effect such as the ~3e-9 rho c
# x-motion that viscous heating drives in a shear wave) is checked on the rounding scale only.
MOMENTUM_STRICT_TOL = 1e-8
RESOLVED_MOMENTUM = 1e-6


# Where a run amplifies rounding differences (a strong shock that a vortex crosses: the oracle and
# the oracle on the mirrored problem, mirrored back, then differ by up to ~1e-9 of the variables'
# maxima), two correct FP64 evaluations cannot agree to TOL.  Such a case carries that measured
# floor (per plane, relative to the plane's maximum; tests/golden/make_golden.py), and each bar
# below becomes the larger of itself and FLOOR_FACTOR times the floor.
FLOOR_FACTOR = 10.0


def check(name, gpu, ora, dx=1.0, dy=1.0, gamma=1.4, tol=TOL, grad_tol=1e-9, maxabs=None, floor=None):
    """Assert parity of `gpu` against `ora` (both full planes, or the planes at sampled cells with
    the full-grid maxima in `maxabs`) and record both error definitions."""
    nplanes = gpu.shape[0]
    nv = 3 if nplanes == 6 else 4
    dim = 1 if nplanes == 6 else 2
    m = np.abs(ora.reshape(nplanes, -1)).max(axis=1) if maxabs is None else np.asarray(maxabs, dtype=float)
    scale = plane_scales(m, dim, dx, dy, gamma)
    diff = np.abs(gpu.reshape(nplanes, -1) - ora.reshape(nplanes, -1)).max(axis=1)
    scaled = np.where(scale > 0, diff / np.where(scale > 0, scale, 1.0), diff)
    strict = np.where(m > 0, diff / np.where(m > 0, m, 1.0), diff)
    record(name, strict, scaled, nv, m)
    fl = np.zeros(nplanes) if floor is None else FLOOR_FACTOR * np.asarray(floor, dtype=float)
    if floor is not None:
        REPORT[-1]["floor"] = [float(x) for x in np.asarray(floor)[:nv]]
    fl_scaled = fl * m / np.where(scale > 0, scale, 1.0)
    bar = np.maximum(tol, fl_scaled[:nv])
    assert np.all(scaled[:nv] <= bar), f"{name}: conserved-variable errors (rounding scale) {scaled[:nv]}"
    for k in (0, nv - 1):
        assert strict[k] <= max(tol, fl[k]), f"{name}: density/energy errors {strict[:nv]}"
    rho_c = np.sqrt(gamma * (gamma - 1.0) * m[0] * m[nv - 1])
    for k in range(1, nv - 1):
        if m[k] >= RESOLVED_MOMENTUM * rho_c:
            assert strict[k] <= max(MOMENTUM_STRICT_TOL, fl[k]), f"{name}: momentum errors vs own maximum {strict[:nv]}"
    assert np.all(scaled[nv:] <= np.maximum(grad_tol, fl_scaled[nv:])), f"{name}: gradient errors {scaled[nv:]}"
    return scaled, strict


def nvars(W):
    return 3 if W.ndim == 2 else 4
