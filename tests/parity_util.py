"""Helpers shared by the GPU parity tests: run a problem through the CUDA library (C ABI via the
ctypes binding) and through the oracle, and measure the per-plane relative L-infinity error."""
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


def nvars(W):
    return 3 if W.ndim == 2 else 4
