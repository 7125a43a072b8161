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


def rel_errors(gpu, ora):
    """err_p = max |gpu - oracle| / max |oracle_p| for every plane p (0 when the plane is all zero)."""
    nplanes = gpu.shape[0]
    g = gpu.reshape(nplanes, -1)
    o = ora.reshape(nplanes, -1)
    scale = np.abs(o).max(axis=1)
    diff = np.abs(g - o).max(axis=1)
    return np.where(scale > 0, diff / np.where(scale > 0, scale, 1.0), diff)


def nvars(W):
    return 3 if W.ndim == 2 else 4
