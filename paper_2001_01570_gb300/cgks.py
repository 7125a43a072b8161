"""Thin ctypes binding of libcgks (include/cgks.h): argument marshalling only.

Every step of the computation runs in the library's CUDA kernels.  If the
library has not been built, :func:`load` raises; there is no fallback.
Device buffers may be torch CUDA tensors (their data pointers are passed).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

CGKS_OK, CGKS_E_INVAL, CGKS_E_NOMEM, CGKS_E_BUDGET, CGKS_E_CUDA, CGKS_E_NONPHYSICAL, CGKS_E_TIMEOUT, \
    CGKS_E_BUSY, CGKS_E_NOTFOUND = range(9)
CGKS_BC_PERIODIC, CGKS_BC_REFLECT, CGKS_BC_INFLOW, CGKS_BC_OUTFLOW = range(4)

_lib = None


class CgksError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"cgks status {status}: {msg}")
        self.status = status


class cgks_problem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double), ("y0", ctypes.c_double), ("y1", ctypes.c_double),
        ("gamma", ctypes.c_double), ("cfl", ctypes.c_double),
        ("bc", ctypes.c_int * 4), ("inflow", (ctypes.c_double * 4) * 4),
        ("eps_tau", ctypes.c_double), ("c_tau", ctypes.c_double), ("weno_eps", ctypes.c_double),
        ("mu", ctypes.c_double), ("recon_vars", ctypes.c_int), ("order", ctypes.c_int),
    ]


class cgks_serve_cfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_double), ("max_active", ctypes.c_int),
                ("steps_per_round", ctypes.c_int), ("tile_shape", ctypes.c_int), ("cuda_stream", ctypes.c_void_p),
                ("log_path", ctypes.c_char_p), ("order", ctypes.c_int), ("fill_cells", ctypes.c_double)]


CGKS_SERVE_ALL_ACTIVE, CGKS_SERVE_LEAST_WORK_FIRST = 0, 1


class cgks_request(ctypes.Structure):
    _fields_ = [("prob", cgks_problem), ("init_planes", ctypes.POINTER(ctypes.c_double)), ("nsteps", ctypes.c_int)]


class cgks_serve_stats_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_long) for n in ("submitted", "completed", "rejected", "failed", "active", "pending",
                                              "rounds")] + \
               [(n, ctypes.c_double) for n in ("cell_updates", "wall_s", "busy_s", "cell_updates_per_s", "p50_s",
                                                "p99_s", "mean_s", "hbm_in_use", "hbm_peak")] + \
               [("tile_shape", ctypes.c_int), ("update_cpt", ctypes.c_int), ("gpu_s", ctypes.c_double),
                ("round_overhead", ctypes.c_double), ("graph_captures", ctypes.c_long)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


def library_path() -> str:
    return _build.LIB


def load():
    """Load libcgks.so (built by paper_2001_01570_gb300.build / __graft_entry__.build).
    $CGKS_LIBRARY names another build of the same library (the bounds-checked one of the tests)."""
    global _lib
    if _lib is not None:
        return _lib
    path = os.environ.get("CGKS_LIBRARY") or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libcgks is not built ({path} missing): run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
    L.cgks_create.argtypes = [ctypes.POINTER(cgks_problem), vp, ctypes.POINTER(vp)]
    L.cgks_destroy.argtypes = [vp]
    L.cgks_set_state.argtypes = [vp, vp, ctypes.c_int, ctypes.c_double]
    L.cgks_restore_state.argtypes = [vp, vp, ctypes.c_int, ctypes.c_double, ctypes.c_long]
    L.cgks_get_state.argtypes = [vp, vp, ctypes.c_int, dp, ctypes.POINTER(ctypes.c_long)]
    L.cgks_step.argtypes = [vp, ctypes.c_int, ctypes.c_double, dp]
    L.cgks_step_fused.argtypes = [vp, ctypes.c_int, ctypes.c_double, dp]
    L.cgks_batch_step.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int]
    L.cgks_step_profiled.argtypes = [vp, ctypes.c_int, dp]
    for name in ("cgks_create", "cgks_destroy", "cgks_set_state", "cgks_restore_state", "cgks_get_state", "cgks_step",
                 "cgks_step_fused", "cgks_batch_step", "cgks_step_profiled"):
        getattr(L, name).restype = ctypes.c_int
    L.cgks_set_tile_shape.argtypes = [vp, ctypes.c_int]
    L.cgks_set_tile_shape.restype = ctypes.c_int
    L.cgks_tile_shape.argtypes = [vp]
    L.cgks_tile_shape.restype = ctypes.c_int
    L.cgks_batch_tile_shape.argtypes = [ctypes.POINTER(vp), ctypes.c_int]
    L.cgks_batch_tile_shape.restype = ctypes.c_int
    L.cgks_batch_update_cpt.argtypes = [ctypes.POINTER(vp), ctypes.c_int]
    L.cgks_batch_update_cpt.restype = ctypes.c_int
    L.cgks_serve_start.argtypes = [ctypes.POINTER(cgks_serve_cfg), ctypes.POINTER(vp)]
    L.cgks_serve_submit.argtypes = [vp, ctypes.POINTER(cgks_request), ctypes.POINTER(ctypes.c_long)]
    L.cgks_serve_poll.argtypes = [vp, ctypes.c_long, dp, ctypes.POINTER(ctypes.c_int)]
    L.cgks_serve_wait.argtypes = [vp, ctypes.c_long, ctypes.c_double, dp]
    L.cgks_serve_stats.argtypes = [vp, ctypes.POINTER(cgks_serve_stats_t)]
    L.cgks_serve_stop.argtypes = [vp]
    for name in ("cgks_serve_start", "cgks_serve_submit", "cgks_serve_poll", "cgks_serve_wait", "cgks_serve_stats",
                 "cgks_serve_stop"):
        getattr(L, name).restype = ctypes.c_int
    L.cgks_serve_last_error.restype = ctypes.c_char_p
    L.cgks_step_noalloc.argtypes = [ctypes.POINTER(cgks_problem), vp, ctypes.c_int, dp, vp]
    L.cgks_step_noalloc.restype = ctypes.c_int
    L.cgks_noalloc_last_error.restype = ctypes.c_char_p
    L.cgks_status_string.argtypes = [ctypes.c_int]
    L.cgks_status_string.restype = ctypes.c_char_p
    L.cgks_last_error.restype = ctypes.c_char_p
    L.cgks_last_launch_count.restype = ctypes.c_long
    L.cgks_problem_device_bytes.argtypes = [ctypes.POINTER(cgks_problem)]
    L.cgks_problem_device_bytes.restype = ctypes.c_double
    _lib = L
    return L


def _check(st):
    if st != CGKS_OK:
        L = load()
        raise CgksError(st, L.cgks_last_error().decode())


def inflow_sides(inflow):
    """One primitive state (rho, u, v, p) for every side, or four of them (x-low, x-high, y-low,
    y-high) -> a 4 x 4 nested list."""
    a = np.asarray(inflow, dtype=np.float64)
    if a.shape == (4,):
        a = np.tile(a, (4, 1))
    if a.shape != (4, 4):
        raise ValueError("inflow: one state (4 values) or one per side (4 x 4)")
    return a.tolist()


def make_problem(dim, nx, ny, x0, x1, y0=0.0, y1=1.0, gamma=1.4, cfl=0.5, bc=(0, 0, 0, 0),
                 inflow=(1.0, 0.0, 0.0, 1.0), eps_tau=0.01, c_tau=1.0, weno_eps=1e-6, mu=0.0, recon_vars=0,
                 order=8) -> cgks_problem:
    p = cgks_problem()
    p.dim, p.nx, p.ny = int(dim), int(nx), int(ny)
    p.x0, p.x1, p.y0, p.y1 = float(x0), float(x1), float(y0), float(y1)
    p.gamma, p.cfl = float(gamma), float(cfl)
    sides = inflow_sides(inflow)
    for k in range(4):
        p.bc[k] = int(bc[k])
        for m in range(4):
            p.inflow[k][m] = sides[k][m]
    p.eps_tau, p.c_tau, p.weno_eps = float(eps_tau), float(c_tau), float(weno_eps)
    p.mu = float(mu)
    p.recon_vars = int(recon_vars)
    p.order = int(order)
    return p


def problem_from_spec(spec) -> cgks_problem:
    """From a workloads.ProblemSpec."""
    return make_problem(spec.dim, spec.nx, spec.ny if spec.dim == 2 else 1, spec.x0, spec.x1, spec.y0, spec.y1,
                        spec.gamma, spec.cfl, spec.bc, spec.inflow, spec.eps_tau, spec.c_tau, spec.weno_eps,
                        getattr(spec, "mu", 0.0), getattr(spec, "recon_vars", 0), getattr(spec, "order", 8))


# ---------------------------------------------------------------------------- C-ABI names
def cgks_create(problem: cgks_problem, stream=None):
    L = load()
    out = ctypes.c_void_p()
    _check(L.cgks_create(ctypes.byref(problem), ctypes.c_void_p(stream or 0), ctypes.byref(out)))
    return out


def cgks_destroy(solver):
    _check(load().cgks_destroy(solver))


def _ptr(buf):
    if hasattr(buf, "data_ptr"):
        return ctypes.c_void_p(buf.data_ptr()), 1
    arr = buf
    if not (isinstance(arr, np.ndarray) and arr.dtype == np.float64 and arr.flags.c_contiguous):
        raise TypeError("host planes must be a C-contiguous float64 numpy array")
    return ctypes.c_void_p(arr.ctypes.data), 0


def cgks_set_state(solver, planes, t=0.0):
    p, dev = _ptr(planes)
    _check(load().cgks_set_state(solver, p, dev, float(t)))


def cgks_restore_state(solver, planes, t, steps):
    """Resume from a checkpoint (planes, t and the step count cgks_get_state returned)."""
    p, dev = _ptr(planes)
    _check(load().cgks_restore_state(solver, p, dev, float(t), int(steps)))


def cgks_get_state(solver, planes=None):
    """Copy the state into ``planes`` (numpy array or CUDA tensor); returns (t, steps)."""
    t = ctypes.c_double()
    steps = ctypes.c_long()
    if planes is None:
        p, dev = ctypes.c_void_p(0), 0
    else:
        p, dev = _ptr(planes)
    _check(load().cgks_get_state(solver, p, dev, ctypes.byref(t), ctypes.byref(steps)))
    return t.value, steps.value


def cgks_step(solver, nsteps, t_end=0.0):
    t = ctypes.c_double()
    _check(load().cgks_step(solver, int(nsteps), float(t_end), ctypes.byref(t)))
    return t.value


def cgks_step_fused(solver, nsteps, t_end=0.0):
    """cgks_step with both stages of each step in one kernel launch (2D; the same results)."""
    t = ctypes.c_double()
    _check(load().cgks_step_fused(solver, int(nsteps), float(t_end), ctypes.byref(t)))
    return t.value


def cgks_batch_step(solvers, nsteps):
    arr = (ctypes.c_void_p * len(solvers))(*[s.value if isinstance(s, ctypes.c_void_p) else s for s in solvers])
    _check(load().cgks_batch_step(arr, len(solvers), int(nsteps)))


def cgks_step_profiled(solver, nsteps):
    """Average per-launch milliseconds of (step-begin, stage-1 records, stage-1 flux, stage-1 update,
    stage-2 records, stage-2 flux, stage-2 update, step-end)."""
    ms = (ctypes.c_double * 8)()
    _check(load().cgks_step_profiled(solver, int(nsteps), ms))
    return list(ms)


def cgks_problem_device_bytes(prob) -> float:
    """Device bytes a solver of this problem holds (the server's admission unit)."""
    return float(load().cgks_problem_device_bytes(ctypes.byref(prob)))


TILE_SHAPES = ("16x8", "8x16", "32x4", "64x1", "16x7", "7x16", "14x8", "24x8", "16x14", "20x11", "15x15",
               "22x10", "18x12", "20x12", "15x16", "17x14", "16x16", "24x16", "32x12")


def cgks_set_tile_shape(solver, shape):
    """shape: index or name from TILE_SHAPES, -1 for the default."""
    if isinstance(shape, str):
        shape = TILE_SHAPES.index(shape)
    _check(load().cgks_set_tile_shape(solver, int(shape)))


def cgks_tile_shape(solver) -> str:
    """The solver's current tile shape, e.g. "8x16"."""
    return TILE_SHAPES[load().cgks_tile_shape(solver)]


def cgks_batch_tile_shape(solvers) -> int:
    arr = (ctypes.c_void_p * len(solvers))(*[s.value if isinstance(s, ctypes.c_void_p) else s for s in solvers])
    return int(load().cgks_batch_tile_shape(arr, len(solvers)))


def cgks_batch_update_cpt(solvers) -> int:
    arr = (ctypes.c_void_p * len(solvers))(*[s.value if isinstance(s, ctypes.c_void_p) else s for s in solvers])
    return int(load().cgks_batch_update_cpt(arr, len(solvers)))


def _scheck(st):
    if st != CGKS_OK:
        raise CgksError(st, load().cgks_serve_last_error().decode())


def cgks_serve_start(hbm_budget_bytes, max_active=64, steps_per_round=8, tile_shape=-1, stream=None, log_path=None,
                     order=CGKS_SERVE_LEAST_WORK_FIRST, fill_cells=4.0e6):
    cfg = cgks_serve_cfg(float(hbm_budget_bytes), int(max_active), int(steps_per_round), int(tile_shape),
                         ctypes.c_void_p(stream or 0), None if log_path is None else str(log_path).encode(),
                         int(order), float(fill_cells))
    out = ctypes.c_void_p()
    _scheck(load().cgks_serve_start(ctypes.byref(cfg), ctypes.byref(out)))
    return out


def cgks_serve_submit(server, problem: cgks_problem, planes: np.ndarray, nsteps: int) -> int:
    planes = np.ascontiguousarray(planes, dtype=np.float64)
    req = cgks_request(problem, planes.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(nsteps))
    rid = ctypes.c_long()
    _scheck(load().cgks_serve_submit(server, ctypes.byref(req), ctypes.byref(rid)))
    return rid.value


def cgks_serve_poll(server, req_id, out=None):
    """Returns True when finished (copying the result into ``out`` if given)."""
    done = ctypes.c_int()
    p = out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if out is not None else None
    _scheck(load().cgks_serve_poll(server, int(req_id), p, ctypes.byref(done)))
    return bool(done.value)


def cgks_serve_wait(server, req_id, timeout_s, out):
    _scheck(load().cgks_serve_wait(server, int(req_id), float(timeout_s),
                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))


def cgks_serve_stats(server) -> dict:
    st = cgks_serve_stats_t()
    _scheck(load().cgks_serve_stats(server, ctypes.byref(st)))
    return st.as_dict()


def cgks_serve_stop(server):
    _scheck(load().cgks_serve_stop(server))


NOALLOC_MAX_CELLS = 65536
NOALLOC_MAX_SIDE = 4096


def cgks_step_noalloc(problem: cgks_problem, planes_device, nsteps, t=0.0, stream=None):
    """Advance the 2D state held in ``planes_device`` (a CUDA tensor of 12 x ny x nx float64, or a
    raw device pointer) by ``nsteps`` steps in place, without any device allocation.
    Returns the new time."""
    ptr = planes_device.data_ptr() if hasattr(planes_device, "data_ptr") else int(planes_device)
    tt = ctypes.c_double(float(t))
    st = load().cgks_step_noalloc(ctypes.byref(problem), ctypes.c_void_p(ptr), int(nsteps), ctypes.byref(tt),
                                  ctypes.c_void_p(stream or 0))
    if st != CGKS_OK:
        raise CgksError(st, load().cgks_noalloc_last_error().decode())
    return tt.value


def cgks_last_launch_count() -> int:
    return int(load().cgks_last_launch_count())


# ---------------------------------------------------------------------------- convenience
class Solver:
    """Owns one cgks_solver handle."""

    def __init__(self, problem: cgks_problem, stream=None):
        self.problem = problem
        self.handle = cgks_create(problem, stream)
        self.dim = problem.dim
        self.nx = problem.nx
        self.ny = problem.ny if problem.dim == 2 else 1

    @property
    def shape(self):
        return (12, self.ny, self.nx) if self.dim == 2 else (6, self.nx)

    def set_state(self, planes, t=0.0):
        cgks_set_state(self.handle, planes, t)

    def restore(self, planes, t, steps):
        cgks_restore_state(self.handle, planes, t, steps)

    def get_state(self):
        out = np.empty(self.shape, dtype=np.float64)
        t, steps = cgks_get_state(self.handle, out)
        return out, t, steps

    def step(self, nsteps, t_end=0.0, fused=False):
        return (cgks_step_fused if fused else cgks_step)(self.handle, nsteps, t_end)

    def close(self):
        if self.handle is not None:
            cgks_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
