"""FP64 CPU oracle of the compact 8th-order gas-kinetic scheme (arXiv 2001.01570).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow reference that the
CUDA library is checked against; it shares no code with the library.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The product path never calls it.

The arithmetic lives in ``cgks_oracle.c`` (plain C, compiled with
``-ffp-contract=off`` so that every multiply and add rounds separately); this
module only compiles it and marshals numpy arrays through ctypes.

Parity status of each oracle function (pins in ``tests/test_oracle_*.py``):
  linear reconstruction (Sec. 3.2)        pinned: polynomial exactness, degree <= 7
  6th-order variant (named in Sec. 3.2)   pinned: exactness to degree 5, weights recover the
                                          degree-5 fit from the printed q_k, design order 6
  candidate polynomials q_k (Sec. 3.3)    pinned: the paper's printed q_k, d_k
  WENO-Z weights, beta_k, Z_ref           pinned: beta by quadrature, recovery of P7
  Maxwellian moments (Sec. 2.1)           pinned: Gauss-Hermite / adaptive quadrature
  Euler time derivatives (CK)             pinned: symbolic differentiation
  gas-kinetic flux (Sec. 2.1-2.2)         pinned: Euler limit, symmetry, 1D = 2D
  boundaries, tangential profiles         pinned: walls = mirrored periodic domain, uniform
                                          inflow on every side, polynomial exactness of the
                                          segment profiles, x -> s x / t -> s t invariance
  collision time (Sec. 4)                 pinned: limits of the pressure-jump term, its damping
                                          of shock oscillations, viscous mu/p (decay rates)
  S2O4 step (Sec. 2.2)                    pinned: uniform flow, conservation, Table 1/3
                                          design order, Sod/Lax vs exact Riemann
Every pin set above is itself checked against planted mistakes (tests/test_oracle_mutants.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cgks_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

BC_PERIODIC, BC_REFLECT, BC_INFLOW, BC_OUTFLOW = 0, 1, 2, 3


class Problem(ctypes.Structure):
    """Mirror of ``oc_problem`` in cgks_oracle.c."""

    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double),
        ("gamma", ctypes.c_double), ("cfl", ctypes.c_double),
        ("bc", ctypes.c_int * 4), ("inflow", (ctypes.c_double * 4) * 4),
        ("eps_tau", ctypes.c_double), ("c_tau", ctypes.c_double), ("weno_eps", ctypes.c_double),
        ("mu", ctypes.c_double), ("recon_vars", ctypes.c_int), ("order", ctypes.c_int),
    ]


def inflow_sides(inflow):
    """One primitive state (rho, u, v, p) for every side, or four of them (x-low, x-high, y-low,
    y-high) -> a 4 x 4 nested list."""
    a = np.asarray(inflow, dtype=np.float64)
    if a.shape == (4,):
        a = np.tile(a, (4, 1))
    if a.shape != (4, 4):
        raise ValueError("inflow: one state (4 values) or one per side (4 x 4)")
    return a.tolist()


def make_problem(dim, nx, ny, dx, dy, gamma=1.4, cfl=0.5, bc=(0, 0, 0, 0), inflow=(1.0, 0.0, 0.0, 1.0),
                 eps_tau=0.01, c_tau=1.0, weno_eps=1e-6, mu=0.0, recon_vars=0, order=8) -> Problem:
    p = Problem()
    p.dim, p.nx, p.ny = int(dim), int(nx), int(ny)
    p.dx, p.dy = float(dx), float(dy)
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


def compile_to(src: str, out: str) -> None:
    """gcc the C source ``src`` into the shared library ``out`` (the oracle's flags)."""
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=gnu11",
           "-o", out, src, "-lm"]
    subprocess.run(cmd, check=True)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    compile_to(_SRC, tmp)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # CGKS_ORACLE_LIB: a library built by compile_to() from an edited copy of the source
            # (the pin tests' planted-mistake check); unset, the committed source is built
            path = os.environ.get("CGKS_ORACLE_LIB") or build()
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            L.oc_linear_recon.argtypes = [dp, dp, dp]
            L.oc_weno_left.argtypes = [dp, ctypes.c_double, dp, dp, dp]
            L.oc_weno_right.argtypes = [dp, ctypes.c_double, dp, dp]
            L.oc_linear_recon_order.argtypes = [ctypes.c_int, dp, dp, dp]
            L.oc_weno_left_order.argtypes = [ctypes.c_int, dp, ctypes.c_double, dp, dp, dp]
            L.oc_weno_right_order.argtypes = [ctypes.c_int, dp, ctypes.c_double, dp, dp]
            L.oc_linear_weights.argtypes = [ctypes.c_int, dp]
            L.oc_poly_coef_matrix.argtypes = [ctypes.c_int, dp]
            L.oc_char_basis.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp, dp]
            L.oc_tang_weno.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, dp, dp, dp]
            L.oc_seg_profile.argtypes = [ctypes.c_int, dp, ctypes.c_double, dp]
            L.oc_moments_u.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, dp]
            L.oc_mom_psi_poly.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp]
            L.oc_euler_time_derivs.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp, dp, dp, dp, dp, dp, dp]
            L.oc_gks_point_flat.argtypes = [ctypes.POINTER(Problem), ctypes.c_int, dp, ctypes.c_double, dp]
            L.oc_gks_point_flat.restype = ctypes.c_int
            L.oc_cfl_dt.argtypes = [ctypes.POINTER(Problem), dp]
            L.oc_cfl_dt.restype = ctypes.c_double
            L.oc_run.argtypes = [ctypes.POINTER(Problem), dp, ctypes.c_int, ctypes.c_double, dp,
                                 ctypes.POINTER(ctypes.c_long), dp]
            L.oc_run.restype = ctypes.c_int
            L.oc_run_fixed_dt.argtypes = [ctypes.POINTER(Problem), dp, ctypes.c_int, ctypes.c_double]
            L.oc_run_fixed_dt.restype = ctypes.c_int
            L.oc_face1d_debug.argtypes = [ctypes.POINTER(Problem), dp, ctypes.c_int, ctypes.c_double, dp]
            L.oc_face1d_debug.restype = ctypes.c_int
            L.oc_set_threads.argtypes = [ctypes.c_int]
            L.oc_step2d_halo.argtypes = [ctypes.POINTER(Problem), dp, ctypes.c_double, EXCHANGE_FN, ctypes.c_void_p]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class OracleError(RuntimeError):
    pass


# ----------------------------------------------------------------------------- pieces
def linear_recon(Q, hQp, order=8):
    """Sec. 3.2: (P7, h P7_x, h^2 P7_xx) at x_{i+1/2}; order=6: the same from the degree-5 fit
    of the compact 6th-order variant."""
    Q, hQp, out = _f64(Q), _f64(hQp), np.zeros(3)
    if order == 8:
        lib().oc_linear_recon(_dp(Q), _dp(hQp), _dp(out))
    else:
        lib().oc_linear_recon_order(int(order), _dp(Q), _dp(hQp), _dp(out))
    return out


def linear_weights(order=8):
    """Sec. 3.3: the linear weights d_k of the candidates q_0..q_6 for the given order."""
    out = np.zeros(7)
    lib().oc_linear_weights(int(order), _dp(out))
    return out


def weno_left(s, eps=1e-6, diag=False, order=8):
    """Sec. 3.3: left value and h*slope at x_{i+1/2} from s = (Q_{i-1..i+2}, hQ'_{i-1..i+2})."""
    s = _f64(s)
    v, sl, d = np.zeros(1), np.zeros(1), np.zeros(28)
    lib().oc_weno_left_order(int(order), _dp(s), eps, _dp(v), _dp(sl), _dp(d))
    if diag:
        return v[0], sl[0], dict(q=d[0:7].copy(), qs=d[7:14].copy(), beta=d[14:21].copy(), delta=d[21:28].copy())
    return v[0], sl[0]


def weno_right(s, eps=1e-6, order=8):
    s = _f64(s)
    v, sl = np.zeros(1), np.zeros(1)
    lib().oc_weno_right_order(int(order), _dp(s), eps, _dp(v), _dp(sl))
    return v[0], sl[0]


def char_basis(D, gamma, Wref):
    """Right eigenvectors R (columns) of the normal Euler flux Jacobian at Wref and L = R^-1."""
    nv = D + 2
    Wref = _f64(Wref)
    R, L = np.zeros(nv * nv), np.zeros(nv * nv)
    lib().oc_char_basis(int(D), float(gamma), _dp(Wref), _dp(R), _dp(L))
    return R.reshape(nv, nv), L.reshape(nv, nv)


def tang_weno(v, eta, eps=1e-6):
    """2D reading: nonlinear point value along a face at eta from n = 5 or 3 segment means.

    Returns (value, derivative per unit eta, nonlinear weights omega)."""
    v = _f64(v)
    assert v.size in (3, 5)
    val, dval, om = np.zeros(1), np.zeros(1), np.zeros(3)
    lib().oc_tang_weno(int(v.size), _dp(v), float(eta), float(eps), _dp(val), _dp(dval), _dp(om))
    return val[0], dval[0], om[: v.size // 2 + 1].copy()


def seg_profile(v, eta):
    """2D reading: value, first and second derivative (per unit eta) at eta of the linear profile
    (degree n - 1) through n = 5 or 3 means over unit segments centred at -(n // 2) .. n // 2."""
    v = _f64(v)
    assert v.size in (3, 5)
    out = np.zeros(3)
    lib().oc_seg_profile(int(v.size), _dp(v), float(eta), _dp(out))
    return out


def poly_coef_matrix(p):
    """Monomial coefficients (rows, in xi) of candidate polynomial p as a map of the 8 stencil data."""
    out = np.zeros(40)
    lib().oc_poly_coef_matrix(int(p), _dp(out))
    return out.reshape(5, 8)


def moments_u(U, lam, half=0):
    out = np.zeros(9)
    lib().oc_moments_u(float(U), float(lam), int(half), _dp(out))
    return out


def mom_psi_poly(D, U, V, lam, K, half, a0, b0, coef=None):
    """< u^a0 v^b0 psi_k (coef . psi) > (or < u^a0 v^b0 psi_k > with coef None)."""
    out = np.zeros(D + 2)
    if coef is None:
        lib().oc_mom_psi_poly(D, U, V, lam, K, half, a0, b0, None, _dp(out))
    else:
        c = _f64(coef)
        lib().oc_mom_psi_poly(D, U, V, lam, K, half, a0, b0, _dp(c), _dp(out))
    return out


def euler_time_derivs(D, gamma, W0, Wx, Wy, Wxx, Wxy, Wyy):
    nv = D + 2
    arr = [_f64(np.resize(np.asarray(a, dtype=np.float64), 4)) for a in (W0, Wx, Wy, Wxx, Wxy, Wyy)]
    Wt, Wtt = np.zeros(4), np.zeros(4)
    lib().oc_euler_time_derivs(D, gamma, *[_dp(a) for a in arr], _dp(Wt), _dp(Wtt))
    return Wt[:nv], Wtt[:nv]


POINT_FIELDS = ("W0", "W0n", "W0t", "W0nn", "W0nt", "W0tt", "Wl", "Wln", "Wlt", "Wr", "Wrn", "Wrt")
POINT_OUT = ("S1", "S2", "Wt", "Wtt", "NEh", "NEf")


def gks_point(problem: Problem, D: int, dt: float, **fields):
    """Sec. 2.1: one quadrature point in the face frame; returns dict of outputs."""
    buf = np.zeros(48)
    for k, name in enumerate(POINT_FIELDS):
        if name in fields:
            v = np.asarray(fields[name], dtype=np.float64)
            buf[4 * k:4 * k + len(v)] = v
    out = np.zeros(25)
    err = lib().oc_gks_point_flat(ctypes.byref(problem), D, _dp(buf), dt, _dp(out))
    if err:
        raise OracleError(f"gks_point failed with {err}")
    res = {name: out[4 * k:4 * k + D + 2].copy() for k, name in enumerate(POINT_OUT)}
    res["tau"] = out[24]
    return res


def face1d(problem: Problem, W: np.ndarray, f: int, dt: float):
    W = _f64(W)
    out = np.zeros(15)
    err = lib().oc_face1d_debug(ctypes.byref(problem), _dp(W), int(f), dt, _dp(out))
    if err:
        raise OracleError(f"face1d failed with {err}")
    return dict(Fb=out[0:3], Ft=out[3:6], Wm=out[6:9], B=out[9:12], Wtt=out[12:15])


def cfl_dt(problem: Problem, W: np.ndarray) -> float:
    W = _f64(W)
    return lib().oc_cfl_dt(ctypes.byref(problem), _dp(W))


# ----------------------------------------------------------------------------- domain decomposition
BC_HALO = 4   # oracle-only side type: ghost columns supplied by the caller
EXCHANGE_FN = ctypes.CFUNCTYPE(None, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                               ctypes.c_void_p)


def step2d_halo(problem: Problem, W: np.ndarray, dt: float, exchange):
    """One S2O4 step of a subdomain whose x-sides may be BC_HALO.

    exchange(stage, state, halo) is called before each stage with the state that stage reads
    (12, ny, nx) and must fill halo (2 sides, 12 planes, 2 ghost columns, ny): side 0 column m is
    ghost column -1-m, side 1 column m is ghost column nx+m.  Returns the new state."""
    nx, ny = problem.nx, problem.ny
    Wc = _f64(W).copy()

    def cb(stage, state_p, halo_p, ctx):
        state = np.ctypeslib.as_array(state_p, shape=(12, ny, nx))
        halo = np.ctypeslib.as_array(halo_p, shape=(2, 12, 2, ny))
        exchange(stage, state, halo)

    fn = EXCHANGE_FN(cb)
    st = lib().oc_step2d_halo(ctypes.byref(problem), _dp(Wc), float(dt), fn, None)
    if st != 0:
        raise OracleError(f"oracle step failed with status {st}")
    return Wc


# ----------------------------------------------------------------------------- stepping
def set_threads(n: int):
    """OpenMP threads used by the oracle's loops from now on."""
    lib().oc_set_threads(int(n))


def run(problem: Problem, W: np.ndarray, nsteps: int, t_end: float = 0.0, t0: float = 0.0, threads=None):
    """Advance ``nsteps`` S2O4 steps (stopping at t_end when t_end > 0).

    Returns (W_new, t, steps, last_dt).  W has planes (6, nx) in 1D and
    (12, ny, nx) in 2D."""
    if threads is not None:
        set_threads(threads)
    Wc = _f64(W).copy()
    t = np.array([t0], dtype=np.float64)
    steps = ctypes.c_long(0)
    last = np.zeros(1)
    err = lib().oc_run(ctypes.byref(problem), _dp(Wc), int(nsteps), float(t_end), _dp(t),
                       ctypes.byref(steps), _dp(last))
    if err:
        raise OracleError(f"oracle run failed with status {err}")
    return Wc, float(t[0]), int(steps.value), float(last[0])


def run_fixed_dt(problem: Problem, W: np.ndarray, nsteps: int, dt: float):
    Wc = _f64(W).copy()
    err = lib().oc_run_fixed_dt(ctypes.byref(problem), _dp(Wc), int(nsteps), float(dt))
    if err:
        raise OracleError(f"oracle run failed with status {err}")
    return Wc
