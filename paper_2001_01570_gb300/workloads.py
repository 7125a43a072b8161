"""Seeded synthetic inputs: initial conditions as cell averages and cell-averaged gradients.

This module holds no arithmetic of the scheme itself.  It turns analytic
initial conditions into the two kinds of data the compact scheme evolves
(Sec. 3.1): cell averages of the conservative variables and cell-averaged
gradients, the latter by the divergence theorem (face line-averages of the
initial field, Eq. compact-deriv-1).  Both the CPU oracle tests and the CUDA
path read the arrays produced here, so the two sides start from identical
inputs.

Plane layout (the library's layout): 2D ``(12, ny, nx)`` = rho, rhoU, rhoV,
rhoE, then their x-gradients, then their y-gradients; 1D ``(6, nx)`` = rho,
rhoU, rhoE, then their x-gradients.

Quadrature: 6-point Gauss-Legendre per direction for cell averages (6x6 per
cell) and for face line-averages.  Discontinuities in the initial data are
placed on cell faces; face values are taken as one-sided limits from inside
the cell.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

NG = 6
_GX, _GW = np.polynomial.legendre.leggauss(NG)
GAUSS_X = 0.5 * _GX          # nodes on [-1/2, 1/2]
GAUSS_W = 0.5 * _GW          # weights summing to 1
_INSIDE = 1e-9               # one-sided face evaluation, in cell widths

BC_PERIODIC, BC_REFLECT, BC_INFLOW, BC_OUTFLOW = 0, 1, 2, 3


@dataclass
class ProblemSpec:
    """Statement of an Euler problem (gamma, grid, CFL, boundary types), Sec. 4."""
    dim: int
    nx: int
    ny: int
    x0: float
    x1: float
    y0: float = 0.0
    y1: float = 1.0
    gamma: float = 1.4
    cfl: float = 0.5
    bc: tuple = (BC_PERIODIC,) * 4
    inflow: tuple = (1.0, 0.0, 0.0, 1.0)   # one primitive state, or one per side (x-lo, x-hi, y-lo, y-hi)
    eps_tau: float = 0.01
    c_tau: float = 1.0
    weno_eps: float = 1e-6
    mu: float = 0.0
    recon_vars: int = 0          # nonlinear reconstruction: 0 conservative, 1 characteristic
    order: int = 8               # 8: the paper's compact 8th-order scheme; 6: compact 6th-order variant
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def dx(self) -> float:
        return (self.x1 - self.x0) / self.nx

    @property
    def dy(self) -> float:
        return (self.y1 - self.y0) / self.ny if self.dim == 2 else 1.0

    @property
    def cells(self) -> int:
        return self.nx * (self.ny if self.dim == 2 else 1)

    def as_kwargs(self) -> dict:
        return dict(dim=self.dim, nx=self.nx, ny=self.ny if self.dim == 2 else 1, dx=self.dx, dy=self.dy,
                    gamma=self.gamma, cfl=self.cfl, bc=tuple(self.bc), inflow=tuple(self.inflow),
                    eps_tau=self.eps_tau, c_tau=self.c_tau, weno_eps=self.weno_eps, mu=self.mu,
                    recon_vars=self.recon_vars, order=self.order)


def prim_to_cons(rho, u, v, p, gamma):
    return rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)


# ----------------------------------------------------------------------------- 1D
def cell_state_1d(fun, nx, x0, x1, gamma):
    """fun(x) -> (rho, u, p).  Returns planes (6, nx)."""
    dx = (x1 - x0) / nx
    xc = x0 + (np.arange(nx) + 0.5) * dx
    out = np.zeros((6, nx))
    for gx, gw in zip(GAUSS_X, GAUSS_W):
        r, u, p = fun(xc + gx * dx)
        W = prim_to_cons(r, u, 0.0, p, gamma)
        out[0] += gw * W[0]
        out[1] += gw * W[1]
        out[2] += gw * W[3]
    lo = prim_to_cons(*_pad_uv(fun(xc - 0.5 * dx + _INSIDE * dx)), gamma)
    hi = prim_to_cons(*_pad_uv(fun(xc + 0.5 * dx - _INSIDE * dx)), gamma)
    for k, comp in enumerate((0, 1, 3)):
        out[3 + k] = (hi[comp] - lo[comp]) / dx
    return out


def _pad_uv(rup):
    r, u, p = rup
    return r, u, 0.0 * u, p


# ----------------------------------------------------------------------------- 2D
def cell_state_2d(fun, nx, ny, x0, x1, y0, y1, gamma, row_chunk=64):
    """fun(x, y) -> (rho, u, v, p) on arrays.  Returns planes (12, ny, nx)."""
    dx, dy = (x1 - x0) / nx, (y1 - y0) / ny
    xc = x0 + (np.arange(nx) + 0.5) * dx
    out = np.zeros((12, ny, nx))
    for j0 in range(0, ny, row_chunk):
        j1 = min(ny, j0 + row_chunk)
        yc = y0 + (np.arange(j0, j1) + 0.5) * dy
        Y, X = np.meshgrid(yc, xc, indexing="ij")
        acc = np.zeros((4, j1 - j0, nx))
        for gy, wy in zip(GAUSS_X, GAUSS_W):
            for gx, wx in zip(GAUSS_X, GAUSS_W):
                W = prim_to_cons(*fun(X + gx * dx, Y + gy * dy), gamma)
                for k in range(4):
                    acc[k] += (wx * wy) * W[k]
        out[0:4, j0:j1] = acc
        # divergence theorem: x-gradient from the line averages on the x-faces
        lo = np.zeros((4, j1 - j0, nx))
        hi = np.zeros((4, j1 - j0, nx))
        for gy, wy in zip(GAUSS_X, GAUSS_W):
            Wl = prim_to_cons(*fun(X - 0.5 * dx + _INSIDE * dx, Y + gy * dy), gamma)
            Wh = prim_to_cons(*fun(X + 0.5 * dx - _INSIDE * dx, Y + gy * dy), gamma)
            for k in range(4):
                lo[k] += wy * Wl[k]
                hi[k] += wy * Wh[k]
        out[4:8, j0:j1] = (hi - lo) / dx
        lo[:] = 0.0
        hi[:] = 0.0
        for gx, wx in zip(GAUSS_X, GAUSS_W):
            Wl = prim_to_cons(*fun(X + gx * dx, Y - 0.5 * dy + _INSIDE * dy), gamma)
            Wh = prim_to_cons(*fun(X + gx * dx, Y + 0.5 * dy - _INSIDE * dy), gamma)
            for k in range(4):
                lo[k] += wx * Wl[k]
                hi[k] += wx * Wh[k]
        out[8:12, j0:j1] = (hi - lo) / dy
    return out


def state_1d_as_2d(W1):
    """Embed 1D planes (6, nx) as 2D planes (12, 1, nx) with rhoV = 0 and no y-variation."""
    nx = W1.shape[1]
    W = np.zeros((12, 1, nx))
    W[0, 0], W[1, 0], W[3, 0] = W1[0], W1[1], W1[2]
    W[4, 0], W[5, 0], W[7, 0] = W1[3], W1[4], W1[5]
    return W


# ----------------------------------------------------------------------------- problems
def density_wave_1d(n=100, eps=0.2, gamma=1.4, cfl=0.3, eps_tau=0.01):
    """rho = 1 + eps sin(pi x), U = 1, p = 1 on periodic [0, 2] (Sec. 4.1)."""
    spec = ProblemSpec(dim=1, nx=n, ny=1, x0=0.0, x1=2.0, gamma=gamma, cfl=cfl, eps_tau=eps_tau,
                       name=f"density-wave-1d-{n}")

    def fun(x):
        return 1.0 + eps * np.sin(np.pi * x), np.ones_like(x), np.ones_like(x)

    return spec, cell_state_1d(fun, n, 0.0, 2.0, gamma)


def density_wave_1d_exact(n, t, eps=0.2, gamma=1.4):
    def fun(x):
        return 1.0 + eps * np.sin(np.pi * (x - t)), np.ones_like(x), np.ones_like(x)
    return cell_state_1d(fun, n, 0.0, 2.0, gamma)


def acoustic_wave_1d(n=16, eps=1e-5, omega=6.0 * math.pi, gamma=1.4, cfl=0.2, eps_tau=0.01):
    """Sec. 4's 1D acoustic wave: u = eps a cos(omega x), rho = rho_inf (1 + eps cos(2 omega x)),
    p = p_inf (rho/rho_inf)^gamma on the periodic [0, 1/3] (rho_inf = 1.1771, p_inf = 101325)."""
    rho_inf, p_inf = 1.1771, 101325.0
    a = math.sqrt(gamma * p_inf / rho_inf)
    spec = ProblemSpec(dim=1, nx=n, ny=1, x0=0.0, x1=1.0 / 3.0, gamma=gamma, cfl=cfl, eps_tau=eps_tau,
                       name=f"acoustic-wave-1d-{n}")

    def fun(x):
        rho = rho_inf * (1.0 + eps * np.cos(2.0 * omega * x))
        return rho, eps * a * np.cos(omega * x), p_inf * (rho / rho_inf) ** gamma

    return spec, cell_state_1d(fun, n, 0.0, 1.0 / 3.0, gamma)


SOD = ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
LAX = ((0.445, 0.698, 3.528), (0.5, 0.0, 0.571))


def shock_tube_1d(n=100, states=SOD, gamma=1.4, cfl=0.5, eps_tau=0.01):
    """Riemann problem on [0,1] with the jump at x = 0.5 (on a face for even n), outflow ends."""
    (rl, ul, pl), (rr, ur, pr) = states
    spec = ProblemSpec(dim=1, nx=n, ny=1, x0=0.0, x1=1.0, gamma=gamma, cfl=cfl,
                       bc=(BC_OUTFLOW, BC_OUTFLOW, BC_PERIODIC, BC_PERIODIC), eps_tau=eps_tau,
                       name=f"shock-tube-{n}")

    def fun(x):
        left = x < 0.5
        return (np.where(left, rl, rr), np.where(left, ul, ur), np.where(left, pl, pr))

    return spec, cell_state_1d(fun, n, 0.0, 1.0, gamma)


def _vortex_fun(xc, yc, L, strength, gamma, uinf=1.0, vinf=1.0):
    def fun(x, y):
        dxv = (x - xc + 0.5 * L) % L - 0.5 * L
        dyv = (y - yc + 0.5 * L) % L - 0.5 * L
        r2 = dxv * dxv + dyv * dyv
        e = np.exp(0.5 * (1.0 - r2))
        du = -strength / (2.0 * math.pi) * e * dyv
        dv = strength / (2.0 * math.pi) * e * dxv
        T = 1.0 - (gamma - 1.0) * strength ** 2 / (8.0 * gamma * math.pi ** 2) * e * e
        rho = T ** (1.0 / (gamma - 1.0))
        return rho, uinf + du, vinf + dv, rho * T
    return fun


def isentropic_vortex(n=512, L=10.0, strength=5.0, gamma=1.4, cfl=0.5, t=0.0, eps_tau=0.01):
    """Isentropic vortex on free stream (1,1,1,1), periodic [0,L]^2; at time t it is the
    initial vortex translated by (t, t)."""
    spec = ProblemSpec(dim=2, nx=n, ny=n, x0=0.0, x1=L, y0=0.0, y1=L, gamma=gamma, cfl=cfl, eps_tau=eps_tau,
                       name=f"isentropic-vortex-{n}")
    fun = _vortex_fun(0.5 * L + t, 0.5 * L + t, L, strength, gamma)
    return spec, cell_state_2d(fun, n, n, 0.0, L, 0.0, L, gamma)


def shock_vortex(nx=1024, ny=512, mach=1.1, vortex_mach=0.3, a=0.05, b=0.2, center=(0.25, 0.5),
                 gamma=1.4, cfl=0.5, eps_tau=0.01):
    """Stationary normal shock at x=0.5 on [0,2]x[0,1] (upstream rho=1, p=1, Mach `mach`), with a
    vortex (peak speed vortex_mach * c, linear core of radius a, decaying to zero at b) upstream.
    Inflow at x=0, outflow at x=2, reflecting walls in y."""
    g = gamma
    c1 = math.sqrt(g)
    u1 = mach * c1
    rho2 = (g + 1.0) * mach ** 2 / ((g - 1.0) * mach ** 2 + 2.0)
    p2 = 1.0 + 2.0 * g / (g + 1.0) * (mach ** 2 - 1.0)
    u2 = u1 / rho2
    vm = vortex_mach * c1
    k = vm * a / (a * a - b * b)
    cfac = (g - 1.0) / g
    Ta = 1.0 - cfac * k * k * (b ** 4 / (2.0 * a * a) - a * a / 2.0 - 2.0 * b * b * math.log(b / a))
    xc, yc = center

    def fun(x, y):
        dxv, dyv = x - xc, y - yc
        r = np.sqrt(dxv * dxv + dyv * dyv)
        rs = np.maximum(r, 1e-300)
        vt = np.where(r <= a, vm * r / a, np.where(r <= b, k * (r - b * b / rs), 0.0))
        T_out = 1.0 - cfac * k * k * (b ** 4 / (2.0 * rs * rs) - rs * rs / 2.0 - 2.0 * b * b * np.log(b / rs))
        T_in = Ta - cfac * vm * vm * (a * a - r * r) / (2.0 * a * a)
        T = np.where(r <= a, T_in, np.where(r <= b, T_out, 1.0))
        rho_v = T ** (1.0 / (g - 1.0))
        up = x < 0.5
        rho = np.where(up, rho_v, rho2)
        p = np.where(up, rho_v * T, p2)
        u = np.where(up, u1 - vt * dyv / rs, u2)
        v = np.where(up, vt * dxv / rs, 0.0)
        return rho, u, v, p

    spec = ProblemSpec(dim=2, nx=nx, ny=ny, x0=0.0, x1=2.0, y0=0.0, y1=1.0, gamma=g, cfl=cfl,
                       bc=(BC_INFLOW, BC_OUTFLOW, BC_REFLECT, BC_REFLECT), inflow=(1.0, u1, 0.0, 1.0),
                       eps_tau=eps_tau, name=f"shock-vortex-{nx}x{ny}-M{mach:g}")
    return spec, cell_state_2d(fun, nx, ny, 0.0, 2.0, 0.0, 1.0, g)


def oblique_shock_state(mach, angle_deg, gamma=1.4):
    """State behind a planar shock at angle_deg to a uniform stream (rho = 1, p = 1/gamma, Mach
    `mach` along +x), the shock running down and to the right: Rankine-Hugoniot for the normal
    component, tangential velocity unchanged.  Returns primitive (rho, u, v, p)."""
    g = gamma
    b = math.radians(angle_deg)
    u1 = mach                                      # c = 1 upstream
    un1, ut = u1 * math.sin(b), u1 * math.cos(b)
    mn2 = un1 * un1                                # normal Mach number squared (c = 1)
    r2 = (g + 1.0) * mn2 / ((g - 1.0) * mn2 + 2.0)
    p2 = (1.0 / g) * (1.0 + 2.0 * g / (g + 1.0) * (mn2 - 1.0))
    un2 = un1 / r2
    # shock tangent (cos b, -sin b), downstream normal (sin b, cos b)
    return r2, ut * math.cos(b) + un2 * math.sin(b), -ut * math.sin(b) + un2 * math.cos(b), p2


def shock_reflection(nx=200, ny=50, mach=2.9, angle_deg=29.0, gamma=1.4, cfl=0.5, eps_tau=0.01):
    """Regular shock reflection (Sec. 4, 2D shock test): [0,4] x [0,1], Mach-2.9 stream entering on
    the left, the state behind a 29-degree incident shock entering through the top, reflecting
    bottom wall, outflow on the right; the domain starts in the free-stream state."""
    g = gamma
    free = (1.0, mach, 0.0, 1.0 / g)
    post = oblique_shock_state(mach, angle_deg, g)
    spec = ProblemSpec(dim=2, nx=nx, ny=ny, x0=0.0, x1=4.0, y0=0.0, y1=1.0, gamma=g, cfl=cfl,
                       bc=(BC_INFLOW, BC_OUTFLOW, BC_REFLECT, BC_INFLOW),
                       inflow=(free, free, free, post), eps_tau=eps_tau,
                       name=f"shock-reflection-{nx}x{ny}")
    W = np.zeros((12, ny, nx))
    W[:4] = np.asarray(prim_to_cons(*free, g)).reshape(4, 1, 1)
    return spec, W


def acoustic_pulse(N, A, b, cx, cy, gamma=1.4, cfl=0.5, eps_tau=0.01):
    """rho = 1, u = v = 0, p = 1/gamma + A exp(-ln2 r^2 / b^2) on periodic [0,N]^2, dx = 1,
    r the minimum-image distance to (cx, cy) (pulse shape of Sec. 4, plane pressure pulse)."""
    spec = ProblemSpec(dim=2, nx=N, ny=N, x0=0.0, x1=float(N), y0=0.0, y1=float(N), gamma=gamma, cfl=cfl,
                       eps_tau=eps_tau, name=f"acoustic-pulse-{N}")
    L = float(N)

    def fun(x, y):
        dxv = (x - cx + 0.5 * L) % L - 0.5 * L
        dyv = (y - cy + 0.5 * L) % L - 0.5 * L
        p = 1.0 / gamma + A * np.exp(-math.log(2.0) * (dxv * dxv + dyv * dyv) / (b * b))
        return np.ones_like(x), np.zeros_like(x), np.zeros_like(x), p

    return spec, cell_state_2d(fun, N, N, 0.0, L, 0.0, L, gamma)


def shear_wave(n=32, amp=1e-3, mu=0.01, gamma=1.4, cfl=0.5, kind="shear"):
    """Viscous decay test on periodic [0,1]^2 (rho = 1, c = 1): kind "shear" has v = amp sin(2 pi x),
    kind "entropy" has rho = 1 + amp sin(2 pi x) at constant pressure.  Both decay like
    exp(-nu k^2 t), nu = mu / rho, k = 2 pi (Prandtl number 1)."""
    p0 = 1.0 / gamma

    def fun(x, y):
        s = np.sin(2.0 * math.pi * x)
        if kind == "shear":
            return np.ones_like(x), np.zeros_like(x), amp * s, np.full_like(x, p0)
        return 1.0 + amp * s, np.zeros_like(x), np.zeros_like(x), np.full_like(x, p0)

    spec = ProblemSpec(dim=2, nx=n, ny=n, x0=0.0, x1=1.0, y0=0.0, y1=1.0, gamma=gamma, cfl=cfl, mu=mu,
                       name=f"{kind}-wave-{n}")
    return spec, cell_state_2d(fun, n, n, 0.0, 1.0, 0.0, 1.0, gamma)


def tam_webb(n=200, gamma=1.4, cfl=0.3, eps_tau=0.01):
    """Acoustic, entropy and vorticity pulses on a Mach 0.5 stream over [-100,100]^2 (Sec. 4.6)."""
    e1, e2, e3 = 1e-2, 1e-3, 4e-4
    a1, a2, a3 = math.log(2) / 9.0, math.log(2) / 25.0, math.log(2) / 25.0
    x1, x2 = -100.0 / 3.0, 100.0 / 3.0
    pinf = 1.0 / gamma

    def fun(x, y):
        r1 = (x - x1) ** 2 + y ** 2
        r2 = (x - x2) ** 2 + y ** 2
        g1, g2, g3 = np.exp(-a1 * r1), np.exp(-a2 * r2), np.exp(-a3 * r2)
        return 1.0 + e1 * g1 + e2 * g2, 0.5 + e3 * g3 * y, -e3 * g3 * (x - x2), pinf + e1 * g1

    spec = ProblemSpec(dim=2, nx=n, ny=n, x0=-100.0, x1=100.0, y0=-100.0, y1=100.0, gamma=gamma, cfl=cfl,
                       eps_tau=eps_tau, name=f"tam-webb-{n}")
    return spec, cell_state_2d(fun, n, n, -100.0, 100.0, -100.0, 100.0, gamma)


# ----------------------------------------------------------------------------- seeded workloads
def batched_pulses(seed=1570, count=256, nmin=64, nmax=512):
    """Parameters of the batched workload: square periodic grids, sizes log-uniform in
    [nmin, nmax], pulse amplitude log-uniform in [1e-5, 1e-3], half-width uniform in [3, 10]
    cells, centre uniform in the domain."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        N = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        A = 10.0 ** rng.uniform(-5.0, -3.0)
        b = rng.uniform(3.0, 10.0)
        cx, cy = rng.uniform(0.0, N), rng.uniform(0.0, N)
        out.append(dict(N=N, A=A, b=b, cx=cx, cy=cy))
    return out


def batched_acoustic_1d(seed=618, count=2048, nmin=12, nmax=48):
    """Parameters of the small-amplitude 1D batch: copies of the 1D acoustic-wave test with grid
    sizes log-uniform in [nmin, nmax] cells (the coarse meshes of Sec. 4 use 12 to 24)."""
    rng = np.random.default_rng(seed)
    return [dict(N=int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))) for _ in range(count)]


def served_requests(seed=2001, count=2000, rate=50.0, nmin=128, nmax=2048, smin=100, smax=2000):
    """Poisson request stream: exponential inter-arrivals (mean 1/rate s), grid N log-uniform,
    steps log-uniform, initial condition uniform over {pulse, vortex, shock-vortex}, shock Mach
    uniform in [1.05, 1.5]."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    kinds = ("pulse", "vortex", "shock-vortex")
    for rid in range(count):
        t += rng.exponential(1.0 / rate)
        N = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        steps = int(round(math.exp(rng.uniform(math.log(smin), math.log(smax)))))
        kind = kinds[int(rng.integers(0, 3))]
        req = dict(id=rid, arrival=t, N=N, steps=steps, kind=kind)
        if kind == "pulse":
            req.update(A=10.0 ** rng.uniform(-5.0, -3.0), b=rng.uniform(3.0, 10.0),
                       cx=rng.uniform(0.0, N), cy=rng.uniform(0.0, N))
        elif kind == "shock-vortex":
            req.update(mach=rng.uniform(1.05, 1.5))
        out.append(req)
    return out


def request_problem(req, gamma=1.4, cfl=0.5):
    """Materialise a served request (dict from served_requests) as (spec, planes)."""
    N = req["N"]
    if req["kind"] == "pulse":
        return acoustic_pulse(N, req["A"], req["b"], req["cx"], req["cy"], gamma=gamma, cfl=cfl)
    if req["kind"] == "vortex":
        return isentropic_vortex(N, gamma=gamma, cfl=cfl)
    return shock_vortex(nx=N, ny=max(2, N // 2), mach=req["mach"], gamma=gamma, cfl=cfl)
