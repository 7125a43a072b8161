"""Exact solution of the 1D Riemann problem for the Euler equations (ideal gas).

Textbook construction: the star-region pressure solves f_L(p) + f_R(p) + (u_R - u_L) = 0, where
f_K is the shock (Rankine-Hugoniot) branch for p > p_K and the isentropic rarefaction branch
otherwise; the self-similar solution is then sampled at x/t.  Used only to pin the oracle on the
shock-tube problems.
"""
import math

import numpy as np


def _fk(p, rk, pk, ck, g):
    if p > pk:
        A = 2.0 / ((g + 1.0) * rk)
        B = (g - 1.0) / (g + 1.0) * pk
        s = math.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (p + B))
    r = p / pk
    f = 2.0 * ck / (g - 1.0) * (r ** ((g - 1.0) / (2.0 * g)) - 1.0)
    df = 1.0 / (rk * ck) * r ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(left, right, g=1.4):
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    p = max(1e-8, 0.5 * (pl + pr))
    for _ in range(100):
        fl, dl = _fk(p, rl, pl, cl, g)
        fr, dr = _fk(p, rr, pr, cr, g)
        dp = (fl + fr + ur - ul) / (dl + dr)
        pn = max(1e-10, p - dp)
        if abs(pn - p) < 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fk(p, rl, pl, cl, g)
    fr, _ = _fk(p, rr, pr, cr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(left, right, s, g=1.4):
    """Primitive (rho, u, p) at similarity coordinate s = (x - x0)/t (array)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    ps, us = star_state(left, right, g)
    s = np.asarray(s, dtype=float)
    rho, u, p = np.empty_like(s), np.empty_like(s), np.empty_like(s)
    gm = (g - 1.0) / (g + 1.0)
    for idx, x in np.ndenumerate(s):
        if x <= us:   # left of contact
            if ps > pl:   # left shock
                rs = rl * (ps / pl + gm) / (gm * ps / pl + 1.0)
                sl = ul - cl * math.sqrt((g + 1.0) / (2.0 * g) * ps / pl + (g - 1.0) / (2.0 * g))
                val = (rl, ul, pl) if x <= sl else (rs, us, ps)
            else:         # left rarefaction
                rs = rl * (ps / pl) ** (1.0 / g)
                cs = cl * (ps / pl) ** ((g - 1.0) / (2.0 * g))
                sh, st = ul - cl, us - cs
                if x <= sh:
                    val = (rl, ul, pl)
                elif x >= st:
                    val = (rs, us, ps)
                else:
                    uu = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul + x)
                    c = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * (ul - x))
                    rr_ = rl * (c / cl) ** (2.0 / (g - 1.0))
                    val = (rr_, uu, pl * (c / cl) ** (2.0 * g / (g - 1.0)))
        else:
            if ps > pr:   # right shock
                rs = rr * (ps / pr + gm) / (gm * ps / pr + 1.0)
                sr = ur + cr * math.sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g))
                val = (rr, ur, pr) if x >= sr else (rs, us, ps)
            else:
                rs = rr * (ps / pr) ** (1.0 / g)
                cs = cr * (ps / pr) ** ((g - 1.0) / (2.0 * g))
                sh, st = ur + cr, us + cs
                if x >= sh:
                    val = (rr, ur, pr)
                elif x <= st:
                    val = (rs, us, ps)
                else:
                    uu = 2.0 / (g + 1.0) * (-cr + 0.5 * (g - 1.0) * ur + x)
                    c = 2.0 / (g + 1.0) * (cr - 0.5 * (g - 1.0) * (ur - x))
                    rr_ = rr * (c / cr) ** (2.0 / (g - 1.0))
                    val = (rr_, uu, pr * (c / cr) ** (2.0 * g / (g - 1.0)))
        rho[idx], u[idx], p[idx] = val
    return rho, u, p


def cell_average_density(left, right, t, n, x0=0.5, g=1.4, sub=64):
    """Cell averages of the exact density on n cells of [0, 1] at time t (midpoint sub-sampling)."""
    dx = 1.0 / n
    xs = (np.arange(n * sub) + 0.5) * (dx / sub)
    rho, _, _ = sample(left, right, (xs - x0) / t, g)
    return rho.reshape(n, sub).mean(axis=1)
