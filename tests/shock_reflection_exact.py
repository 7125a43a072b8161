"""Exact steady states of the regular shock reflection: oblique-shock (Rankine-Hugoniot) relations
for the incident shock (given angle) and for the reflected shock, which turns the flow back to
parallel with the wall (weak solution of the theta-beta-Mach relation)."""
import math

from scipy.optimize import brentq


def oblique(rho, u, v, p, beta, gamma):
    """State behind a shock at angle beta (radians) to the flow direction of (rho, u, v, p)."""
    c = math.sqrt(gamma * p / rho)
    mn = math.hypot(u, v) / c * math.sin(beta)
    rr = (gamma + 1.0) * mn * mn / ((gamma - 1.0) * mn * mn + 2.0)
    pr = 1.0 + 2.0 * gamma / (gamma + 1.0) * (mn * mn - 1.0)
    return rho * rr, p * pr


def regions(mach=2.9, angle_deg=29.0, gamma=1.4):
    """(rho, p) of the free stream, behind the incident shock, behind the reflected shock."""
    g = gamma
    r1, p1 = 1.0, 1.0 / g
    b1 = math.radians(angle_deg)
    r2, p2 = oblique(r1, mach, 0.0, p1, b1, g)
    # deflection across the incident shock from the theta-beta-Mach relation
    m1 = mach
    th = math.atan(2.0 / math.tan(b1) * (m1 * m1 * math.sin(b1) ** 2 - 1.0)
                   / (m1 * m1 * (g + math.cos(2.0 * b1)) + 2.0))
    # speed behind the incident shock: tangential component kept, normal one divided by r2
    ut, un = m1 * math.cos(b1), m1 * math.sin(b1) / r2
    q2 = math.hypot(ut, un)
    m2 = q2 / math.sqrt(g * p2 / r2)

    def turn(b):
        return math.tan(th) - 2.0 / math.tan(b) * (m2 * m2 * math.sin(b) ** 2 - 1.0) / (
            m2 * m2 * (g + math.cos(2.0 * b)) + 2.0)

    b2 = brentq(turn, math.asin(1.0 / m2) + 1e-12, math.radians(60.0))
    r3, p3 = oblique(r2, q2, 0.0, p2, b2, g)
    return (r1, p1), (r2, p2), (r3, p3)
