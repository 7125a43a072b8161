"""Linear acoustics solution of the 1D acoustic-wave test: the Riemann variables
w+- = u' +- (a/rho_inf) rho' travel at +-a on the periodic domain."""
import math

import numpy as np


def acoustic_wave_exact(x, t, eps=1e-5, omega=6.0 * math.pi, gamma=1.4, rho_inf=1.1771, p_inf=101325.0):
    """(rho, u, p) at points x and time t to first order in eps."""
    a = math.sqrt(gamma * p_inf / rho_inf)

    def w(xx, sign):
        return eps * a * (np.cos(omega * xx) + sign * np.cos(2.0 * omega * xx))

    wp, wm = w(x - a * t, +1.0), w(x + a * t, -1.0)
    u = 0.5 * (wp + wm)
    rho1 = rho_inf / (2.0 * a) * (wp - wm)
    return rho_inf + rho1, u, p_inf + a * a * rho1
