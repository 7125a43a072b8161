"""Generate cgks_erfcx_table.h: piecewise polynomials of erfcx(t) = exp(t^2) erfc(t) on [0, 28).

Method: the interval [0, 28) is cut into 112 pieces of width 1/4; on each piece erfcx is
approximated by its degree-DEG polynomial in z = t - centre, obtained by least squares on
Chebyshev nodes from values computed with mpmath at 40 significant digits.  The kernels use it as
erfc(t) = exp(-t^2) * erfcx(t) with the exp(-t^2) the half-line Maxwellian moments need anyway;
beyond t = 28, exp(-t^2) underflows and erfc(t) is 0 in double precision.

Run: python paper_2001_01570_gb300/csrc/gen_erfcx_table.py  (needs mpmath; writes the header and
prints the worst relative error of the table against mpmath on a dense sample).
"""
import os

import mpmath as mp
import numpy as np

mp.mp.dps = 40
WIDTH = 0.25
NPIECE = 112
DEG = 11
HERE = os.path.dirname(os.path.abspath(__file__))


def erfcx(t):
    return mp.exp(t * t) * mp.erfc(t)


def fit_piece(k):
    c = (k + 0.5) * WIDTH
    h = 0.5 * WIDTH
    n = 4 * DEG
    nodes = [mp.mpf(c) + mp.mpf(h) * mp.cos(mp.pi * (2 * j + 1) / (2 * n)) for j in range(n)]
    # least squares in extended precision: normal equations of the monomial basis in z
    A = mp.matrix(n, DEG + 1)
    b = mp.matrix(n, 1)
    for i, x in enumerate(nodes):
        z = x - c
        fx = erfcx(x)
        for m in range(DEG + 1):
            A[i, m] = z ** m / fx          # relative-error weighting
        b[i] = 1
    coef = mp.lu_solve(A.T * A, A.T * b)
    return c, [coef[m] for m in range(DEG + 1)]


def main():
    pieces = [fit_piece(k) for k in range(NPIECE)]
    worst = 0.0
    for k, (c, co) in enumerate(pieces):
        for j in range(41):
            t = k * WIDTH + WIDTH * j / 40.0
            z = t - c
            approx = 0.0
            for m in range(DEG, -1, -1):
                approx = approx * z + float(co[m])
            ref = erfcx(mp.mpf(t))
            worst = max(worst, abs(float((approx - ref) / ref)))
    lines = ["// Generated by gen_erfcx_table.py: erfcx(t) = exp(t^2) erfc(t) on [0, 28) in 112 pieces of",
             f"// width 1/4, degree-{DEG} polynomials in z = t - (k + 1/2)/4 (highest degree first).",
             f"// Worst relative error against 40-digit mpmath on a dense sample: {worst:.2e}.",
             "#pragma once",
             f"#define CGKS_ERFCX_PIECES {NPIECE}",
             f"#define CGKS_ERFCX_DEG {DEG}",
             f"__device__ const double cgks_erfcx_coef[{NPIECE}][{DEG + 1}] = {{"]
    for c, co in pieces:
        lines.append("    {" + ", ".join(repr(float(co[m])) for m in range(DEG, -1, -1)) + "},")
    lines.append("};")
    with open(os.path.join(HERE, "cgks_erfcx_table.h"), "w") as f:
        f.write("\n".join(lines) + "\n")
    print(f"worst relative error {worst:.3e}")


if __name__ == "__main__":
    main()
