// cgks_device.cuh -- device arithmetic of the compact 8th-order gas-kinetic scheme
// (Zhao, Ji, Shyy, Xu, arXiv 2001.01570) for sm_103a.  Everything is FP64.
//
// On GB300 the FP64 pipe issues about one warp instruction per 16 SM cycles, and
// only in the register-only DFMA form (RegK below), so the arithmetic is
// written in that form and to minimise the FP64 instruction count:
//   * WENO smoothness indicators as quadratic forms in first differences, with
//     the 19 pair products shared by the left and the mirrored right stencil;
//   * WENO-Z weights normalised with one reciprocal (leave-one-out products);
//   * the Euler flux and its time derivative in closed form; only the terms that
//     genuinely need velocity-space moments (the tau-terms and the half-line
//     moments of the non-equilibrium states) use them;
//   * the flux and its time derivative over [0, dt] taken from closed-form
//     window coefficients instead of differencing two time integrals;
//   * Euler time derivatives W_t, W_tt by Cauchy-Kowalevski in primitive form.
// This header holds the shared pieces and the normal reconstruction (record
// kernel); cgks_flux.cuh holds the flux kernel's arithmetic.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "cgks_erfcx_table.h"
#include "../../include/cgks.h"

namespace cgks {

// fields of a face-row record
enum { RV = 0, RN = 1, RNN = 2, RL = 3, RR = 4, RLN = 5, RRN = 6, NREC = 7 };

// boundary mapping of one index along an axis; returns the source index and
// sets the transform kind: 0 none, 1 reflect, 2 inflow, 3 outflow
__device__ __forceinline__ int map_axis(int i, int n, int bclo, int bchi, int& kind)
{
    kind = 0;
    if (i < 0) {
        const int m = -1 - i;
        if (bclo == CGKS_BC_PERIODIC) { int r = i % n; return r < 0 ? r + n : r; }
        if (bclo == CGKS_BC_REFLECT) { kind = 1; return min(m, n - 1); }
        if (bclo == CGKS_BC_INFLOW) { kind = 2; return 0; }
        kind = 3; return 0;
    }
    if (i >= n) {
        const int m = i - n;
        if (bchi == CGKS_BC_PERIODIC) return i % n;
        if (bchi == CGKS_BC_REFLECT) { kind = 1; return max(n - 1 - m, 0); }
        if (bchi == CGKS_BC_INFLOW) { kind = 2; return n - 1; }
        kind = 3; return n - 1;
    }
    return i;
}

// ------------------------------------------------------------------------
// FP64 issue forms.  A DFMA whose three operands are all registers issues at
// the full FP64 rate of this GPU (1.98 per SM and cycle); DADD, DMUL, and any
// FP64 instruction with an immediate or constant-bank operand issue at 5/6 of
// it (measured: 600 against 505 G instructions/s).  The record and flux
// kernels therefore write their adds and multiplies as register-only DFMAs --
// x + y as fma(x, 1, y), x * y as fma(x, y, -0), both exact -- and read their
// coefficients from a shared-memory table at run time, so that no compiler can
// fold 1, -0 or a coefficient back into an immediate operand.  The table is
// read through volatile loads at each use, which keeps the coefficients out of
// the register allocation.
struct RegK {
    const double* tab;   // shared-memory coefficient table (read through volatile loads)
    double one, nzero;   // 1.0 and -0.0 in registers
    __device__ __forceinline__ double k(int i) const { return ((volatile const double*)tab)[i]; }
#ifdef CGKS_OPCOUNT_HOST
    // the host operation count (csrc/opcount): each method is the operation it stands for
    double add(double x, double y) const { return x + y; }
    double sub(double x, double y) const { return x - y; }
    double mul(double x, double y) const { return x * y; }
    double kfma(int i, double x, double y) const { return fma(k(i), x, y); }
    double kmul(int i, double x) const { return k(i) * x; }
    double rcp(double x) const { return cgks_opcount_rcp(x); }
#else
    __device__ __forceinline__ double add(double x, double y) const { return fma(x, one, y); }
    __device__ __forceinline__ double sub(double x, double y) const { return fma(x, one, -y); }
    __device__ __forceinline__ double mul(double x, double y) const { return fma(x, y, nzero); }
    // c_i * x + y and c_i * x with c_i from the table
    __device__ __forceinline__ double kfma(int i, double x, double y) const { return fma(k(i), x, y); }
    __device__ __forceinline__ double kmul(int i, double x) const { return fma(k(i), x, nzero); }
    // 1/x for normal positive or negative x: the hardware approximation
    // (rcp.approx.ftz.f64, about 20 correct bits) refined by two Newton-Raphson
    // steps y <- y + y (1 - x y), each doubling the correct bits
    __device__ __forceinline__ double rcp(double x) const
    {
        double y;
        asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
        double e = fma(-x, y, one);
        y = fma(y, e, y);
        e = fma(-x, y, one);
        return fma(y, e, y);
    }
#endif
};

// Layout of the reconstruction coefficient table: one block per order (8, 6),
// each starting with 1.0 and -0.0.  Indices are offsets within a block.
enum ReconK {
    RK_ONE = 0, RK_NZERO,
    RK_LV,          // linear value: (a+d), (b+c), (A-D), (B-C)
    RK_LS = RK_LV + 4,    // linear h*slope: (c-b), (d-a), (A+D), (B+C)
    RK_LC = RK_LS + 4,    // linear h^2*curvature: ((b+c)-(a+d)), (A-D), (B-C)
    RK_E0 = RK_LC + 3,    // smoothness indicators e0..e6 (beta_k + eps)
    RK_E1 = RK_E0 + 3, RK_E2 = RK_E1 + 6, RK_E3 = RK_E2 + 6, RK_E4 = RK_E3 + 3, RK_E5 = RK_E4 + 3,
    RK_E6 = RK_E5 + 10,
    RK_Z = RK_E6 + 10,    // Z_ref: 3, -2
    RK_W = RK_Z + 2,      // linear weights d_0..d_6
    RK_Q0 = RK_W + 7, RK_Q13 = RK_Q0 + 2, RK_Q2 = RK_Q13 + 2, RK_Q4 = RK_Q2 + 3, RK_Q5 = RK_Q4 + 2,
    RK_Q6 = RK_Q5 + 4,    // candidate values (d_k folded where one candidate carries the weight)
    RK_S0 = RK_Q6 + 4, RK_S2 = RK_S0 + 2, RK_S5 = RK_S2 + 3, RK_S6 = RK_S5 + 4,   // candidate slopes
    RK_N = RK_S6 + 4
};

// ------------------------------------------------------------------------
// Sec. 3.2, Eq. (recons-8th-val): linear compact reconstruction at x_{i+1/2}
// from Q_{i-1..i+2} (a, b, c, d) and h*Q' (A, B, C, D):
//   P7       = (25 (a+d) + 185 (b+c) + 6 (A-D) + 102 (B-C)) / 420
//   h P7_x   = (270 (c-b) + 14 (d-a) - 3 (A+D) - 99 (B+C)) / 108
//   h^2 P7_xx = (b+c) - (a+d) - (A-D)/4 - 9 (B-C)/4
// ORDER = 6: the compact 6th-order variant Sec. 3.2 names, read as the degree-5
// polynomial with the four cell averages and the slopes of the two cells next
// to the face (no A, D terms):
//   P5 = ((a+d) + 29 (b+c))/60 + (B-C)/5,  h P5_x = 9 (c-b)/4 + (d-a)/36 - 2 (B+C)/3,
//   h^2 P5_xx = ((b+c) - (a+d))/4 - 3 (B-C)/2.
// The coefficients come from the table block of the grid's order.
template <int ORDER>
__device__ __forceinline__ void linear_recon_rk(const RegK& r, double a, double b, double c, double d,
                                                double A, double B, double C, double D,
                                                double& v, double& hvx, double& h2vxx)
{
    const double ad = r.add(a, d), bc = r.add(b, c), BmC = r.sub(B, C);
    const double cb = r.sub(c, b), da = r.sub(d, a), BpC = r.add(B, C), diff = r.sub(bc, ad);
    if constexpr (ORDER == 6) {
        v = r.kfma(RK_LV + 0, ad, r.kfma(RK_LV + 1, bc, r.kmul(RK_LV + 3, BmC)));
        hvx = r.kfma(RK_LS + 0, cb, r.kfma(RK_LS + 1, da, r.kmul(RK_LS + 3, BpC)));
        h2vxx = r.kfma(RK_LC + 0, diff, r.kmul(RK_LC + 2, BmC));
    } else {
        const double AmD = r.sub(A, D), ApD = r.add(A, D);
        v = r.kfma(RK_LV + 0, ad, r.kfma(RK_LV + 1, bc, r.kfma(RK_LV + 2, AmD, r.kmul(RK_LV + 3, BmC))));
        hvx = r.kfma(RK_LS + 0, cb, r.kfma(RK_LS + 1, da, r.kfma(RK_LS + 2, ApD, r.kmul(RK_LS + 3, BpC))));
        h2vxx = r.kfma(RK_LC + 1, AmD, r.kfma(RK_LC + 2, BmC, diff));
    }
}

// ------------------------------------------------------------------------
// Sec. 3.3: nonlinear compact reconstruction.  With d1 = b-a, d2 = c-b,
// d3 = d-c the candidate values q_k - b, the interface slopes h*q_k'(x_{i+1/2})
// and the smoothness indicators beta_k (beta_1 taken from the cubic on
// {Q_i-1, Q_i, Q_i+1, Q'_i-1}) follow from the sub-stencil definitions; the
// mirrored (right) stencil is d1 <-> d3, A <-> D, B <-> C with all signs flipped,
// which leaves every pair product unchanged.
struct PairProducts {
    double d11, d12, d22, d23, d33, AA, Ad1, Ad2, AB, BB, Bd1, Bd2, CC, CD, Cd2, Cd3, DD, Dd2, Dd3;
};

__device__ __forceinline__ void pair_products_rk(const RegK& r, double d1, double d2, double d3, double A, double B,
                                                 double C, double D, PairProducts& p)
{
    p.d11 = r.mul(d1, d1); p.d12 = r.mul(d1, d2); p.d22 = r.mul(d2, d2); p.d23 = r.mul(d2, d3); p.d33 = r.mul(d3, d3);
    p.AA = r.mul(A, A); p.Ad1 = r.mul(A, d1); p.Ad2 = r.mul(A, d2); p.AB = r.mul(A, B); p.BB = r.mul(B, B);
    p.Bd1 = r.mul(B, d1); p.Bd2 = r.mul(B, d2);
    p.CC = r.mul(C, C); p.CD = r.mul(C, D); p.Cd2 = r.mul(C, d2); p.Cd3 = r.mul(C, d3); p.DD = r.mul(D, D);
    p.Dd2 = r.mul(D, d2); p.Dd3 = r.mul(D, d3);
}

// Left-biased interface value and h*slope.  The argument order names the
// stencil as seen from the side being reconstructed (for the right side the
// caller passes the mirrored quantities).  Products: (x11, x12, x22, x23, x33)
// are the difference products in that orientation, (aa, ad1, ad2, ab, bb, bd1,
// bd2) the products of the two slopes on the near side, (cc, cd, cd2, cd3, dd,
// dd2, dd3) those on the far side.  The smoothness indicators of Eq.
// (smooth-indicator) are quadratic forms in these products, with the WENO
// epsilon as the first addend: e_k = beta_k + eps.  WENO-Z weights, Eq.
// (WENO-Z-w): alpha_k = d_k (e_k + Z) / e_k, normalised with one reciprocal by
// multiplying all numerators by prod_{j != k} e_j (t_k = (e_k + Z) prod_{j!=k}
// e_j); the linear weights d_k are folded into the candidate coefficients where
// a t_k multiplies a single candidate.  Coefficients: the table block of the
// grid's order (d^8 or the variant's d^6).
__device__ __forceinline__ void weno_side_rk(const RegK& r, double base, double d1, double d2, double d3,
                                             double A, double B, double C, double D,
                                             double x11, double x12, double x22, double x23, double x33,
                                             double aa, double ad1, double ad2, double ab, double bb, double bd1,
                                             double bd2, double cc, double cd, double cd2, double cd3, double dd,
                                             double dd2, double dd3, double eps, double& val, double& hslope)
{
    const double e0 = r.kfma(RK_E0 + 2, x11, r.kfma(RK_E0 + 1, ad1, r.kfma(RK_E0 + 0, aa, eps)));
    const double e1 = r.kfma(RK_E1 + 5, x22, r.kfma(RK_E1 + 4, x12, r.kfma(RK_E1 + 3, x11,
                      r.kfma(RK_E1 + 2, ad2, r.kfma(RK_E1 + 1, ad1, r.kfma(RK_E1 + 0, aa, eps))))));
    const double e2 = r.kfma(RK_E2 + 5, x33, r.kfma(RK_E2 + 4, x23, r.kfma(RK_E2 + 3, x22,
                      r.kfma(RK_E2 + 2, dd3, r.kfma(RK_E2 + 1, dd2, r.kfma(RK_E2 + 0, dd, eps))))));
    const double e3 = r.kfma(RK_E3 + 2, x22, r.kfma(RK_E3 + 1, x12, r.kfma(RK_E3 + 0, x11, eps)));
    const double e4 = r.kfma(RK_E4 + 2, x33, r.kfma(RK_E4 + 1, x23, r.kfma(RK_E4 + 0, x22, eps)));
    double e5 = r.kfma(RK_E5 + 0, aa, eps);
    e5 = r.kfma(RK_E5 + 1, ab, e5); e5 = r.kfma(RK_E5 + 2, ad1, e5); e5 = r.kfma(RK_E5 + 3, ad2, e5);
    e5 = r.kfma(RK_E5 + 4, bb, e5); e5 = r.kfma(RK_E5 + 5, bd1, e5); e5 = r.kfma(RK_E5 + 6, bd2, e5);
    e5 = r.kfma(RK_E5 + 7, x11, e5); e5 = r.kfma(RK_E5 + 8, x12, e5); e5 = r.kfma(RK_E5 + 9, x22, e5);
    double e6 = r.kfma(RK_E6 + 0, cc, eps);
    e6 = r.kfma(RK_E6 + 1, cd, e6); e6 = r.kfma(RK_E6 + 2, cd2, e6); e6 = r.kfma(RK_E6 + 3, cd3, e6);
    e6 = r.kfma(RK_E6 + 4, dd, e6); e6 = r.kfma(RK_E6 + 5, dd2, e6); e6 = r.kfma(RK_E6 + 6, dd3, e6);
    e6 = r.kfma(RK_E6 + 7, x22, e6); e6 = r.kfma(RK_E6 + 8, x23, e6); e6 = r.kfma(RK_E6 + 9, x33, e6);
    // Z_ref = |3 e0 - 2 e4 - e3| (the epsilons cancel)
    const double Z = fabs(r.kfma(RK_Z + 0, e0, r.kfma(RK_Z + 1, e4, -e3)));
    const double p01 = r.mul(e0, e1), p012 = r.mul(p01, e2), p0123 = r.mul(p012, e3), p01234 = r.mul(p0123, e4);
    const double s56 = r.mul(e5, e6), s456 = r.mul(e4, s56), s3456 = r.mul(e3, s456), s23456 = r.mul(e2, s3456);
    // t_k = (e_k + Z) L_k = P + Z L_k with L_k the product of the other six and P of all seven
    const double P = r.mul(p01234, s56);
    const double t0 = fma(Z, r.mul(e1, s23456), P);
    const double t1 = fma(Z, r.mul(e0, s23456), P);
    const double t2 = fma(Z, r.mul(p01, s3456), P);
    const double t3 = fma(Z, r.mul(p012, s456), P);
    const double t4 = fma(Z, r.mul(p0123, s56), P);
    const double t5 = fma(Z, r.mul(p01234, e6), P);
    const double t6 = fma(Z, r.mul(p01234, e5), P);
    const double n13 = r.kfma(RK_W + 1, t1, r.kmul(RK_W + 3, t3)), n4 = r.kmul(RK_W + 4, t4);
    const double den = r.kfma(RK_W + 6, t6, r.kfma(RK_W + 5, t5, r.add(r.kfma(RK_W + 2, t2, r.kfma(RK_W + 0, t0, n13)), n4)));
    const double inv = r.rcp(den);
    const double q0 = r.kfma(RK_Q0 + 0, d1, r.kmul(RK_Q0 + 1, A));
    const double q13 = r.kfma(RK_Q13 + 0, d1, r.kmul(RK_Q13 + 1, d2));
    const double q2 = r.kfma(RK_Q2 + 0, D, r.kfma(RK_Q2 + 1, d2, r.kmul(RK_Q2 + 2, d3)));
    const double q4 = r.kfma(RK_Q4 + 0, d2, r.kmul(RK_Q4 + 1, d3));
    const double q5 = r.kfma(RK_Q5 + 0, A, r.kfma(RK_Q5 + 1, B, r.kfma(RK_Q5 + 2, d1, r.kmul(RK_Q5 + 3, d2))));
    const double q6 = r.kfma(RK_Q6 + 0, d2, r.kfma(RK_Q6 + 1, d3, r.kfma(RK_Q6 + 2, C, r.kmul(RK_Q6 + 3, D))));
    const double s0 = r.kfma(RK_S0 + 0, d1, r.kmul(RK_S0 + 1, A));
    const double s2 = r.kfma(RK_S2 + 0, d2, r.kfma(RK_S2 + 1, d3, r.kmul(RK_S2 + 2, D)));
    const double s5 = r.kfma(RK_S5 + 0, A, r.kfma(RK_S5 + 1, B, r.kfma(RK_S5 + 2, d1, r.kmul(RK_S5 + 3, d2))));
    const double s6 = r.kfma(RK_S6 + 0, C, r.kfma(RK_S6 + 1, D, r.kfma(RK_S6 + 2, d2, r.kmul(RK_S6 + 3, d3))));
    const double nv = fma(t6, q6, fma(t5, q5, fma(n4, q4, fma(t2, q2, fma(n13, q13, r.mul(t0, q0))))));
    const double ns = fma(t6, s6, fma(t5, s5, fma(t2, s2, fma(r.add(n13, n4), d2, r.mul(t0, s0)))));
    val = fma(nv, inv, base);
    hslope = r.mul(ns, inv);
}

__device__ __forceinline__ void weno_pair_rk(const RegK& r, double a, double b, double c, double d, double A,
                                             double B, double C, double D, double eps, double& vl, double& sl,
                                             double& vr, double& sr)
{
    const double d1 = r.sub(b, a), d2 = r.sub(c, b), d3 = r.sub(d, c);
    PairProducts p;
    pair_products_rk(r, d1, d2, d3, A, B, C, D, p);
    weno_side_rk(r, b, d1, d2, d3, A, B, C, D, p.d11, p.d12, p.d22, p.d23, p.d33,
                 p.AA, p.Ad1, p.Ad2, p.AB, p.BB, p.Bd1, p.Bd2, p.CC, p.CD, p.Cd2, p.Cd3, p.DD, p.Dd2, p.Dd3,
                 eps, vl, sl);
    double s;
    weno_side_rk(r, c, -d3, -d2, -d1, -D, -C, -B, -A, p.d33, p.d23, p.d22, p.d12, p.d11,
                 p.DD, p.Dd3, p.Dd2, p.CD, p.CC, p.Cd3, p.Cd2, p.BB, p.AB, p.Bd2, p.Bd1, p.AA, p.Ad2, p.Ad1,
                 eps, vr, s);
    sr = -s;
}

// ------------------------------------------------------------------------
// Characteristic variables (Sec. 3.2 allows them for the reconstruction):
// eigenvectors of the normal Euler flux Jacobian in the face frame at the state
// W (rho, m_n, m_t, E); fields 0: U-c, 1: entropy, 2: shear, 3: U+c.
struct CharState { double U, V, c, H, q2, b1, b2, ic; };

__device__ __forceinline__ void char_state(const double W[4], double gamma, CharState& s)
{
    const double ir = __drcp_rn(W[0]);
    s.U = W[1] * ir;
    s.V = W[2] * ir;
    s.q2 = s.U * s.U + s.V * s.V;
    const double p = (gamma - 1.0) * (W[3] - 0.5 * W[0] * s.q2);
    s.c = sqrt(gamma * p * ir);
    s.ic = __drcp_rn(s.c);
    s.H = (W[3] + p) * ir;
    s.b2 = (gamma - 1.0) * s.ic * s.ic;
    s.b1 = 0.5 * s.b2 * s.q2;
}

// row m of the left eigenvector matrix
__device__ __forceinline__ void char_left_row(const CharState& s, int m, double l[4])
{
    if (m == 0) { l[0] = 0.5 * (s.b1 + s.U * s.ic); l[1] = -0.5 * (s.b2 * s.U + s.ic); l[2] = -0.5 * s.b2 * s.V; l[3] = 0.5 * s.b2; }
    else if (m == 1) { l[0] = 1.0 - s.b1; l[1] = s.b2 * s.U; l[2] = s.b2 * s.V; l[3] = -s.b2; }
    else if (m == 2) { l[0] = -s.V; l[1] = 0.0; l[2] = 1.0; l[3] = 0.0; }
    else { l[0] = 0.5 * (s.b1 - s.U * s.ic); l[1] = -0.5 * (s.b2 * s.U - s.ic); l[2] = -0.5 * s.b2 * s.V; l[3] = 0.5 * s.b2; }
}

// conservative = R . characteristic
__device__ __forceinline__ void char_to_cons(const CharState& s, const double w[4], double out[4])
{
    out[0] = w[0] + w[1] + w[3];
    out[1] = (s.U - s.c) * w[0] + s.U * w[1] + (s.U + s.c) * w[3];
    out[2] = s.V * (w[0] + w[1] + w[3]) + w[2];
    out[3] = (s.H - s.U * s.c) * w[0] + 0.5 * s.q2 * w[1] + s.V * w[2] + (s.H + s.U * s.c) * w[3];
}

}  // namespace cgks
