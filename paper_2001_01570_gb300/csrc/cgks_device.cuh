// cgks_device.cuh -- device arithmetic of the compact 8th-order gas-kinetic scheme
// (Zhao, Ji, Shyy, Xu, arXiv 2001.01570) for sm_103a.  Everything is FP64.
//
// On GB300 the FP64 pipe issues about one warp instruction per 16 SM cycles, so
// the code below is written to minimise FP64 instruction count:
//   * WENO smoothness indicators as quadratic forms in first differences, with
//     the 19 pair products shared by the left and the mirrored right stencil;
//   * WENO-Z weights normalised with one reciprocal (leave-one-out products);
//   * the Euler flux and its time derivative in closed form; only the terms that
//     genuinely need velocity-space moments (the tau-terms and the half-line
//     moments of the non-equilibrium states) use them;
//   * the flux and its time derivative over [0, dt] taken from closed-form
//     window coefficients instead of differencing two time integrals;
//   * Euler time derivatives W_t, W_tt by Cauchy-Kowalevski in primitive form.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "cgks_erfcx_table.h"
#include "../../include/cgks.h"

namespace cgks {

// erfc(t) for t >= 0 from e = exp(-t^2): e * erfcx(t), erfcx from the piecewise
// polynomials of cgks_erfcx_table.h (relative error ~2e-16); 11 FMAs instead
// of a full erfc evaluation, since the half-line moments need e anyway.  Past
// t = 27.3 e underflows to 0; a NaN t selects the last piece and stays NaN.
__device__ __forceinline__ double erfc_scaled(double t, double e)
{
    const int k = (int)(fmin(t, 27.9) * 4.0);
    const double* c = cgks_erfcx_coef[k];
    const double z = t - (0.25 * (double)k + 0.125);
    double r = c[0];
#pragma unroll
    for (int m = 1; m <= CGKS_ERFCX_DEG; ++m) r = fma(r, z, c[m]);
    return e * r;
}

// the two lowest half-line u-moments of a Maxwellian with mean U and
// sqrt(lambda) = sq: <u^0> = erfc(-+ s)/2, <u^1> = U <u^0> +- e^{-s^2}/(2 sqrt(pi lambda)),
// s = U sqrt(lambda); side = +1 for u > 0, -1 for u < 0
__device__ __forceinline__ void half_moments01(double U, double sq, double inv_sq, int side, double& m0, double& m1)
{
    const double s = U * sq;
    const double e = exp(-s * s);
    const double hE = 0.5 * erfc_scaled(fabs(s), e);          // erfc(|s|)/2
    // side +1: erfc(-s)/2 = 1 - erfc(s)/2 for s >= 0, erfc(|s|)/2 for s < 0; side -1 mirrored
    const bool pos = (side > 0) ? (s >= 0.0) : (s < 0.0);
    m0 = pos ? 1.0 - hE : hE;
    m1 = U * m0 + (double)side * e * inv_sq * 0.28209479177387814;   // 1/(2 sqrt(pi))
}

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
// Sec. 3.2, Eq. (recons-8th-val): linear compact reconstruction at x_{i+1/2}
// from Q_{i-1..i+2} (a, b, c, d) and h*Q' (A, B, C, D).
// ORDER = 6: the compact 6th-order variant Sec. 3.2 names, read as the
// degree-5 polynomial with the four cell averages and the cell-averaged
// slopes of the two cells next to the face (the outer slopes A, D unused).
template <int ORDER>
__device__ __forceinline__ void linear_recon(double a, double b, double c, double d,
                                             double A, double B, double C, double D,
                                             double& v, double& hvx, double& h2vxx)
{
    if constexpr (ORDER == 6) {
        v = ((a + d) + 29.0 * (b + c)) * (1.0 / 60.0) + 0.2 * (B - C);
        hvx = (d - a) * (1.0 / 36.0) + 2.25 * (c - b) - (2.0 / 3.0) * (B + C);
        h2vxx = 0.25 * ((b + c) - (a + d)) - 1.5 * (B - C);
    } else {
        v = (25.0 * (a + d) + 185.0 * (b + c) + 6.0 * (A - D) + 102.0 * (B - C)) * (1.0 / 420.0);
        hvx = (270.0 * (c - b) + 14.0 * (d - a) - 3.0 * (A + D) - 99.0 * (B + C)) * (1.0 / 108.0);
        h2vxx = (4.0 * ((b + c) - (a + d)) - (A - D) - 9.0 * (B - C)) * 0.25;
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

__device__ __forceinline__ void pair_products(double d1, double d2, double d3, double A, double B, double C,
                                              double D, PairProducts& p)
{
    p.d11 = d1 * d1; p.d12 = d1 * d2; p.d22 = d2 * d2; p.d23 = d2 * d3; p.d33 = d3 * d3;
    p.AA = A * A; p.Ad1 = A * d1; p.Ad2 = A * d2; p.AB = A * B; p.BB = B * B; p.Bd1 = B * d1; p.Bd2 = B * d2;
    p.CC = C * C; p.CD = C * D; p.Cd2 = C * d2; p.Cd3 = C * d3; p.DD = D * D; p.Dd2 = D * d2; p.Dd3 = D * d3;
}

// left-biased interface value and h*slope with the linear weights of the given
// order (ORDER = 6: the weights that recombine the candidates into the degree-5
// interface value, d = (3, 5, 8, 7, 7, 20, 20)/70).  The argument order names the
// stencil as seen from the side being reconstructed (for the right side the
// caller passes the mirrored quantities).  Products: (x11, x12, x22, x23, x33)
// are the difference products in that orientation, (aa, ad1, ad2, ab, bb, bd1,
// bd2) the products of the two slopes on the near side, (cc, cd, cd2, cd3, dd,
// dd2, dd3) those on the far side.
template <int ORDER>
__device__ __forceinline__ void weno_side(double base, double d1, double d2, double d3,
                                          double A, double B, double C, double D,
                                          double x11, double x12, double x22, double x23, double x33,
                                          double aa, double ad1, double ad2, double ab, double bb, double bd1, double bd2,
                                          double cc, double cd, double cd2, double cd3, double dd, double dd2, double dd3,
                                          double eps, double& val, double& hslope)
{
    // smoothness indicators, Eq. (smooth-indicator), with the WENO epsilon
    // already added: e_k = beta_k + eps (one multiply-add chain each)
    const double e0 = eps + (16.0 / 3.0) * aa - (38.0 / 3.0) * ad1 + (25.0 / 3.0) * x11;
    const double e1 = eps + (801.0 / 80.0) * aa - (2443.0 / 80.0) * ad1 + (761.0 / 80.0) * ad2
                      + (23627.0 / 960.0) * x11 - (7769.0 / 480.0) * x12 + (3443.0 / 960.0) * x22;
    const double e2 = eps + (1641.0 / 80.0) * dd + (2401.0 / 80.0) * dd2 - (5523.0 / 80.0) * dd3
                      + (12683.0 / 960.0) * x22 - (25169.0 / 480.0) * x23 + (56387.0 / 960.0) * x33;
    const double e3 = eps + (4.0 / 3.0) * x11 - (5.0 / 3.0) * x12 + (4.0 / 3.0) * x22;
    const double e4 = eps + (10.0 / 3.0) * x22 - (11.0 / 3.0) * x23 + (4.0 / 3.0) * x33;
    const double e5 = eps + (4405.0 / 28.0) * aa + (4405.0 / 7.0) * ab - (110433.0 / 140.0) * ad1
                      - (21717.0 / 140.0) * ad2 + (93707.0 / 140.0) * bb - (226333.0 / 140.0) * bd1
                      - (48901.0 / 140.0) * bd2 + (209917.0 / 210.0) * x11 + (17063.0 / 42.0) * x12
                      + (5153.0 / 105.0) * x22;
    const double e6 = eps + (265067.0 / 140.0) * cc + (11104.0 / 7.0) * cd - (160551.0 / 140.0) * cd2
                      - (592783.0 / 140.0) * cd3 + (9529.0 / 28.0) * dd - (65327.0 / 140.0) * dd2
                      - (252323.0 / 140.0) * dd3 + (38131.0 / 210.0) * x22 + (52763.0 / 42.0) * x23
                      + (251276.0 / 105.0) * x33;
    // global reference Z_ref, Eq. (tau): |3 beta_0 - 2 beta_4 - beta_3| (the epsilons cancel)
    const double Z = fabs(3.0 * e0 - 2.0 * e4 - e3);
    // WENO-Z: alpha_k = d_k (e_k + Z) / e_k; normalised with one reciprocal by
    // multiplying the numerators by prod_{j != k} e_j: t_k = (e_k + Z) prod_{j != k} e_j,
    // alpha_k proportional to d_k t_k.  The linear weights d_k are folded into the
    // candidate coefficients below where a t_k multiplies a single candidate.
    constexpr bool six = ORDER == 6;
    constexpr double d0 = six ? 3.0 / 70.0 : 3.0 / 98.0, d1w = six ? 5.0 / 70.0 : 5.0 / 98.0;
    constexpr double d2w = six ? 8.0 / 70.0 : 4.0 / 49.0, d3w = six ? 7.0 / 70.0 : 7.0 / 98.0;
    constexpr double d4w = six ? 7.0 / 70.0 : 7.0 / 98.0;
    constexpr double d5 = six ? 20.0 / 70.0 : 17.0 / 49.0, d6 = six ? 20.0 / 70.0 : 17.0 / 49.0;
    const double p01 = e0 * e1, p012 = p01 * e2, p0123 = p012 * e3, p01234 = p0123 * e4;
    const double s56 = e5 * e6, s456 = e4 * s56, s3456 = e3 * s456, s23456 = e2 * s3456;
    const double t0 = (e0 + Z) * (e1 * s23456);
    const double t1 = (e1 + Z) * (e0 * s23456);
    const double t2 = (e2 + Z) * (p01 * s3456);
    const double t3 = (e3 + Z) * (p012 * s456);
    const double t4 = (e4 + Z) * (p0123 * s56);
    const double t5 = (e5 + Z) * (p01234 * e6);
    const double t6 = (e6 + Z) * (p01234 * e5);
    const double n13 = d1w * t1 + d3w * t3, n4 = d4w * t4;
    const double inv = __drcp_rn(d0 * t0 + n13 + d2w * t2 + n4 + d5 * t5 + d6 * t6);
    // candidate values minus Q_i, Eq. (sub-stencil) (q0, q2, q5, q6 times their d_k)
    const double q0 = (d0 * 7.0 / 6.0) * d1 - (d0 * 2.0 / 3.0) * A;
    const double q13 = (1.0 / 6.0) * d1 + (1.0 / 3.0) * d2;
    const double q2 = (d2w * 0.25) * D + (d2w * 19.0 / 24.0) * d2 - (d2w * 13.0 / 24.0) * d3;
    const double q4 = (2.0 / 3.0) * d2 - (1.0 / 6.0) * d3;
    const double q5 = (d5 * 0.1) * A + (d5 * 0.7) * B - (d5 / 3.0) * d1 + (d5 / 30.0) * d2;
    const double q6 = (d6 * 29.0 / 30.0) * d2 + (d6 / 3.0) * d3 - (d6 * 0.7) * C - (d6 * 0.1) * D;
    // candidate slopes h q_k'(x_{i+1/2}) (s0, s2, s5, s6 times their d_k)
    const double s0 = (d0 * 3.0) * d1 - (d0 * 2.0) * A;
    const double s2 = (d2w * 0.875) * d2 + (d2w * 0.375) * d3 - (d2w * 0.25) * D;
    const double s5 = (d5 * 0.5) * A + (d5 * 1.5) * B - (d5 * 1.5) * d1 + (d5 * 0.5) * d2;
    const double s6 = (d6 * 1.5) * C + (d6 * 0.5) * D + (d6 * 0.5) * d2 - (d6 * 1.5) * d3;
    const double nv = t0 * q0 + n13 * q13 + t2 * q2 + n4 * q4 + t5 * q5 + t6 * q6;
    const double ns = t0 * s0 + (n13 + n4) * d2 + t2 * s2 + t5 * s5 + t6 * s6;
    val = base + nv * inv;
    hslope = ns * inv;
}

// left and right non-equilibrium values and h*slopes at x_{i+1/2}
template <int ORDER>
__device__ __forceinline__ void weno_pair(double a, double b, double c, double d, double A, double B, double C,
                                          double D, double eps, double& vl, double& sl, double& vr, double& sr)
{
    const double d1 = b - a, d2 = c - b, d3 = d - c;
    PairProducts p;
    pair_products(d1, d2, d3, A, B, C, D, p);
    weno_side<ORDER>(b, d1, d2, d3, A, B, C, D, p.d11, p.d12, p.d22, p.d23, p.d33,
              p.AA, p.Ad1, p.Ad2, p.AB, p.BB, p.Bd1, p.Bd2, p.CC, p.CD, p.Cd2, p.Cd3, p.DD, p.Dd2, p.Dd3,
              eps, vl, sl);
    // mirrored stencil: (d1,d2,d3) -> -(d3,d2,d1), (A,B,C,D) -> -(D,C,B,A); products unchanged
    double s;
    weno_side<ORDER>(c, -d3, -d2, -d1, -D, -C, -B, -A, p.d33, p.d23, p.d22, p.d12, p.d11,
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

// ------------------------------------------------------------------------
// Nonlinear point values along a face (2D): WENO-Z over the line averages of
// neighbouring face rows at the Gauss points eta = +-1/(2 sqrt 3) of the face
// segment (the linear tangential fits turn negative across a discontinuity
// that runs through the faces).
//
// Five means v_{-2..2}: three quadratic candidates on consecutive segments.  At
// a Gauss point each one is v_0 + (eta/2) D_k with
//   D_0 = 3 v_0 - 4 v_-1 + v_-2,  D_1 = v_1 - v_-1,  D_2 = 4 v_1 - v_2 - 3 v_0;
// linear weights (d_lo, 11/18, d_hi) at eta > 0 and (d_hi, 11/18, d_lo) at
// eta < 0, d_lo,hi = 7/36 -+ sqrt(3)/1080, make the combination the quartic
// through the five means; beta_k = 13/12 (second difference)^2 + D_k^2 / 4 is
// the indicator of candidate k over the central segment; Z = |beta_0 - beta_2|;
// alpha_k = d_k (e_k + Z) / e_k with e_k = beta_k + eps, normalised with one
// reciprocal through the common denominator e_0 e_1 e_2.
// Both Gauss points are evaluated at once (eta = -g and +g): the indicators
// and the unnormalised weights are shared, only the linear weights and the
// final normalisation differ.
__device__ __forceinline__ void tang_weno5_pair(double vmm, double vm, double v0, double vp, double vpp, double g,
                                                double eps, double& at_minus, double& at_plus)
{
    const double D0 = (3.0 * v0 - 4.0 * vm) + vmm;
    const double D1 = vp - vm;
    const double D2 = (4.0 * vp - vpp) - 3.0 * v0;
    const double s0 = (vmm - 2.0 * vm) + v0, s1 = (vm - 2.0 * v0) + vp, s2 = (v0 - 2.0 * vp) + vpp;
    const double e0 = eps + ((13.0 / 12.0) * s0) * s0 + (0.25 * D0) * D0;
    const double e1 = eps + ((13.0 / 12.0) * s1) * s1 + (0.25 * D1) * D1;
    const double e2 = eps + ((13.0 / 12.0) * s2) * s2 + (0.25 * D2) * D2;
    const double Z = fabs(e0 - e2);
    constexpr double d_lo = 7.0 / 36.0 - 1.7320508075688772 / 1080.0;
    constexpr double d_hi = 7.0 / 36.0 + 1.7320508075688772 / 1080.0;
    const double P0 = (e0 + Z) * (e1 * e2), P1 = (11.0 / 18.0) * (e1 + Z) * (e0 * e2), P2 = (e2 + Z) * (e0 * e1);
    const double Q0 = P0 * D0, Q1 = P1 * D1, Q2 = P2 * D2;
    // eta > 0: weights (d_lo, 11/18, d_hi); eta < 0: (d_hi, 11/18, d_lo)
    at_plus = v0 + (0.5 * g) * (((d_lo * Q0 + Q1) + d_hi * Q2) * __drcp_rn((d_lo * P0 + P1) + d_hi * P2));
    at_minus = v0 - (0.5 * g) * (((d_hi * Q0 + Q1) + d_lo * Q2) * __drcp_rn((d_hi * P0 + P1) + d_lo * P2));
}

// Three means v_{-1..1}: two linear candidates with slopes v_0 - v_-1 and
// v_1 - v_0, linear weights 1/2 at both Gauss points (the quadratic through the
// three means has no eta^2 - 1/12 term there), beta_k = slope_k^2, Z = |beta_0 -
// beta_1|.  The weights do not depend on eta: returns the nonlinear slope per
// unit eta; the point value is v_0 + eta * slope.
__device__ __forceinline__ double tang_weno3_slope(double vm, double v0, double vp, double eps)
{
    const double dm = v0 - vm, dp = vp - v0;
    const double e0 = eps + dm * dm, e1 = eps + dp * dp;
    const double Z = fabs(e0 - e1);
    const double n0 = (e0 + Z) * e1, n1 = (e1 + Z) * e0;
    return (n0 * dm + n1 * dp) * __drcp_rn(n0 + n1);
}

// ------------------------------------------------------------------------
// Sec. 2.1: Maxwellian velocity moments.  theta = p/rho = 1/(2 lambda).
struct Moments {
    double u[7];     // <u^n>, n = 0..6 (whole line or half line)
    double v[6];     // <v^n>, n = 0..5 (whole line)
    double x1, x2;   // <xi^2>, <xi^4>
};

__device__ __forceinline__ void moments_tail(Moments& m, double U, double V, double theta, double K)
{
    const double t2 = 2.0 * theta, t3 = 3.0 * theta, t4 = 4.0 * theta, t5 = 5.0 * theta;
    m.u[2] = U * m.u[1] + theta * m.u[0];
    m.u[3] = U * m.u[2] + t2 * m.u[1];
    m.u[4] = U * m.u[3] + t3 * m.u[2];
    m.u[5] = U * m.u[4] + t4 * m.u[3];
    m.u[6] = U * m.u[5] + t5 * m.u[4];
    m.v[0] = 1.0;
    m.v[1] = V;
    m.v[2] = V * V + theta;
    m.v[3] = V * m.v[2] + t2 * V;
    m.v[4] = V * m.v[3] + t3 * m.v[2];
    m.v[5] = V * m.v[4] + t4 * m.v[3];
    m.x1 = K * theta;
    m.x2 = K * (K + 2.0) * theta * theta;
}

// <u^A v^B psi>
template <int A, int B>
__device__ __forceinline__ void psi_uv(const Moments& m, double o[4])
{
    const double base = m.u[A] * m.v[B];
    o[0] = base;
    o[1] = m.u[A + 1] * m.v[B];
    o[2] = m.u[A] * m.v[B + 1];
    o[3] = 0.5 * (m.u[A + 2] * m.v[B] + m.u[A] * m.v[B + 2] + base * m.x1);
}

// <psi u^A (u (a1 . psi) + v (a2 . psi))> for a Maxwellian, with a . psi =
// a0 + a1 u + a2 v + a3 (u^2 + v^2 + xi^2)/2: the slope terms of the half-line
// moments (A = 1: the flux part, A = 0: the interface-state part).  The
// polynomial in the bracket, times u^A, is grouped by powers of v,
//   v^0: a1_0 u + a1_1 u^2 + h1 u^3  (+ h1 u xi^2),  v^1: a2_0 + c12 u + h2 u^2  (+ h2 xi^2),
//   v^2: a2_2 + h1 u,                v^3: h2,
// (h = a_3/2, c12 = a1_2 + a2_1), so each psi component is a short sum of
// products of the factorised u-, v- and xi-moments.
template <int A>
__device__ __forceinline__ void q_moments(const Moments& m, const double a1[4], const double a2[4], double o[4])
{
    const double h1 = 0.5 * a1[3], h2 = 0.5 * a2[3], c12 = a1[2] + a2[1];
    // sums over u for the v^j groups at u-shift s (S_j[s]) and the xi^2 parts (Z_j[s])
    double S0[3], S1[3], S2[3], S3[3], Z0[3], Z1[3];
#pragma unroll
    for (int s2 = 0; s2 < 3; ++s2) {
        S0[s2] = a1[0] * m.u[A + 1 + s2] + a1[1] * m.u[A + 2 + s2] + h1 * m.u[A + 3 + s2];
        S1[s2] = a2[0] * m.u[A + s2] + c12 * m.u[A + 1 + s2] + h2 * m.u[A + 2 + s2];
        S2[s2] = a2[2] * m.u[A + s2] + h1 * m.u[A + 1 + s2];
        S3[s2] = h2 * m.u[A + s2];
        Z0[s2] = h1 * m.u[A + 1 + s2];
        Z1[s2] = h2 * m.u[A + s2];
    }
    const double x1 = m.x1, x2 = m.x2;   // m.v[0] = 1
    auto sum = [&](int s2, int sh) {     // sum_j v[j+sh] S_j[s2] + x1 (v[sh] Z0[s2] + v[sh+1] Z1[s2])
        return m.v[sh] * S0[s2] + m.v[sh + 1] * S1[s2] + m.v[sh + 2] * S2[s2] + m.v[sh + 3] * S3[s2]
               + x1 * (m.v[sh] * Z0[s2] + m.v[sh + 1] * Z1[s2]);
    };
    const double plain0 = S0[0] + m.v[1] * S1[0] + m.v[2] * S2[0] + m.v[3] * S3[0];
    const double xi0 = Z0[0] + m.v[1] * Z1[0];
    o[0] = plain0 + x1 * xi0;
    o[1] = sum(1, 0);
    o[2] = sum(0, 1);
    o[3] = 0.5 * (sum(2, 0) + sum(0, 2) + x1 * plain0 + x2 * xi0);
}

// micro-slope coefficients a with <psi psi^T> a = b for a Maxwellian
// (closed form of the 4x4 moment system)
struct SlopeCtx { double U, V, Bm, inv_theta, c4; };

__device__ __forceinline__ void slope_ctx(double U, double V, double theta, double inv_theta, double K,
                                          double inv_K2, SlopeCtx& s)
{
    s.U = U; s.V = V;
    s.Bm = U * U + V * V + (K + 2.0) * theta;
    s.inv_theta = inv_theta;
    s.c4 = inv_theta * inv_theta * inv_K2;
}

__device__ __forceinline__ void micro_slope(const SlopeCtx& s, const double b[4], double a[4])
{
    const double R4 = 2.0 * b[3] - s.Bm * b[0];
    const double R3 = b[2] - s.V * b[0];
    const double R2 = b[1] - s.U * b[0];
    a[3] = s.c4 * (R4 - 2.0 * (s.U * R2 + s.V * R3));
    a[2] = R3 * s.inv_theta - s.V * a[3];
    a[1] = R2 * s.inv_theta - s.U * a[3];
    a[0] = b[0] - s.U * a[1] - s.V * a[2] - 0.5 * a[3] * s.Bm;
}

// ------------------------------------------------------------------------
// Euler time derivatives by Cauchy-Kowalevski in primitive variables.
// Inputs: conservative W and its x (normal), y (tangential) derivatives up to
// second order.  Outputs conservative W_t, W_tt and the flux time derivative
// F_t of the normal Euler flux.
// TNS is rho <(a_n u + a_t v + A) u psi> of the equilibrium state, i.e. the
// Chapman-Enskog Navier-Stokes flux of the BGK model per unit collision time
// (mu = tau p, bulk part 2/(K+2), heat conduction (K+4)/2 tau p grad(p/rho)).
struct EulerTD { double Wt[4], Wtt[4], Ft[4], F[4], TNS[4]; };

__device__ __forceinline__ void euler_time_derivs(const double W[4], const double Wx[4], const double Wy[4],
                                                  const double Wxx[4], const double Wxy[4], const double Wyy[4],
                                                  double gamma, double inv_gm1, double K2inv2, double Kheat,
                                                  double ir, double U, double V, double p, EulerTD& o)
{
    const double gm1 = gamma - 1.0;
    const double rho = W[0], m = W[1], E = W[3];
    // primitive first derivatives
    const double rx = Wx[0], ry = Wy[0];
    const double Ux = (Wx[1] - U * rx) * ir, Uy = (Wy[1] - U * ry) * ir;
    const double Vx = (Wx[2] - V * rx) * ir, Vy = (Wy[2] - V * ry) * ir;
    // kinetic energy KE = rho q^2 / 2: KE_x = u . m_x - rho_x q^2/2,
    // KE_xx = rho |u_x|^2 + u . m_xx - rho_xx q^2/2, KE_xy = rho u_x . u_y + u . m_xy - rho_xy q^2/2
    const double hq2 = 0.5 * (U * U + V * V);
    const double KEx = U * Wx[1] + V * Wx[2] - hq2 * rx;
    const double KEy = U * Wy[1] + V * Wy[2] - hq2 * ry;
    const double px = gm1 * (Wx[3] - KEx), py = gm1 * (Wy[3] - KEy);
    // primitive second derivatives
    const double rxx = Wxx[0], rxy = Wxy[0], ryy = Wyy[0];
    const double Uxx = (Wxx[1] - 2.0 * Ux * rx - U * rxx) * ir;
    const double Uxy = (Wxy[1] - Ux * ry - Uy * rx - U * rxy) * ir;
    const double Uyy = (Wyy[1] - 2.0 * Uy * ry - U * ryy) * ir;
    const double Vxx = (Wxx[2] - 2.0 * Vx * rx - V * rxx) * ir;
    const double Vxy = (Wxy[2] - Vx * ry - Vy * rx - V * rxy) * ir;
    const double Vyy = (Wyy[2] - 2.0 * Vy * ry - V * ryy) * ir;
    const double KExx = rho * (Ux * Ux + Vx * Vx) + U * Wxx[1] + V * Wxx[2] - hq2 * rxx;
    const double KExy = rho * (Ux * Uy + Vx * Vy) + U * Wxy[1] + V * Wxy[2] - hq2 * rxy;
    const double KEyy = rho * (Uy * Uy + Vy * Vy) + U * Wyy[1] + V * Wyy[2] - hq2 * ryy;
    const double pxx = gm1 * (Wxx[3] - KExx), pxy = gm1 * (Wxy[3] - KExy), pyy = gm1 * (Wyy[3] - KEyy);
    // first time derivatives
    const double Dv = Ux + Vy;
    const double rt = -(U * rx + V * ry + rho * Dv);
    const double Ut = -(U * Ux + V * Uy + px * ir);
    const double Vt = -(U * Vx + V * Vy + py * ir);
    const double pt = -(U * px + V * py + gamma * p * Dv);
    // mixed derivatives d/dx, d/dy of the first time derivatives
    const double Dx = Uxx + Vxy, Dy = Uxy + Vyy;
    const double rxt = -(Ux * rx + U * rxx + Vx * ry + V * rxy + rx * Dv + rho * Dx);
    const double ryt = -(Uy * rx + U * rxy + Vy * ry + V * ryy + ry * Dv + rho * Dy);
    const double Uxt = -(Ux * Ux + U * Uxx + Vx * Uy + V * Uxy + (pxx - px * rx * ir) * ir);
    const double Vyt = -(Uy * Vx + U * Vxy + Vy * Vy + V * Vyy + (pyy - py * ry * ir) * ir);
    const double Uyt = -(Uy * Ux + U * Uxy + Vy * Uy + V * Uyy + (pxy - px * ry * ir) * ir);
    const double Vxt = -(Ux * Vx + U * Vxx + Vx * Vy + V * Vxy + (pxy - py * rx * ir) * ir);
    const double pxt = -(Ux * px + U * pxx + Vx * py + V * pxy + gamma * (px * Dv + p * Dx));
    const double pyt = -(Uy * px + U * pxy + Vy * py + V * pyy + gamma * (py * Dv + p * Dy));
    // second time derivatives
    const double Dt = Uxt + Vyt;
    const double rtt = -(Ut * rx + U * rxt + Vt * ry + V * ryt + rt * Dv + rho * Dt);
    const double Utt = -(Ut * Ux + U * Uxt + Vt * Uy + V * Uyt + (pxt - px * rt * ir) * ir);
    const double Vtt = -(Ut * Vx + U * Vxt + Vt * Vy + V * Vyt + (pyt - py * rt * ir) * ir);
    const double ptt = -(Ut * px + U * pxt + Vt * py + V * pyt + gamma * (pt * Dv + p * Dt));
    // back to conservative variables
    const double q2 = U * U + V * V;
    const double uut = U * Ut + V * Vt;
    o.Wt[0] = rt;
    o.Wt[1] = rt * U + rho * Ut;
    o.Wt[2] = rt * V + rho * Vt;
    o.Wt[3] = pt * inv_gm1 + 0.5 * rt * q2 + rho * uut;
    o.Wtt[0] = rtt;
    o.Wtt[1] = rtt * U + 2.0 * rt * Ut + rho * Utt;
    o.Wtt[2] = rtt * V + 2.0 * rt * Vt + rho * Vtt;
    o.Wtt[3] = ptt * inv_gm1 + 0.5 * rtt * q2 + 2.0 * rt * uut + rho * (Ut * Ut + U * Utt + Vt * Vt + V * Vtt);
    // normal Euler flux and its time derivative
    o.F[0] = m;
    o.F[1] = m * U + p;
    o.F[2] = m * V;
    o.F[3] = U * (E + p);
    const double mt = o.Wt[1];
    o.Ft[0] = mt;
    o.Ft[1] = mt * U + m * Ut + pt;
    o.Ft[2] = mt * V + m * Vt;
    o.Ft[3] = Ut * (E + p) + U * (o.Wt[3] + pt);
    // BGK Navier-Stokes flux per unit tau in the face-normal direction
    const double sxx = p * (2.0 * Ux - K2inv2 * Dv);
    const double sxy = p * (Uy + Vx);
    const double thx = (px - p * ir * rx) * ir;            // d/dx (p / rho)
    o.TNS[0] = 0.0;
    o.TNS[1] = sxx;
    o.TNS[2] = sxy;
    o.TNS[3] = U * sxx + V * sxy + Kheat * p * thx;
}

struct Params {
    double gamma, K, eps_tau, c_tau, dt, mu;
    double idt, inv_K2, inv_gm1;   // 1/dt, 1/(K+2), 1/(gamma-1)
    double K2inv2, Kheat;          // 2/(K+2), (K+4)/2
};

// ------------------------------------------------------------------------
// One interface quadrature point in the face frame (Sec. 2.1-2.2).
// Inputs of one Gauss point are pulled from the caller's loader when they are
// consumed, so that the 48 reconstructed quantities are never live at once:
//   src.eq_value(W0)                          equilibrium state
//   src.eq_derivs(W0n, W0t, W0nn, W0nt, W0tt)  its derivatives (face frame)
//   src.ne_value(side, W, Wt)                 left (0) / right (1) state and its
//                                             tangential derivative
//   src.ne_normal(side, Wn)                   its normal derivative
template <int STAGE, class Src>
__device__ __forceinline__ bool gks_point(const Src& src, const Params& P,
                                          double Fb[4], double Ft[4], double Wm[4], double Wb[4], double Wtt[4])
{
    const double gm1 = P.gamma - 1.0, K = P.K, dt = P.dt;
    // equilibrium state g0
    double W0[4];
    src.eq_value(W0);
    const double ir0 = __drcp_rn(W0[0]);
    const double U0 = W0[1] * ir0, V0 = W0[2] * ir0;
    const double p0 = gm1 * (W0[3] - 0.5 * (W0[1] * U0 + W0[2] * V0));
    // non-equilibrium states
    double Wl[4], Wlt[4], Wr[4], Wrt[4];
    src.ne_value(0, Wl, Wlt);
    src.ne_value(1, Wr, Wrt);
    const double irl = __drcp_rn(Wl[0]);
    const double Ul = Wl[1] * irl, Vl = Wl[2] * irl;
    const double pl = gm1 * (Wl[3] - 0.5 * (Wl[1] * Ul + Wl[2] * Vl));
    const double irr = __drcp_rn(Wr[0]);
    const double Ur = Wr[1] * irr, Vr = Wr[2] * irr;
    const double pr = gm1 * (Wr[3] - 0.5 * (Wr[1] * Ur + Wr[2] * Vr));
    const bool ok = (W0[0] > 0.0) && (p0 > 0.0) && (Wl[0] > 0.0) && (pl > 0.0) && (Wr[0] > 0.0) && (pr > 0.0);
    const double thl = pl * irl, thr = pr * irr;

    // Sec. 4: collision time with pressure-jump enhancement; viscous flow: mu/p
    // with p the equilibrium pressure at the point
    const double tau = (P.mu > 0.0 ? P.mu * __drcp_rn(p0) : P.eps_tau * dt)
                       + P.c_tau * fabs((pl - pr) * __drcp_rn(pl + pr)) * dt;
    // h = exp(-dt / (2 tau)) weights the non-equilibrium part of the interface state.
    // For dt > 80 tau, h < 4e-18: then 1 - h and 3 - h round to 1 and 3, and the
    // remaining h-terms change the window coefficients by under 2e-14 of a term
    // that is itself O(tau^2), so h is taken as 0 without evaluating the exponential
    double h = 0.0;
    if (tau > 0.0 && dt < 80.0 * tau) h = exp(-0.5 * dt * __drcp_rn(tau));
    // below 1e-20 that part is under 1e-20 of the state it is added to: far below one ulp,
    // so its velocity moments are not evaluated (the flux terms, weighted by O(tau), are)
    const bool need_ne = (STAGE == 1) && (h >= 1e-20);

    // half-line moments of g_l (u > 0) and g_r (u < 0)
    double Fh[4], Th[4], Wh[4] = {0, 0, 0, 0}, Wsl[4] = {0, 0, 0, 0};
    {
        Moments ml;
        const double ithl = __drcp_rn(thl);
        const double sq = rsqrt(2.0 * thl);            // sqrt(lambda_l)
        half_moments01(Ul, sq, 2.0 * thl * sq, +1, ml.u[0], ml.u[1]);
        moments_tail(ml, Ul, Vl, thl, K);
        SlopeCtx sl;
        slope_ctx(Ul, Vl, thl, ithl, K, P.inv_K2, sl);
        // micro-slopes of g_l: M^-1 (dW / rho); the 1/rho cancels against the rho in front
        // of the slope moments, so M^-1 is applied to dW itself
        double b1[4], a1[4], a2[4], o1[4], f[4];
        src.ne_normal(0, b1);
        micro_slope(sl, b1, a1);
        micro_slope(sl, Wlt, a2);
        psi_uv<1, 0>(ml, f);
        q_moments<1>(ml, a1, a2, o1);
        for (int k = 0; k < 4; ++k) { Fh[k] = Wl[0] * f[k]; Th[k] = o1[k]; }
        if (need_ne) {
            psi_uv<0, 0>(ml, f);
            q_moments<0>(ml, a1, a2, o1);
            for (int k = 0; k < 4; ++k) { Wh[k] = Wl[0] * f[k]; Wsl[k] = o1[k]; }
        }
    }
    {
        Moments mr;
        const double ithr = __drcp_rn(thr);
        const double sq = rsqrt(2.0 * thr);
        half_moments01(Ur, sq, 2.0 * thr * sq, -1, mr.u[0], mr.u[1]);
        moments_tail(mr, Ur, Vr, thr, K);
        SlopeCtx sr;
        slope_ctx(Ur, Vr, thr, ithr, K, P.inv_K2, sr);
        double b1[4], a1[4], a2[4], o1[4], f[4];
        src.ne_normal(1, b1);
        micro_slope(sr, b1, a1);
        micro_slope(sr, Wrt, a2);
        psi_uv<1, 0>(mr, f);
        q_moments<1>(mr, a1, a2, o1);
        for (int k = 0; k < 4; ++k) { Fh[k] += Wr[0] * f[k]; Th[k] += o1[k]; }
        if (need_ne) {
            psi_uv<0, 0>(mr, f);
            q_moments<0>(mr, a1, a2, o1);
            for (int k = 0; k < 4; ++k) { Wh[k] += Wr[0] * f[k]; Wsl[k] += o1[k]; }
        }
    }

    // Euler derivatives of the equilibrium state (W_t, W_tt, F, F_t), evaluated after the
    // half-line moments so that the two sets of intermediates are never live together
    EulerTD e;
    {
        double W0n[4], W0t[4], W0nn[4], W0nt[4], W0tt[4];
        src.eq_derivs(W0n, W0t, W0nn, W0nt, W0tt);
        euler_time_derivs(W0, W0n, W0t, W0nn, W0nt, W0tt, P.gamma, P.inv_gm1, P.K2inv2, P.Kheat, ir0,
                          U0, V0, p0, e);
    }

    // tau-terms of g0: rho <(a_n u + a_t v) u psi> = TNS - F_t (the time part is the Euler F_t)
    double T2[4];
    for (int k = 0; k < 4; ++k) T2[k] = e.TNS[k] - e.Ft[k];

    const double omh = 1.0 - h;
    const double idt = P.idt;
    const double ta = tau * omh;
    const double a = ta * (3.0 - h) * idt;
    const double g = 4.0 * ta * omh * idt * idt;
    const double b4 = tau * (tau * omh * (3.0 - h) - dt * h * (2.0 - h)) * idt;
    const double f4 = 4.0 * ta * (dt * h - ta) * idt * idt;
    for (int k = 0; k < 4; ++k) {
        const double dTh = T2[k] - Th[k];
        const double dFh = Fh[k] - e.F[k];
        Ft[k] = e.Ft[k] - g * dFh + f4 * dTh;
        if (STAGE == 1) Fb[k] = e.F[k] + a * dFh - tau * e.TNS[k] + b4 * dTh;
    }
    if (STAGE == 1) {
        // interface state W(t) = W0 + t W_t + t^2/2 W_tt + e^{-t/tau} [W_ne(t) - W0 - t W_t]
        const double th = 0.5 * dt, h2 = h * h;
        for (int k = 0; k < 4; ++k) {
            Wm[k] = W0[k] + th * e.Wt[k] + (0.125 * dt * dt) * e.Wtt[k];
            Wb[k] = W0[k] + dt * e.Wt[k] + (dt * dt / 6.0) * e.Wtt[k];
            if (need_ne) {
                Wm[k] += h * ((Wh[k] - th * Wsl[k]) - W0[k] - th * e.Wt[k]);
                Wb[k] += h2 * ((Wh[k] - dt * Wsl[k]) - W0[k] - dt * e.Wt[k]);
            }
        }
    } else {
        for (int k = 0; k < 4; ++k) Wtt[k] = e.Wtt[k];
    }
    return ok;
}

}  // namespace cgks
