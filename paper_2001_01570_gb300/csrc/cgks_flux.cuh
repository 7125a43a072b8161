// cgks_flux.cuh -- device arithmetic of the flux kernel: the reconstruction
// along a face (Gauss-point values and derivatives), the Maxwellian moments,
// the micro-slopes, the Euler time derivatives and the gas-kinetic evaluation
// at one interface quadrature point (Sec. 2.1-2.2, Sec. 4).
//
// All of it is written in the register-only DFMA forms of RegK (see
// cgks_device.cuh): x + y = fma(x, 1, y), x * y = fma(x, y, -0), and every
// coefficient -- the fixed ones and the per-grid / per-tile ones (gamma, K,
// dt and their combinations) -- is read from the shared-memory table FluxK at
// its point of use.
#pragma once
#include "cgks_device.cuh"
#include "cgks_internal.h"

namespace cgks {

// Layout of the flux kernel's shared-memory table.  Fixed constants first
// (copied from kFluxFixed), then the values of the tile's grid and time step
// (written by the CTA's first thread at the start of each tile).
enum FluxK {
    FK_ONE = 0, FK_NZERO, FK_HALF, FK_MHALF, FK_2, FK_M2, FK_3, FK_4, FK_5, FK_M3, FK_M4, FK_QUARTER, FK_EIGHTH,
    FK_ERFC_TMAX,                          // last table piece of erfcx
    FK_T13_3, FK_DLO, FK_DHI,              // tangential WENO-Z: 4 x beta weight, linear weights at the Gauss points
    FK_HG, FK_MHG,                         // +-eta/2 at the Gauss point eta = 1/(2 sqrt 3)
    FK_A1T, FK_A2T, FK_S1T, FK_S2T, FK_M0T,         // quartic: d/deta coefficients
    FK_S1TT, FK_S2TT, FK_M0TT,                      // quartic: d^2/deta^2 coefficients
    FK_M0N, FK_S1N, FK_S2N, FK_A1N, FK_A2N,         // quartic: value at the Gauss points
    FK_C0P, FK_C0M,                                  // +-1/(2 sqrt(pi))
    FK_X32LN2, FK_SHIFT, FK_LN2HI, FK_LN2LO,         // exponential: argument reduction
    FK_P2, FK_P3, FK_P4, FK_P5, FK_P6,               // exponential: 1/k! of the Taylor polynomial
    FK_NFIX,
    FK_EXP2 = FK_NFIX,                               // 2^(j/32), j = 0..31 (computed per CTA)
    FK_NFIX2 = FK_EXP2 + 32,
    // per grid and tile
    FK_DT = FK_NFIX2, FK_IDT, FK_4IDT2, FK_HDT, FK_MHDT, FK_EPSDT, FK_CTAUDT, FK_C8, FK_C6,
    FK_W1A, FK_W1B, FK_W2A, FK_W2B, FK_W3,          // Gauss-average weights of the face results
    FK_GAMMA, FK_GM1, FK_K, FK_K2, FK_KK2, FK_INVK2, FK_K2INV2, FK_KHEAT, FK_MU,
    FK_IDX, FK_IDY, FK_WEPS, FK_WEPS4,
    FK_N
};

struct FluxFixed { double v[FK_NFIX]; };

constexpr FluxFixed make_flux_fixed()
{
    FluxFixed t{};
    double* k = t.v;
    k[FK_ONE] = 1.0; k[FK_NZERO] = -0.0; k[FK_HALF] = 0.5; k[FK_MHALF] = -0.5; k[FK_2] = 2.0; k[FK_M2] = -2.0;
    k[FK_3] = 3.0; k[FK_4] = 4.0; k[FK_5] = 5.0; k[FK_M3] = -3.0; k[FK_M4] = -4.0; k[FK_QUARTER] = 0.25;
    k[FK_EIGHTH] = 0.125; k[FK_ERFC_TMAX] = 27.9;
    const double gq = 0.28867513459481287;               // 1/(2 sqrt 3)
    // the linear weights (d_lo, 11/18, d_hi) divided by 11/18 (the weights' normalisation
    // cancels the common factor)
    k[FK_T13_3] = 13.0 / 3.0;
    k[FK_DLO] = (7.0 / 36.0 - 1.7320508075688772 / 1080.0) * (18.0 / 11.0);
    k[FK_DHI] = (7.0 / 36.0 + 1.7320508075688772 / 1080.0) * (18.0 / 11.0);
    k[FK_HG] = 0.5 * gq; k[FK_MHG] = -0.5 * gq;
    // the quartic p(eta) through the five segment means (see SegmentRows::eq_derivs)
    k[FK_A1T] = 8.0 / 12.0; k[FK_A2T] = -1.0 / 12.0; k[FK_S1T] = 13.0 / 9.0; k[FK_S2T] = -1.0 / 9.0;
    k[FK_M0T] = -24.0 / 9.0;
    k[FK_S1TT] = 16.0 / 12.0; k[FK_S2TT] = -1.0 / 12.0; k[FK_M0TT] = -30.0 / 12.0;
    k[FK_M0N] = 1.0 - 6.0 / 4320.0; k[FK_S1N] = 4.0 / 4320.0; k[FK_S2N] = -1.0 / 4320.0;
    k[FK_A1N] = 50.0 / 72.0; k[FK_A2N] = -7.0 / 72.0;
    k[FK_C0P] = 0.28209479177387814; k[FK_C0M] = -0.28209479177387814;
    k[FK_X32LN2] = 32.0 / 0.6931471805599453;             // 32 / ln 2
    k[FK_SHIFT] = 6755399441055744.0;                      // 1.5 * 2^52: rounds to an integer in the low bits
    k[FK_LN2HI] = 0.6931471805599453 / 32.0;               // ln 2 / 32 and the remainder of its rounding
    k[FK_LN2LO] = 2.3190468138462996e-17 / 32.0;
    k[FK_P2] = 1.0 / 2.0; k[FK_P3] = 1.0 / 6.0; k[FK_P4] = 1.0 / 24.0; k[FK_P5] = 1.0 / 120.0;
    k[FK_P6] = 1.0 / 720.0;
    return t;
}

// per-tile entries of the table for a grid and its time step
__device__ __forceinline__ void flux_table_tile(double* t, const GridDev& G, double dt)
{
    t[FK_DT] = dt;
    t[FK_IDT] = __drcp_rn(dt);
    t[FK_4IDT2] = 4.0 * __drcp_rn(dt * dt);
    t[FK_HDT] = 0.5 * dt;
    t[FK_MHDT] = -0.5 * dt;
    t[FK_EPSDT] = G.eps_tau * dt;
    t[FK_CTAUDT] = G.c_tau * dt;
    t[FK_C8] = 0.125 * dt * dt;
    t[FK_C6] = dt * dt / 6.0;
    // stage 1: half of (dt/2, dt^2/8) and of (dt, dt^2/6) per Gauss point; stage 2: half of dt^2/3
    t[FK_W1A] = 0.25 * dt;
    t[FK_W1B] = dt * dt * (1.0 / 16.0);
    t[FK_W2A] = 0.5 * dt;
    t[FK_W2B] = dt * dt * (1.0 / 12.0);
    t[FK_W3] = dt * dt * (1.0 / 6.0);
    t[FK_GAMMA] = G.gamma;
    t[FK_GM1] = G.gamma - 1.0;
    t[FK_K] = G.K;
    t[FK_K2] = G.K + 2.0;
    t[FK_KK2] = G.K * (G.K + 2.0);
    t[FK_INVK2] = __drcp_rn(G.K + 2.0);
    t[FK_K2INV2] = 2.0 * __drcp_rn(G.K + 2.0);
    t[FK_KHEAT] = 0.5 * (G.K + 4.0);
    t[FK_MU] = G.mu;
    t[FK_IDX] = G.inv_dx;
    t[FK_IDY] = G.inv_dy;
    t[FK_WEPS] = G.weno_eps;
    t[FK_WEPS4] = 4.0 * G.weno_eps;
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
// final normalisation differ.  The weights are homogeneous in (e_k, Z) and in
// (d_k), so the code carries 4 e_k = D_k^2 + 13/3 (second difference)^2 + 4 eps
// (eps4 = 4 eps) and the linear weights divided by 11/18.
// The caller passes A1 = v_1 - v_-1 and S1 = v_1 + v_-1, which the tangential
// derivatives use too.
__device__ __forceinline__ void tang_weno5_pair(const RegK& r, double vmm, double vm, double v0, double vp,
                                                double vpp, double A1, double S1, double eps4, double& at_minus,
                                                double& at_plus)
{
    const double D0 = r.kfma(FK_3, v0, r.kfma(FK_M4, vm, vmm));
    const double D1 = A1;
    const double D2 = r.kfma(FK_4, vp, r.kfma(FK_M3, v0, -vpp));
    const double s0 = r.kfma(FK_M2, vm, r.add(vmm, v0));
    const double s1 = r.kfma(FK_M2, v0, S1);
    const double s2 = r.kfma(FK_M2, vp, r.add(v0, vpp));
    const double e0 = fma(D0, D0, fma(r.kmul(FK_T13_3, s0), s0, eps4));
    const double e1 = fma(D1, D1, fma(r.kmul(FK_T13_3, s1), s1, eps4));
    const double e2 = fma(D2, D2, fma(r.kmul(FK_T13_3, s2), s2, eps4));
    const double Z = fabs(r.sub(e0, e2));
    // (e_k + Z) times the other two = E + Z times the other two, E = e0 e1 e2
    const double e12 = r.mul(e1, e2), E = r.mul(e0, e12);
    const double P0 = fma(Z, e12, E);
    const double P1 = fma(Z, r.mul(e0, e2), E);
    const double P2 = fma(Z, r.mul(e0, e1), E);
    const double Q0 = r.mul(P0, D0), Q1 = r.mul(P1, D1), Q2 = r.mul(P2, D2);
    const double np = r.kfma(FK_DHI, Q2, r.kfma(FK_DLO, Q0, Q1)), dp = r.kfma(FK_DHI, P2, r.kfma(FK_DLO, P0, P1));
    const double nm = r.kfma(FK_DLO, Q2, r.kfma(FK_DHI, Q0, Q1)), dm = r.kfma(FK_DLO, P2, r.kfma(FK_DHI, P0, P1));
    const double inv = r.rcp(r.mul(dp, dm));             // one reciprocal for both points
    at_plus = r.kfma(FK_HG, r.mul(np, r.mul(dm, inv)), v0);
    at_minus = r.kfma(FK_MHG, r.mul(nm, r.mul(dp, inv)), v0);
}

// Three means v_{-1..1}: two linear candidates with slopes v_0 - v_-1 and
// v_1 - v_0, linear weights 1/2 at both Gauss points (the quadratic through the
// three means has no eta^2 - 1/12 term there), beta_k = slope_k^2, Z = |beta_0 -
// beta_1|.  The weights do not depend on eta: the nonlinear slope per unit eta
// is num / den; the point value is v_0 + eta * slope.
__device__ __forceinline__ void tang_weno3_parts(const RegK& r, double vm, double v0, double vp, double eps,
                                                 double& num, double& den)
{
    const double dm = r.sub(v0, vm), dp = r.sub(vp, v0);
    const double e0 = fma(dm, dm, eps), e1 = fma(dp, dp, eps);
    const double Z = fabs(r.sub(e0, e1));
    const double e01 = r.mul(e0, e1);
    const double n0 = fma(Z, e1, e01), n1 = fma(Z, e0, e01);          // (e0 + Z) e1, (e1 + Z) e0
    num = fma(n1, dp, r.mul(n0, dm));
    den = r.add(n0, n1);
}

// the slopes of the left and right states' rows, with one reciprocal for both
__device__ __forceinline__ void tang_weno3_slopes(const RegK& r, double lm, double l0, double lp, double rm,
                                                  double r0, double rp, double eps, double& sl, double& sr)
{
    double nl, dl, nr, dr;
    tang_weno3_parts(r, lm, l0, lp, eps, nl, dl);
    tang_weno3_parts(r, rm, r0, rp, eps, nr, dr);
    const double inv = r.rcp(r.mul(dl, dr));
    sl = r.mul(nl, r.mul(dr, inv));
    sr = r.mul(nr, r.mul(dl, inv));
}

// ------------------------------------------------------------------------
// e^x for x <= 0 by Tang's table-driven method (ACM TOMS 15, 1989): x = (32 m +
// j) ln2/32 + r with |r| <= ln2/64, e^x = 2^m 2^(j/32) e^r, e^r from its Taylor
// polynomial of degree 6 (truncation below 4e-18 relative), 2^(j/32) from the
// table, 2^m added to the exponent field.  Below -700 (e^x < 1e-304) it returns 0.
__device__ __forceinline__ double exp_neg(const RegK& r, double x)
{
#ifdef CGKS_OPCOUNT_HOST
    return cgks_opcount_exp(x);   // one exponential in the host operation count
#endif
    if (x < -700.0) return 0.0;
    const double t = r.kfma(FK_X32LN2, x, r.k(FK_SHIFT));
    const double n = r.sub(t, r.k(FK_SHIFT));             // round(32 x / ln 2), exactly
    const int ni = (int)(unsigned)__double_as_longlong(t);
    const double q = r.kfma(FK_LN2LO, -n, r.kfma(FK_LN2HI, -n, x));
    double p = fma(r.k(FK_P6), q, r.k(FK_P5));
    p = fma(p, q, r.k(FK_P4));
    p = fma(p, q, r.k(FK_P3));
    p = fma(p, q, r.k(FK_P2));
    p = fma(p, q, r.one);
    p = fma(p, q, r.one);
    const double y = r.mul(r.k(FK_EXP2 + (ni & 31)), p);
    return __longlong_as_double(__double_as_longlong(y) + ((long long)(ni >> 5) << 52));
}

// ------------------------------------------------------------------------
// erfc(t) for t >= 0 from e = exp(-t^2): e * erfcx(t), erfcx from the piecewise
// polynomials of cgks_erfcx_table.h (relative error ~2e-16); 11 FMAs instead
// of a full erfc evaluation, since the half-line moments need e anyway.  Past
// t = 27.3 e underflows to 0; a NaN t selects the last piece and stays NaN.
__device__ __forceinline__ double erfc_scaled(const RegK& r, double t, double e)
{
#ifdef CGKS_OPCOUNT_HOST
    return cgks_opcount_erfc(t);   // one erfc in the host operation count
#endif
    const int k = (int)r.kmul(FK_4, fmin(t, r.k(FK_ERFC_TMAX)));
    const double* c = cgks_erfcx_coef[k];
    const double z = r.sub(t, r.kfma(FK_QUARTER, (double)k, r.k(FK_EIGHTH)));
    double v = c[0];
#pragma unroll
    for (int m = 1; m <= CGKS_ERFCX_DEG; ++m) v = fma(v, z, c[m]);
    return r.mul(e, v);
}

// the two lowest half-line u-moments of a Maxwellian with mean U and
// sqrt(lambda) = sq: <u^0> = erfc(-+ s)/2, <u^1> = U <u^0> +- e^{-s^2}/(2 sqrt(pi lambda)),
// s = U sqrt(lambda); SIDE = +1 for u > 0, -1 for u < 0
template <int SIDE>
__device__ __forceinline__ void half_moments01(const RegK& r, double U, double sq, double inv_sq, double& m0,
                                               double& m1)
{
    const double s = r.mul(U, sq);
    const double e = exp_neg(r, -r.mul(s, s));
    const double hE = r.kmul(FK_HALF, erfc_scaled(r, fabs(s), e));    // erfc(|s|)/2
    // SIDE +1: erfc(-s)/2 = 1 - erfc(s)/2 for s >= 0, erfc(|s|)/2 for s < 0; SIDE -1 mirrored
    const bool pos = (SIDE > 0) ? (s >= 0.0) : (s < 0.0);
    m0 = pos ? r.sub(r.one, hE) : hE;
    m1 = fma(U, m0, r.kmul(SIDE > 0 ? FK_C0P : FK_C0M, r.mul(e, inv_sq)));
}

// ------------------------------------------------------------------------
// Sec. 2.1: Maxwellian velocity moments.  theta = p/rho = 1/(2 lambda).
struct Moments {
    double u[7];     // <u^n>, n = 0..6 (whole line or half line)
    double v[6];     // <v^n>, n = 0..5 (whole line); v[0] = 1 is never multiplied
    double x1, x2;   // <xi^2>, <xi^4>
};

__device__ __forceinline__ void moments_tail(const RegK& r, Moments& m, double U, double V, double theta)
{
    const double t2 = r.add(theta, theta), t3 = r.kmul(FK_3, theta), t4 = r.kmul(FK_4, theta),
                 t5 = r.kmul(FK_5, theta);
    m.u[2] = fma(U, m.u[1], r.mul(theta, m.u[0]));
    m.u[3] = fma(U, m.u[2], r.mul(t2, m.u[1]));
    m.u[4] = fma(U, m.u[3], r.mul(t3, m.u[2]));
    m.u[5] = fma(U, m.u[4], r.mul(t4, m.u[3]));
    m.u[6] = fma(U, m.u[5], r.mul(t5, m.u[4]));
    m.v[0] = 1.0;
    m.v[1] = V;
    m.v[2] = fma(V, V, theta);
    m.v[3] = fma(V, m.v[2], r.mul(t2, V));
    m.v[4] = fma(V, m.v[3], r.mul(t3, m.v[2]));
    m.v[5] = fma(V, m.v[4], r.mul(t4, m.v[3]));
    m.x1 = r.mul(r.k(FK_K), theta);
    m.x2 = r.mul(r.mul(r.k(FK_KK2), theta), theta);
}

// <u^A psi> of a Maxwellian (whole-line v-moments, B = 0)
template <int A>
__device__ __forceinline__ void psi_u(const RegK& r, const Moments& m, double o[4])
{
    o[0] = m.u[A];
    o[1] = m.u[A + 1];
    o[2] = r.mul(m.u[A], m.v[1]);
    o[3] = r.kmul(FK_HALF, fma(m.u[A], m.x1, fma(m.u[A], m.v[2], m.u[A + 2])));
}

// <psi u^A (u (a1 . psi) + v (a2 . psi))> for a Maxwellian, with a . psi =
// a0 + a1 u + a2 v + a3 (u^2 + v^2 + xi^2)/2: the slope terms of the half-line
// moments (A = 1: the flux part, A = 0: the interface-state part).  The
// polynomial in the bracket, times u^A, is grouped by powers of v,
//   v^0: a1_0 u + a1_1 u^2 + h1 u^3  (+ h1 u xi^2),  v^1: a2_0 + c12 u + h2 u^2  (+ h2 xi^2),
//   v^2: a2_2 + h1 u,                v^3: h2,
// (h = a_3/2, c12 = a1_2 + a2_1), so each psi component is a short sum of
// products of the factorised u-, v- and xi-moments.
// (a[3] holds h = a_3 / 2, as micro_slope returns it)
template <int A>
__device__ __forceinline__ void q_moments(const RegK& r, const Moments& m, const double a1[4], const double a2[4],
                                          double o[4])
{
    const double h1 = a1[3], h2 = a2[3], c12 = r.add(a1[2], a2[1]);
    // sums over u for the v^j groups at u-shift s2 (S_j) and the xi^2 parts (Z_j); S_3 = Z_1
    double S0[3], S1[3], S2[3], Z0[3], Z1[3];
#pragma unroll
    for (int s2 = 0; s2 < 3; ++s2) {
        Z0[s2] = r.mul(h1, m.u[A + 1 + s2]);
        Z1[s2] = r.mul(h2, m.u[A + s2]);
    }
#pragma unroll
    for (int s2 = 0; s2 < 3; ++s2) {
        // h1 u[A+3] = Z0[2] and h2 u[A+2] = Z1[2] for the first shift
        const double t0 = (s2 == 0) ? Z0[2] : r.mul(h1, m.u[A + 3 + s2]);
        const double t1 = (s2 == 0) ? Z1[2] : r.mul(h2, m.u[A + 2 + s2]);
        S0[s2] = fma(a1[1], m.u[A + 2 + s2], fma(a1[0], m.u[A + 1 + s2], t0));
        S1[s2] = fma(c12, m.u[A + 1 + s2], fma(a2[0], m.u[A + s2], t1));
        S2[s2] = fma(a2[2], m.u[A + s2], Z0[s2]);
    }
    const double x1 = m.x1, x2 = m.x2;
    // sum_j v[j+sh] S_j[s2] + x1 (v[sh] Z0[s2] + v[sh+1] Z1[s2]), v[0] = 1
    auto sum = [&](int s2, int sh) {
        const double lo = (sh == 0) ? S0[s2] : r.mul(m.v[sh], S0[s2]);
        const double z = (sh == 0) ? fma(m.v[1], Z1[s2], Z0[s2]) : fma(m.v[sh + 1], Z1[s2], r.mul(m.v[sh], Z0[s2]));
        return fma(x1, z, fma(m.v[sh + 3], Z1[s2], fma(m.v[sh + 2], S2[s2], fma(m.v[sh + 1], S1[s2], lo))));
    };
    const double plain0 = fma(m.v[3], Z1[0], fma(m.v[2], S2[0], fma(m.v[1], S1[0], S0[0])));
    const double xi0 = fma(m.v[1], Z1[0], Z0[0]);
    o[0] = fma(x1, xi0, plain0);
    o[1] = sum(1, 0);
    o[2] = sum(0, 1);
    o[3] = r.kmul(FK_HALF, fma(x2, xi0, fma(x1, plain0, r.add(sum(2, 0), sum(0, 2)))));
}

// micro-slope coefficients a with <psi psi^T> a = b for a Maxwellian
// (closed form of the 4x4 moment system); a[3] receives h = a_3 / 2, the factor
// q_moments uses (psi_4 carries 1/2)
struct SlopeCtx { double U, V, Bm, inv_theta, c4; };

__device__ __forceinline__ void slope_ctx(const RegK& r, double U, double V, double theta, double inv_theta,
                                          SlopeCtx& s)
{
    s.U = U; s.V = V;
    s.Bm = fma(U, U, fma(V, V, r.mul(r.k(FK_K2), theta)));
    s.inv_theta = inv_theta;
    s.c4 = r.mul(r.mul(inv_theta, inv_theta), r.k(FK_INVK2));
}

__device__ __forceinline__ void micro_slope(const RegK& r, const SlopeCtx& s, const double b[4], double a[4])
{
    const double R4 = fma(-s.Bm, b[0], r.add(b[3], b[3]));
    const double R3 = fma(-s.V, b[0], b[2]);
    const double R2 = fma(-s.U, b[0], b[1]);
    const double a3 = r.mul(s.c4, r.kfma(FK_M2, fma(s.V, R3, r.mul(s.U, R2)), R4));
    const double h = r.kmul(FK_HALF, a3);
    a[2] = fma(-s.V, a3, r.mul(R3, s.inv_theta));
    a[1] = fma(-s.U, a3, r.mul(R2, s.inv_theta));
    a[0] = fma(-h, s.Bm, fma(-s.V, a[2], fma(-s.U, a[1], b[0])));
    a[3] = h;
}

// ------------------------------------------------------------------------
// Euler time derivatives by Cauchy-Kowalevski in primitive variables.
// Inputs: conservative W and its x (normal), y (tangential) derivatives up to
// second order, 1/rho, the velocity, the pressure p and the internal energy per
// volume e = p / (gamma - 1).  The pressure's derivatives are carried as those
// of e (p_x = (gamma - 1) e_x, ...), which are differences of the energy's and
// the kinetic energy's.  Outputs conservative W_t, W_tt and the flux time
// derivative F_t of the normal Euler flux.
// TNS is rho <(a_n u + a_t v + A) u psi> of the equilibrium state, i.e. the
// Chapman-Enskog Navier-Stokes flux of the BGK model per unit collision time
// (mu = tau p, bulk part 2/(K+2), heat conduction (K+4)/2 tau p grad(p/rho)).
struct EulerTD { double Wt[4], Wtt[4], Ft[4], F[4], TNS[4]; };

__device__ __forceinline__ void euler_time_derivs(const RegK& r, const double W[4], const double Wx[4],
                                                  const double Wy[4], const double Wxx[4], const double Wxy[4],
                                                  const double Wyy[4], double ir, double U, double V, double p,
                                                  double e, EulerTD& o)
{
    const double rho = W[0], m = W[1], E = W[3];
    // primitive first derivatives
    const double rx = Wx[0], ry = Wy[0];
    const double Ux = r.mul(fma(-U, rx, Wx[1]), ir), Uy = r.mul(fma(-U, ry, Wy[1]), ir);
    const double Vx = r.mul(fma(-V, rx, Wx[2]), ir), Vy = r.mul(fma(-V, ry, Wy[2]), ir);
    // kinetic energy KE = rho q^2 / 2: KE_x = u . m_x - rho_x q^2/2,
    // KE_xx = rho |u_x|^2 + u . m_xx - rho_xx q^2/2, KE_xy = rho u_x . u_y + u . m_xy - rho_xy q^2/2
    const double q2 = fma(U, U, r.mul(V, V));
    const double hq2 = r.kmul(FK_HALF, q2);
    const double KEx = fma(-hq2, rx, fma(V, Wx[2], r.mul(U, Wx[1])));
    const double KEy = fma(-hq2, ry, fma(V, Wy[2], r.mul(U, Wy[1])));
    const double ex = r.sub(Wx[3], KEx), ey = r.sub(Wy[3], KEy);
    // primitive second derivatives
    const double rxx = Wxx[0], rxy = Wxy[0], ryy = Wyy[0];
    const double rx2 = r.add(rx, rx), ry2 = r.add(ry, ry);
    const double Uxx = r.mul(fma(-U, rxx, fma(-Ux, rx2, Wxx[1])), ir);
    const double Uxy = r.mul(fma(-U, rxy, fma(-Uy, rx, fma(-Ux, ry, Wxy[1]))), ir);
    const double Uyy = r.mul(fma(-U, ryy, fma(-Uy, ry2, Wyy[1])), ir);
    const double Vxx = r.mul(fma(-V, rxx, fma(-Vx, rx2, Wxx[2])), ir);
    const double Vxy = r.mul(fma(-V, rxy, fma(-Vy, rx, fma(-Vx, ry, Wxy[2]))), ir);
    const double Vyy = r.mul(fma(-V, ryy, fma(-Vy, ry2, Wyy[2])), ir);
    const double KExx = fma(-hq2, rxx, fma(V, Wxx[2], fma(U, Wxx[1], r.mul(rho, fma(Ux, Ux, r.mul(Vx, Vx))))));
    const double KExy = fma(-hq2, rxy, fma(V, Wxy[2], fma(U, Wxy[1], r.mul(rho, fma(Ux, Uy, r.mul(Vx, Vy))))));
    const double KEyy = fma(-hq2, ryy, fma(V, Wyy[2], fma(U, Wyy[1], r.mul(rho, fma(Uy, Uy, r.mul(Vy, Vy))))));
    const double exx = r.sub(Wxx[3], KExx), exy = r.sub(Wxy[3], KExy), eyy = r.sub(Wyy[3], KEyy);
    // first time derivatives (p_x / rho = e_x gir)
    const double gamma = r.k(FK_GAMMA);
    const double gir = r.mul(r.k(FK_GM1), ir);
    const double Dv = r.add(Ux, Vy);
    const double rt = -fma(rho, Dv, fma(V, ry, r.mul(U, rx)));
    const double Ut = -fma(ex, gir, fma(V, Uy, r.mul(U, Ux)));
    const double Vt = -fma(ey, gir, fma(V, Vy, r.mul(U, Vx)));
    const double et = -fma(r.mul(gamma, e), Dv, fma(V, ey, r.mul(U, ex)));
    // mixed derivatives d/dx, d/dy of the first time derivatives
    const double Dx = r.add(Uxx, Vxy), Dy = r.add(Uxy, Vyy);
    const double rxt = -fma(rho, Dx, fma(rx, Dv, fma(V, rxy, fma(Vx, ry, fma(U, rxx, r.mul(Ux, rx))))));
    const double ryt = -fma(rho, Dy, fma(ry, Dv, fma(V, ryy, fma(Vy, ry, fma(U, rxy, r.mul(Uy, rx))))));
    const double Uxt = -fma(fma(-r.mul(ex, rx), ir, exx), gir, fma(V, Uxy, fma(Vx, Uy, fma(U, Uxx, r.mul(Ux, Ux)))));
    const double Vyt = -fma(fma(-r.mul(ey, ry), ir, eyy), gir, fma(V, Vyy, fma(Vy, Vy, fma(U, Vxy, r.mul(Uy, Vx)))));
    const double Uyt = -fma(fma(-r.mul(ex, ry), ir, exy), gir, fma(V, Uyy, fma(Vy, Uy, fma(U, Uxy, r.mul(Uy, Ux)))));
    const double Vxt = -fma(fma(-r.mul(ey, rx), ir, exy), gir, fma(V, Vxy, fma(Vx, Vy, fma(U, Vxx, r.mul(Ux, Vx)))));
    const double ext = -fma(gamma, fma(e, Dx, r.mul(ex, Dv)), fma(V, exy, fma(Vx, ey, fma(U, exx, r.mul(Ux, ex)))));
    const double eyt = -fma(gamma, fma(e, Dy, r.mul(ey, Dv)), fma(V, eyy, fma(Vy, ey, fma(U, exy, r.mul(Uy, ex)))));
    // second time derivatives
    const double Dt = r.add(Uxt, Vyt);
    const double rtt = -fma(rho, Dt, fma(rt, Dv, fma(V, ryt, fma(Vt, ry, fma(U, rxt, r.mul(Ut, rx))))));
    const double Utt = -fma(fma(-r.mul(ex, rt), ir, ext), gir, fma(V, Uyt, fma(Vt, Uy, fma(U, Uxt, r.mul(Ut, Ux)))));
    const double Vtt = -fma(fma(-r.mul(ey, rt), ir, eyt), gir, fma(V, Vyt, fma(Vt, Vy, fma(U, Vxt, r.mul(Ut, Vx)))));
    const double ett = -fma(gamma, fma(e, Dt, r.mul(et, Dv)), fma(V, eyt, fma(Vt, ey, fma(U, ext, r.mul(Ut, ex)))));
    // back to conservative variables (E = e + KE)
    const double uut = fma(V, Vt, r.mul(U, Ut));
    o.Wt[0] = rt;
    o.Wt[1] = fma(rho, Ut, r.mul(rt, U));
    o.Wt[2] = fma(rho, Vt, r.mul(rt, V));
    o.Wt[3] = fma(rho, uut, fma(rt, hq2, et));
    const double rt2 = r.add(rt, rt);
    o.Wtt[0] = rtt;
    o.Wtt[1] = fma(rho, Utt, fma(rt2, Ut, r.mul(rtt, U)));
    o.Wtt[2] = fma(rho, Vtt, fma(rt2, Vt, r.mul(rtt, V)));
    o.Wtt[3] = fma(rho, fma(V, Vtt, fma(Vt, Vt, fma(U, Utt, r.mul(Ut, Ut)))), fma(rt2, uut, fma(rtt, hq2, ett)));
    // normal Euler flux and its time derivative
    const double Ep = r.add(E, p);
    const double pt = r.mul(r.k(FK_GM1), et);
    o.F[0] = m;
    o.F[1] = fma(m, U, p);
    o.F[2] = r.mul(m, V);
    o.F[3] = r.mul(U, Ep);
    const double mt = o.Wt[1];
    o.Ft[0] = mt;
    o.Ft[1] = fma(m, Ut, fma(mt, U, pt));
    o.Ft[2] = fma(m, Vt, r.mul(mt, V));
    o.Ft[3] = fma(U, r.add(o.Wt[3], pt), r.mul(Ut, Ep));
    // BGK Navier-Stokes flux per unit tau in the face-normal direction
    const double sxx = r.mul(p, fma(-r.k(FK_K2INV2), Dv, r.add(Ux, Ux)));
    const double sxy = r.mul(p, r.add(Uy, Vx));
    const double thx = r.mul(fma(-r.mul(e, ir), rx, ex), gir);            // d/dx (p / rho)
    o.TNS[0] = 0.0;
    o.TNS[1] = sxx;
    o.TNS[2] = sxy;
    o.TNS[3] = fma(r.mul(r.k(FK_KHEAT), p), thx, fma(V, sxy, r.mul(U, sxx)));
}

// ------------------------------------------------------------------------
// One interface quadrature point in the face frame (Sec. 2.1-2.2).
// Inputs of one Gauss point are pulled from the caller's loader when they are
// consumed, so that the 48 reconstructed quantities are never live at once:
//   src.eq_value(W0)                          equilibrium state
//   src.eq_derivs(W0n, W0t, W0nn, W0nt, W0tt)  its derivatives (face frame)
//   src.ne_value(side, W, Wt)                 left (0) / right (1) state and its
//                                             tangential derivative
//   src.ne_normal(side, Wn)                   its normal derivative
// The caller's table holds the grid's gamma, K and the time step.
template <int STAGE, class Src>
__device__ __forceinline__ bool gks_point(const RegK& r, const Src& src, double Fb[4], double Ft[4], double Wm[4],
                                          double Wb[4], double Wtt[4])
{
    // equilibrium state g0
    double W0[4];
    src.eq_value(W0);
    const double ir0 = r.rcp(W0[0]);
    const double U0 = r.mul(W0[1], ir0), V0 = r.mul(W0[2], ir0);
    const double e0 = r.kfma(FK_MHALF, fma(W0[2], V0, r.mul(W0[1], U0)), W0[3]);   // p0 / (gamma - 1)
    const double p0 = r.mul(r.k(FK_GM1), e0);
    // non-equilibrium states
    double Wl[4], Wlt[4], Wr[4], Wrt[4];
    src.ne_value(0, Wl, Wlt);
    src.ne_value(1, Wr, Wrt);
    const double irl = r.rcp(Wl[0]);
    const double Ul = r.mul(Wl[1], irl), Vl = r.mul(Wl[2], irl);
    const double pl = r.mul(r.k(FK_GM1), r.kfma(FK_MHALF, fma(Wl[2], Vl, r.mul(Wl[1], Ul)), Wl[3]));
    const double irr = r.rcp(Wr[0]);
    const double Ur = r.mul(Wr[1], irr), Vr = r.mul(Wr[2], irr);
    const double pr = r.mul(r.k(FK_GM1), r.kfma(FK_MHALF, fma(Wr[2], Vr, r.mul(Wr[1], Ur)), Wr[3]));
    const bool ok = (W0[0] > 0.0) && (p0 > 0.0) && (Wl[0] > 0.0) && (pl > 0.0) && (Wr[0] > 0.0) && (pr > 0.0);
    const double thl = r.mul(pl, irl), thr = r.mul(pr, irr);

    // Sec. 4: collision time with pressure-jump enhancement; viscous flow: mu/p
    // with p the equilibrium pressure at the point
    const double mu = r.k(FK_MU), dt = r.k(FK_DT);
    const double tau = fma(r.k(FK_CTAUDT), fabs(r.mul(r.sub(pl, pr), r.rcp(r.add(pl, pr)))),
                           mu > 0.0 ? r.mul(mu, r.rcp(p0)) : r.k(FK_EPSDT));
    // h = exp(-dt / (2 tau)) weights the non-equilibrium part of the interface state.
    // For dt > 80 tau, h < 4e-18: then 1 - h and 3 - h round to 1 and 3, and the
    // remaining h-terms change the window coefficients by under 2e-14 of a term
    // that is itself O(tau^2), so h is taken as 0 without evaluating the exponential
    double h = 0.0;
    if (tau > 0.0 && dt < 80.0 * tau) h = exp_neg(r, r.mul(r.k(FK_MHDT), r.rcp(tau)));
    // below 1e-20 that part is under 1e-20 of the state it is added to: far below one ulp,
    // so its velocity moments are not evaluated (the flux terms, weighted by O(tau), are)
    const bool need_ne = (STAGE == 1) && (h >= 1e-20);

    // half-line moments of g_l (u > 0) and g_r (u < 0)
    double Fh[4], Th[4], Wh[4] = {0, 0, 0, 0}, Wsl[4] = {0, 0, 0, 0};
    {
        Moments ml;
        const double th2 = r.add(thl, thl);
        const double sq = rsqrt(th2);                     // sqrt(lambda_l) = 1/sqrt(2 theta)
        const double ithl = r.mul(r.add(sq, sq), sq);     // 1/theta = 2 lambda_l
        half_moments01<+1>(r, Ul, sq, r.mul(th2, sq), ml.u[0], ml.u[1]);
        moments_tail(r, ml, Ul, Vl, thl);
        SlopeCtx sl;
        slope_ctx(r, Ul, Vl, thl, ithl, sl);
        // micro-slopes of g_l: M^-1 (dW / rho); the 1/rho cancels against the rho in front
        // of the slope moments, so M^-1 is applied to dW itself
        double b1[4], a1[4], a2[4], o1[4], f[4];
        src.ne_normal(0, b1);
        micro_slope(r, sl, b1, a1);
        micro_slope(r, sl, Wlt, a2);
        psi_u<1>(r, ml, f);
        q_moments<1>(r, ml, a1, a2, o1);
        for (int k = 0; k < 4; ++k) { Fh[k] = r.mul(Wl[0], f[k]); Th[k] = o1[k]; }
        if (need_ne) {
            psi_u<0>(r, ml, f);
            q_moments<0>(r, ml, a1, a2, o1);
            for (int k = 0; k < 4; ++k) { Wh[k] = r.mul(Wl[0], f[k]); Wsl[k] = o1[k]; }
        }
    }
    {
        Moments mr;
        const double th2 = r.add(thr, thr);
        const double sq = rsqrt(th2);
        const double ithr = r.mul(r.add(sq, sq), sq);
        half_moments01<-1>(r, Ur, sq, r.mul(th2, sq), mr.u[0], mr.u[1]);
        moments_tail(r, mr, Ur, Vr, thr);
        SlopeCtx sr;
        slope_ctx(r, Ur, Vr, thr, ithr, sr);
        double b1[4], a1[4], a2[4], o1[4], f[4];
        src.ne_normal(1, b1);
        micro_slope(r, sr, b1, a1);
        micro_slope(r, sr, Wrt, a2);
        psi_u<1>(r, mr, f);
        q_moments<1>(r, mr, a1, a2, o1);
        for (int k = 0; k < 4; ++k) { Fh[k] = fma(Wr[0], f[k], Fh[k]); Th[k] = r.add(Th[k], o1[k]); }
        if (need_ne) {
            psi_u<0>(r, mr, f);
            q_moments<0>(r, mr, a1, a2, o1);
            for (int k = 0; k < 4; ++k) { Wh[k] = fma(Wr[0], f[k], Wh[k]); Wsl[k] = r.add(Wsl[k], o1[k]); }
        }
    }

    // Euler derivatives of the equilibrium state (W_t, W_tt, F, F_t), evaluated after the
    // half-line moments so that the two sets of intermediates are never live together
    EulerTD e;
    {
        double W0n[4], W0t[4], W0nn[4], W0nt[4], W0tt[4];
        src.eq_derivs(W0n, W0t, W0nn, W0nt, W0tt);
        euler_time_derivs(r, W0, W0n, W0t, W0nn, W0nt, W0tt, ir0, U0, V0, p0, e0, e);
    }

    // tau-terms of g0: rho <(a_n u + a_t v) u psi> = TNS - F_t (the time part is the Euler F_t)
    const double idt = r.k(FK_IDT);
    const double omh = r.sub(r.one, h);
    const double ta = r.mul(tau, omh);                       // tau (1 - h)
    const double q4 = r.mul(ta, r.k(FK_4IDT2));              // 4 tau (1 - h) / dt^2
    const double g = r.mul(q4, omh);
    const double dh = r.mul(dt, h);
    const double f4 = r.mul(q4, r.sub(dh, ta));
    const double tat = r.mul(ta, r.sub(r.k(FK_3), h));       // tau (1 - h) (3 - h)
    const double a = r.mul(tat, idt);
    const double b4 = r.mul(r.mul(tau, fma(-dh, r.sub(r.k(FK_2), h), tat)), idt);
    for (int k = 0; k < 4; ++k) {
        const double dTh = (k == 0) ? -r.add(e.Ft[0], Th[0]) : r.sub(r.sub(e.TNS[k], e.Ft[k]), Th[k]);
        const double dFh = r.sub(Fh[k], e.F[k]);
        Ft[k] = fma(f4, dTh, fma(-g, dFh, e.Ft[k]));
        if (STAGE == 1) Fb[k] = fma(b4, dTh, (k == 0) ? fma(a, dFh, e.F[0]) : fma(-tau, e.TNS[k], fma(a, dFh, e.F[k])));
    }
    if (STAGE == 1) {
        // interface state W(t) = W0 + t W_t + t^2/2 W_tt + e^{-t/tau} [W_ne(t) - W0 - t W_t]
        const double hdt = r.k(FK_HDT), h2 = r.mul(h, h);
        for (int k = 0; k < 4; ++k) {
            Wm[k] = fma(r.k(FK_C8), e.Wtt[k], fma(hdt, e.Wt[k], W0[k]));
            Wb[k] = fma(r.k(FK_C6), e.Wtt[k], fma(dt, e.Wt[k], W0[k]));
            if (need_ne) {
                Wm[k] = fma(h, fma(-hdt, e.Wt[k], r.sub(fma(-hdt, Wsl[k], Wh[k]), W0[k])), Wm[k]);
                Wb[k] = fma(h2, fma(-dt, e.Wt[k], r.sub(fma(-dt, Wsl[k], Wh[k]), W0[k])), Wb[k]);
            }
        }
    } else {
        for (int k = 0; k < 4; ++k) Wtt[k] = e.Wtt[k];
    }
    return ok;
}

}  // namespace cgks
