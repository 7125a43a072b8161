/*
 * cgks_oracle.c -- plain, slow, FP64 CPU oracle of the compact 8th-order
 * gas-kinetic scheme (Zhao, Ji, Shyy, Xu, "An acoustic and shock wave
 * capturing compact high-order gas-kinetic scheme with spectral-like
 * resolution", arXiv 2001.01570).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference the CUDA path is
 * checked against.  It shares no code, header, table or helper with the
 * CUDA library (paper_2001_01570_gb300/csrc) and must never be linked into
 * or called from the product path.  Only tests/, the smoke check and the
 * CPU-baseline leg of bench.py load it.
 *
 * Everything is computed in the order the paper states it:
 *   Sec. 3.2, Eq. (recons-8th-val)  linear compact reconstruction P7, P7_x, P7_xx
 *   Sec. 3.3, Eq. (sub-stencil)     candidate polynomials q_0..q_6 on S_0..S_6,
 *                                   linear weights d_k, WENO-Z weights
 *                                   Eq. (WENO-Z-w), indicators Eq. (smooth-
 *                                   indicator), Z_ref Eq. (tau), beta_1 taken
 *                                   from the cubic on {Q_i-1,Q_i,Q_i+1,Q'_i-1}
 *   Sec. 2.1, Eq. (bgk), (compatibility), (g-to-convar), (g-to-flux),
 *             Eq. (3rd-simplify-flux) with the third-order terms removed for
 *             the flux, and in full for the interface state
 *   Sec. 2.2, Eq. (step-hyper-1)    two-stage fourth-order (S2O4) update, and
 *             the S2O4 update of the interface distribution
 *   Sec. 3.1, Eq. (compact-deriv-1) Gauss-theorem update of cell-averaged
 *             gradients (divergence theorem in 2D)
 *   Sec. 4                          collision time tau, CFL time step
 *
 * Readings where the paper is silent:
 *   - polynomials of the sub-stencils are built from their definition (cell
 *     averages and cell-averaged slopes) by solving the small linear system;
 *     the slope of the non-equilibrium states is sum_k delta_k q_k'(x_i+1/2)
 *   - the right state is the left procedure applied to the mirrored stencil
 *   - the time-dependent flux is reduced to F + F_t t by matching its time
 *     integrals over [0, dt/2] and [0, dt] (both stages use the full dt and
 *     the tau computed from it)
 *   - the interface state is the psi-moment of the third-order distribution:
 *     W(t) = W0 + t W0_t + t^2/2 W0_tt + NE(t); W0_t, W0_tt are the Euler
 *     time derivatives (Cauchy-Kowalevski), NE(t) the non-equilibrium part
 *   - 2D: two Gauss points per face.  Each face row gets the 1D normal
 *     reconstruction; along the face, the equilibrium derivatives at the
 *     Gauss points come from the quartic whose means over the five segments
 *     j-2..j+2 equal the line averages of those rows, and the normal
 *     derivatives of the non-equilibrium states from the quadratic through
 *     rows j-1..j+1.  The point VALUES along the face (and the tangential
 *     slopes of the non-equilibrium states) are nonlinear: WENO-Z on the same
 *     rows with linear weights that reproduce the quartic / quadratic at the
 *     Gauss point, because the linear fits turn negative across a
 *     discontinuity that runs through the faces (a normal shock seen by the
 *     faces parallel to it).
 *     The cell-averaged tangential gradient is used only by the faces normal
 *     to it (a face-interpolated tangential gradient makes the 2D scheme
 *     linearly unstable under advection)
 *   - 1D uses K = (3-gamma)/(gamma-1) internal degrees of freedom
 *   - characteristic reconstruction (optional): eigenvectors of the normal flux
 *     Jacobian at the mean of the two cells sharing the face
 *   - compact 6th-order variant (optional; Sec. 3.2 names it without printing
 *     it): the linear reconstruction is the degree-5 polynomial fixed by the
 *     four cell averages and the two slopes Q'_i, Q'_i+1 next to the face; the
 *     nonlinear one keeps the candidates q_0..q_6 with the linear weights that
 *     recombine them into that polynomial's interface value
 *   - CFL: dt = CFL * min_cells min(dx/(|U|+c), dy/(|V|+c)); with viscosity the
 *     signal speed is |U|+c+2 nu/dx (nu = mu/rho)
 *
 * Build: gcc -O2 -fPIC -shared -fopenmp -ffp-contract=off
 */
#include <math.h>
#include <omp.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

#define OC_OK 0
#define OC_E_INVAL 1
#define OC_E_NONPHYSICAL 5

enum { BC_PERIODIC = 0, BC_REFLECT = 1, BC_INFLOW = 2, BC_OUTFLOW = 3,
       BC_HALO = 4 /* x-sides only: ghost columns supplied by the caller (domain decomposition) */ };

typedef struct {
    int dim, nx, ny;
    double dx, dy;
    double gamma, cfl;
    int bc[4];          /* x-low, x-high, y-low, y-high */
    double inflow[4][4];   /* per side (x-low, x-high, y-low, y-high): primitive rho, u, v, p */
    double eps_tau, c_tau, weno_eps;
    double mu;          /* > 0: viscous collision time mu/p (Sec. 4) */
    int recon_vars;     /* nonlinear reconstruction in 0: conservative, 1: characteristic variables */
    int order;          /* 6: compact 6th-order variant; anything else: the 8th-order scheme */
} oc_problem;

static int recon_order(const oc_problem *P) { return P->order == 6 ? 6 : 8; }

/* ------------------------------------------------------------------ */
/* Sec. 3.2, Eq. (recons-8th-val): linear compact 8th-order reconstruction
 * at x_{i+1/2} from Q_{i-1..i+2} and h*Q'_{i-1..i+2}.
 * out[0] = P7, out[1] = h*P7_x, out[2] = h^2*P7_xx                     */
void oc_linear_recon(const double Q[4], const double hQp[4], double out[3])
{
    out[0] = (25.0 * Q[0] + 185.0 * Q[1] + 185.0 * Q[2] + 25.0 * Q[3]
              + 6.0 * hQp[0] + 102.0 * hQp[1] - 102.0 * hQp[2] - 6.0 * hQp[3]) / 420.0;
    out[1] = (-14.0 * Q[0] - 270.0 * Q[1] + 270.0 * Q[2] + 14.0 * Q[3]
              - 3.0 * hQp[0] - 99.0 * hQp[1] - 99.0 * hQp[2] - 3.0 * hQp[3]) / 108.0;
    out[2] = (-4.0 * Q[0] + 4.0 * Q[1] + 4.0 * Q[2] - 4.0 * Q[3]
              - hQp[0] - 9.0 * hQp[1] + 9.0 * hQp[2] + hQp[3]) / 4.0;
}

/* ------------------------------------------------------------------ */
/* Sec. 3.3: candidate polynomials.  Coordinates are xi = (x - x_i)/h, cell
 * I_k = [k-1/2, k+1/2], the interface x_{i+1/2} is xi = 1/2.  A polynomial
 * is fixed by cell averages and cell-averaged slopes (Eq. compact-deriv),
 * i.e. for a slope datum h*Q'_k = q(k+1/2) - q(k-1/2).
 * Stencil data vector s = (Q_{i-1}, Q_i, Q_{i+1}, Q_{i+2},
 *                          hQ'_{i-1}, hQ'_i, hQ'_{i+1}, hQ'_{i+2}).        */
#define NPOLY 8          /* q0..q6 and the cubic q~1 (index 7) */
#define MAXDEG 4

typedef struct { int deg; int ncon; int kind[5]; int cell[5]; } poly_def;
/* kind 0 = cell average, kind 1 = cell-averaged slope; cell in -1..2 */
static const poly_def POLY_DEFS[NPOLY] = {
    {2, 3, {0, 0, 1}, {-1, 0, -1}},                 /* S0 = {Q_i-1, Q_i, Q'_i-1}            */
    {2, 3, {0, 0, 0}, {-1, 0, 1}},                  /* S1 = {Q_i-1, Q_i, Q_i+1}             */
    {3, 4, {0, 0, 0, 1}, {0, 1, 2, 2}},             /* S2 = {Q_i, Q_i+1, Q_i+2, Q'_i+2}     */
    {2, 3, {0, 0, 0}, {-1, 0, 1}},                  /* S3 = {Q_i-1, Q_i, Q_i+1}             */
    {2, 3, {0, 0, 0}, {0, 1, 2}},                   /* S4 = {Q_i, Q_i+1, Q_i+2}             */
    {4, 5, {0, 0, 0, 1, 1}, {-1, 0, 1, -1, 0}},     /* S5 = {Q_i-1,Q_i,Q_i+1,Q'_i-1,Q'_i}   */
    {4, 5, {0, 0, 0, 1, 1}, {0, 1, 2, 1, 2}},       /* S6 = {Q_i,Q_i+1,Q_i+2,Q'_i+1,Q'_i+2} */
    {3, 4, {0, 0, 0, 1}, {-1, 0, 1, -1}},           /* S~1 = {Q_i-1,Q_i,Q_i+1,Q'_i-1}       */
};

/* coefficient maps: coef[p][m][s] gives monomial coefficient m of poly p as
 * a linear combination of the 8 stencil data                              */
static double COEF[NPOLY][MAXDEG + 1][8];
static int COEF_READY = 0;

/* Compact 6th-order variant (Sec. 3.2 names it; its formulas are not printed).
 * Reading: the degree-5 polynomial whose averages over I_i-1..I_i+2 are
 * Q_i-1..Q_i+2 and whose cell-averaged slopes over I_i and I_i+1 are Q'_i and
 * Q'_i+1 -- the same stencil as P7 without the two outer slopes.
 * LIN6[r][s]: h^r times the r-th derivative of that polynomial at x_{i+1/2},
 * as the weight of stencil datum s (r = 0, 1, 2).                           */
static const int LIN6_KIND[6] = {0, 0, 0, 0, 1, 1};
static const int LIN6_CELL[6] = {-1, 0, 1, 2, 0, 1};
static double LIN6[3][8];

static double ipow(double x, int m) { double r = 1.0; for (int k = 0; k < m; ++k) r *= x; return r; }

static void solve_dense(int n, double *A, double *b)   /* Gaussian elimination, partial pivoting */
{
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r) if (fabs(A[r * n + c]) > fabs(A[piv * n + c])) piv = r;
        if (piv != c) {
            for (int k = 0; k < n; ++k) { double t = A[c * n + k]; A[c * n + k] = A[piv * n + k]; A[piv * n + k] = t; }
            double t = b[c]; b[c] = b[piv]; b[piv] = t;
        }
        for (int r = c + 1; r < n; ++r) {
            double f = A[r * n + c] / A[c * n + c];
            if (f == 0.0) continue;
            for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int k = r + 1; k < n; ++k) s -= A[r * n + k] * b[k];
        b[r] = s / A[r * n + r];
    }
}

static void build_coef(void)
{
    if (COEF_READY) return;
    memset(COEF, 0, sizeof(COEF));
    for (int p = 0; p < NPOLY; ++p) {
        const poly_def *d = &POLY_DEFS[p];
        int n = d->ncon;
        for (int sidx = 0; sidx < 8; ++sidx) {
            double A[25], b[5];
            for (int r = 0; r < n; ++r) {
                double lo = d->cell[r] - 0.5, hi = d->cell[r] + 0.5;
                for (int m = 0; m < n; ++m) {
                    if (d->kind[r] == 0) A[r * n + m] = (ipow(hi, m + 1) - ipow(lo, m + 1)) / (m + 1);
                    else A[r * n + m] = ipow(hi, m) - ipow(lo, m);
                }
                int datum = (d->kind[r] == 0 ? 0 : 4) + d->cell[r] + 1;
                b[r] = (datum == sidx) ? 1.0 : 0.0;
            }
            solve_dense(n, A, b);
            for (int m = 0; m < n; ++m) COEF[p][m][sidx] = b[m];
        }
    }
    /* the degree-5 fit of the 6th-order variant, solved per datum the same way */
    for (int sidx = 0; sidx < 8; ++sidx) {
        double A[36], b[6];
        for (int r = 0; r < 6; ++r) {
            double lo = LIN6_CELL[r] - 0.5, hi = LIN6_CELL[r] + 0.5;
            for (int m = 0; m < 6; ++m) {
                if (LIN6_KIND[r] == 0) A[r * 6 + m] = (ipow(hi, m + 1) - ipow(lo, m + 1)) / (m + 1);
                else A[r * 6 + m] = ipow(hi, m) - ipow(lo, m);
            }
            int datum = (LIN6_KIND[r] == 0 ? 0 : 4) + LIN6_CELL[r] + 1;
            b[r] = (datum == sidx) ? 1.0 : 0.0;
        }
        solve_dense(6, A, b);
        double v = 0.0, d1 = 0.0, d2 = 0.0;
        for (int m = 0; m < 6; ++m) v += b[m] * ipow(0.5, m);
        for (int m = 1; m < 6; ++m) d1 += m * b[m] * ipow(0.5, m - 1);
        for (int m = 2; m < 6; ++m) d2 += m * (m - 1) * b[m] * ipow(0.5, m - 2);
        LIN6[0][sidx] = v; LIN6[1][sidx] = d1; LIN6[2][sidx] = d2;
    }
    COEF_READY = 1;
}

/* monomial coefficients of polynomial p for stencil data s */
static void poly_coeffs(int p, const double s[8], double c[MAXDEG + 1])
{
    for (int m = 0; m <= MAXDEG; ++m) {
        double acc = 0.0;
        for (int k = 0; k < 8; ++k) acc += COEF[p][m][k] * s[k];
        c[m] = acc;
    }
}

/* value q(1/2) and scaled slope h*q'(1/2) at the interface */
static void poly_at_interface(int deg, const double c[MAXDEG + 1], double *val, double *slope)
{
    double v = 0.0, sl = 0.0;
    for (int m = 0; m <= deg; ++m) v += c[m] * ipow(0.5, m);
    for (int m = 1; m <= deg; ++m) sl += m * c[m] * ipow(0.5, m - 1);
    *val = v; *slope = sl;
}

/* Eq. (smooth-indicator): beta = sum_{r=1}^{deg} int_{I_i} (d^r q/dxi^r)^2 dxi
 * (the h^{2r-1} factors cancel in xi units), integrated exactly            */
static double poly_beta(int deg, const double c[MAXDEG + 1])
{
    double d[MAXDEG + 1];
    for (int m = 0; m <= deg; ++m) d[m] = c[m];
    double beta = 0.0;
    for (int r = 1; r <= deg; ++r) {
        /* differentiate once */
        for (int m = 0; m < deg; ++m) d[m] = (m + 1) * d[m + 1];
        d[deg] = 0.0;
        int dd = deg - r;
        for (int m = 0; m <= dd; ++m)
            for (int n = 0; n <= dd; ++n) {
                int e = m + n;
                double integ = (ipow(0.5, e + 1) - ipow(-0.5, e + 1)) / (e + 1);
                beta += d[m] * d[n] * integ;
            }
    }
    return beta;
}

/* exported for the pin tests: coefficient map of polynomial p */
void oc_poly_coef_matrix(int p, double out[(MAXDEG + 1) * 8])
{
    build_coef();
    for (int m = 0; m <= MAXDEG; ++m) for (int k = 0; k < 8; ++k) out[m * 8 + k] = COEF[p][m][k];
}

/* Sec. 3.3: linear weights d^8_k */
static const double DLIN[7] = {3.0 / 98.0, 5.0 / 98.0, 4.0 / 49.0, 7.0 / 98.0, 7.0 / 98.0, 17.0 / 49.0, 17.0 / 49.0};

/* Linear weights of the 6th-order variant (not printed).  Reading: the d_k
 * for which sum_k d_k q_k(x_{i+1/2}) is the interface value of the degree-5
 * fit above for all data.  That fixes every weight but the split between q_1
 * and q_3 (equal point values, different indicators); the split is the one
 * the printed d^8 has: q_0 and q_1 combine into the mirror image of q_2
 * (d_0 + d_1 = d_2, d_0 : d_1 = 3 : 5), d_3 = d_4, d_5 = d_6.               */
static const double DLIN6[7] = {3.0 / 70.0, 5.0 / 70.0, 8.0 / 70.0, 7.0 / 70.0, 7.0 / 70.0, 20.0 / 70.0, 20.0 / 70.0};

static const double *linear_weights(int order) { return order == 6 ? DLIN6 : DLIN; }

/* exported for the pin tests */
void oc_linear_weights(int order, double out[7])
{
    const double *d = linear_weights(order);
    for (int k = 0; k < 7; ++k) out[k] = d[k];
}

/* linear reconstruction of either order: out = (P, h P_x, h^2 P_xx) at x_{i+1/2} */
void oc_linear_recon_order(int order, const double Q[4], const double hQp[4], double out[3])
{
    if (order != 6) { oc_linear_recon(Q, hQp, out); return; }
    build_coef();
    for (int r = 0; r < 3; ++r) {
        double acc = 0.0;
        for (int c = 0; c < 4; ++c) acc += LIN6[r][c] * Q[c] + LIN6[r][4 + c] * hQp[c];
        out[r] = acc;
    }
}

/* Sec. 3.3: left value at x_{i+1/2} and its scaled slope h*dQ/dx with the
 * linear weights of the given order.
 * diag (may be NULL): q[7], qs[7], beta[7], delta[7]                    */
void oc_weno_left_order(int order, const double s[8], double eps, double *val, double *hslope, double *diag)
{
    const double *dlin = linear_weights(order);
    build_coef();
    double q[7], qs[7], beta[7], c[MAXDEG + 1];
    for (int k = 0; k < 7; ++k) {
        poly_coeffs(k, s, c);
        poly_at_interface(POLY_DEFS[k].deg, c, &q[k], &qs[k]);
        beta[k] = poly_beta(POLY_DEFS[k].deg, c);
    }
    /* beta_1 is replaced by the indicator of the cubic on S~1 */
    poly_coeffs(7, s, c);
    beta[1] = poly_beta(POLY_DEFS[7].deg, c);
    /* Eq. (tau): global reference */
    double Z = fabs(3.0 * (beta[0] - beta[4]) + (beta[4] - beta[3]));
    /* Eq. (WENO-Z-w) */
    double alpha[7], asum = 0.0;
    for (int k = 0; k < 7; ++k) { alpha[k] = dlin[k] * (1.0 + Z / (beta[k] + eps)); asum += alpha[k]; }
    double v = 0.0, sl = 0.0, delta[7];
    for (int k = 0; k < 7; ++k) { delta[k] = alpha[k] / asum; v += delta[k] * q[k]; sl += delta[k] * qs[k]; }
    *val = v; *hslope = sl;
    if (diag) {
        for (int k = 0; k < 7; ++k) { diag[k] = q[k]; diag[7 + k] = qs[k]; diag[14 + k] = beta[k]; diag[21 + k] = delta[k]; }
    }
}

/* right value at x_{i+1/2}: the left procedure on the mirrored stencil */
void oc_weno_right_order(int order, const double s[8], double eps, double *val, double *hslope)
{
    double m[8] = {s[3], s[2], s[1], s[0], -s[7], -s[6], -s[5], -s[4]};
    double v, sl;
    oc_weno_left_order(order, m, eps, &v, &sl, NULL);
    *val = v; *hslope = -sl;
}

/* the 8th-order scheme of the paper */
void oc_weno_left(const double s[8], double eps, double *val, double *hslope, double *diag)
{
    oc_weno_left_order(8, s, eps, val, hslope, diag);
}

void oc_weno_right(const double s[8], double eps, double *val, double *hslope)
{
    oc_weno_right_order(8, s, eps, val, hslope);
}

/* ------------------------------------------------------------------ */
/* Sec. 2.1: Maxwellian moments.  For a Maxwellian (rho, U, V, lambda) with
 * K internal degrees of freedom, <u^a v^b xi^{2c}> factorises; the u-moments
 * may be taken over the whole line or a half line.                       */
#define NMOM 9
typedef struct {
    double mu[NMOM];   /* <u^n> (full or half line) */
    double mv[NMOM];   /* <v^n> full line           */
    double mxi[3];     /* <xi^0>, <xi^2>, <xi^4>     */
} moments;

/* half: 0 full, +1 u>0, -1 u<0 */
void oc_moments_u(double U, double lam, int half, double out[NMOM])
{
    if (half == 0) { out[0] = 1.0; out[1] = U; }
    else {
        double s = sqrt(lam);
        double e = exp(-lam * U * U) / (2.0 * sqrt(M_PI * lam));
        if (half > 0) { out[0] = 0.5 * erfc(-s * U); out[1] = U * out[0] + e; }
        else          { out[0] = 0.5 * erfc(s * U);  out[1] = U * out[0] - e; }
    }
    for (int n = 0; n + 2 < NMOM; ++n) out[n + 2] = U * out[n + 1] + (n + 1) / (2.0 * lam) * out[n];
}

static void make_moments(double U, double V, double lam, double K, int half, moments *m)
{
    oc_moments_u(U, lam, half, m->mu);
    oc_moments_u(V, lam, 0, m->mv);
    m->mxi[0] = 1.0;
    m->mxi[1] = K / (2.0 * lam);
    m->mxi[2] = (K * K + 2.0 * K) / (4.0 * lam * lam);
}

/* psi as a list of monomials u^a v^b xi^{2c}, Eq. (compatibility) */
typedef struct { int n; double coef[3]; int a[3], b[3], c[3]; } psi_poly;
static void psi_def(int D, int k, psi_poly *p)
{
    memset(p, 0, sizeof(*p));
    int nv = D + 2;
    if (k == 0) { p->n = 1; p->coef[0] = 1.0; }
    else if (k == 1) { p->n = 1; p->coef[0] = 1.0; p->a[0] = 1; }
    else if (D == 2 && k == 2) { p->n = 1; p->coef[0] = 1.0; p->b[0] = 1; }
    else if (k == nv - 1) {
        if (D == 2) { p->n = 3; p->coef[0] = p->coef[1] = p->coef[2] = 0.5; p->a[0] = 2; p->b[1] = 2; p->c[2] = 1; }
        else { p->n = 2; p->coef[0] = p->coef[1] = 0.5; p->a[0] = 2; p->c[1] = 1; }
    }
}

static double mono(const moments *m, int a, int b, int c) { return m->mu[a] * m->mv[b] * m->mxi[c]; }

/* out_k = < u^a0 v^b0 psi_k > */
static void mom_psi(int D, const moments *m, int a0, int b0, double *out)
{
    int nv = D + 2;
    for (int k = 0; k < nv; ++k) {
        psi_poly pk; psi_def(D, k, &pk);
        double acc = 0.0;
        for (int i = 0; i < pk.n; ++i) acc += pk.coef[i] * mono(m, a0 + pk.a[i], b0 + pk.b[i], pk.c[i]);
        out[k] = acc;
    }
}

/* out_k = < u^a0 v^b0 psi_k (sum_l coef_l psi_l) > */
static void mom_psi_poly(int D, const moments *m, int a0, int b0, const double *cf, double *out)
{
    int nv = D + 2;
    for (int k = 0; k < nv; ++k) {
        psi_poly pk; psi_def(D, k, &pk);
        double acc = 0.0;
        for (int l = 0; l < nv; ++l) {
            if (cf[l] == 0.0) continue;
            psi_poly pl; psi_def(D, l, &pl);
            double s = 0.0;
            for (int i = 0; i < pk.n; ++i)
                for (int j = 0; j < pl.n; ++j)
                    s += pk.coef[i] * pl.coef[j] *
                         mono(m, a0 + pk.a[i] + pl.a[j], b0 + pk.b[i] + pl.b[j], pk.c[i] + pl.c[j]);
            acc += cf[l] * s;
        }
        out[k] = acc;
    }
}

/* solve (< psi psi^T >) a = rhs for the micro-slope coefficients a */
static void solve_slope(int D, const moments *m, const double *rhs, double *a)
{
    int nv = D + 2;
    double M[16], b[4];
    for (int l = 0; l < nv; ++l) {
        double e[4] = {0, 0, 0, 0}; e[l] = 1.0;
        double col[4];
        mom_psi_poly(D, m, 0, 0, e, col);
        for (int k = 0; k < nv; ++k) M[k * nv + l] = col[k];
    }
    for (int k = 0; k < nv; ++k) b[k] = rhs[k];
    solve_dense(nv, M, b);
    for (int k = 0; k < nv; ++k) a[k] = b[k];
}

/* exported for the pin tests */
void oc_mom_psi_poly(int D, double U, double V, double lam, double K, int half,
                     int a0, int b0, const double *cf, double *out)
{
    moments m; make_moments(U, V, lam, K, half, &m);
    if (cf) mom_psi_poly(D, &m, a0, b0, cf, out); else mom_psi(D, &m, a0, b0, out);
}

/* ------------------------------------------------------------------ */
/* Euler time derivatives by Cauchy-Kowalevski.  A 2nd-order Taylor jet in
 * (x, y, t) carries value, gradient and Hessian; the Euler fluxes are
 * evaluated on jets and W_t = -F_x - G_y, W_tt = -F_xt - G_yt.          */
typedef struct { double v, g[3], h[3][3]; } jet;

static jet jconst(double c) { jet r; memset(&r, 0, sizeof(r)); r.v = c; return r; }
static jet jadd(jet a, jet b) { jet r; r.v = a.v + b.v; for (int i = 0; i < 3; ++i) { r.g[i] = a.g[i] + b.g[i]; for (int j = 0; j < 3; ++j) r.h[i][j] = a.h[i][j] + b.h[i][j]; } return r; }
static jet jsub(jet a, jet b) { jet r; r.v = a.v - b.v; for (int i = 0; i < 3; ++i) { r.g[i] = a.g[i] - b.g[i]; for (int j = 0; j < 3; ++j) r.h[i][j] = a.h[i][j] - b.h[i][j]; } return r; }
static jet jscale(jet a, double s) { jet r; r.v = a.v * s; for (int i = 0; i < 3; ++i) { r.g[i] = a.g[i] * s; for (int j = 0; j < 3; ++j) r.h[i][j] = a.h[i][j] * s; } return r; }
static jet jmul(jet a, jet b)
{
    jet r; r.v = a.v * b.v;
    for (int i = 0; i < 3; ++i) {
        r.g[i] = a.v * b.g[i] + a.g[i] * b.v;
        for (int j = 0; j < 3; ++j) r.h[i][j] = a.v * b.h[i][j] + a.g[i] * b.g[j] + a.g[j] * b.g[i] + a.h[i][j] * b.v;
    }
    return r;
}
static jet jrecip(jet a)
{
    jet r; double q = 1.0 / a.v;
    r.v = q;
    for (int i = 0; i < 3; ++i) {
        r.g[i] = -q * q * a.g[i];
        for (int j = 0; j < 3; ++j) r.h[i][j] = -q * q * a.h[i][j] + 2.0 * q * q * q * a.g[i] * a.g[j];
    }
    return r;
}

/* Euler fluxes on jets (normal x, tangential y); nv = D+2 */
static void euler_flux_jet(int D, double gamma, const jet *W, jet *F, jet *G)
{
    jet rho = W[0], m = W[1], E = W[D + 1];
    jet ir = jrecip(rho);
    jet U = jmul(m, ir);
    if (D == 1) {
        jet p = jscale(jsub(E, jscale(jmul(m, U), 0.5)), gamma - 1.0);
        F[0] = m; F[1] = jadd(jmul(m, U), p); F[2] = jmul(U, jadd(E, p));
        return;
    }
    jet n = W[2];
    jet V = jmul(n, ir);
    jet p = jscale(jsub(E, jscale(jadd(jmul(m, U), jmul(n, V)), 0.5)), gamma - 1.0);
    F[0] = m; F[1] = jadd(jmul(m, U), p); F[2] = jmul(m, V); F[3] = jmul(U, jadd(E, p));
    G[0] = n; G[1] = jmul(n, U); G[2] = jadd(jmul(n, V), p); G[3] = jmul(V, jadd(E, p));
}

/* W0, first derivatives Wx, Wy, second derivatives Wxx, Wxy, Wyy ->
 * Wt, Wtt (Euler).  D=1 ignores the y entries.                          */
void oc_euler_time_derivs(int D, double gamma, const double *W0, const double *Wx, const double *Wy,
                          const double *Wxx, const double *Wxy, const double *Wyy,
                          double *Wt, double *Wtt)
{
    int nv = D + 2;
    jet W[4], F[4], G[4];
    for (int k = 0; k < nv; ++k) {
        W[k] = jconst(W0[k]);
        W[k].g[0] = Wx[k]; W[k].h[0][0] = Wxx[k];
        if (D == 2) { W[k].g[1] = Wy[k]; W[k].h[0][1] = W[k].h[1][0] = Wxy[k]; W[k].h[1][1] = Wyy[k]; }
    }
    euler_flux_jet(D, gamma, W, F, G);
    double Wxt[4], Wyt[4];
    for (int k = 0; k < nv; ++k) {
        Wt[k] = -F[k].g[0] - (D == 2 ? G[k].g[1] : 0.0);
        Wxt[k] = -F[k].h[0][0] - (D == 2 ? G[k].h[0][1] : 0.0);
        Wyt[k] = (D == 2) ? (-F[k].h[0][1] - G[k].h[1][1]) : 0.0;
    }
    for (int k = 0; k < nv; ++k) {
        W[k].g[2] = Wt[k];
        W[k].h[0][2] = W[k].h[2][0] = Wxt[k];
        W[k].h[1][2] = W[k].h[2][1] = Wyt[k];
    }
    euler_flux_jet(D, gamma, W, F, G);
    for (int k = 0; k < nv; ++k) Wtt[k] = -F[k].h[0][2] - (D == 2 ? G[k].h[1][2] : 0.0);
}

/* ------------------------------------------------------------------ */
/* Sec. 2.1-2.2: the gas-kinetic evaluation at one interface quadrature point
 * in the face-normal frame.  Inputs (conservative, nv = D+2 entries each):
 *   equilibrium state W0 with derivatives n (normal), t (tangential), nn, nt, tt
 *   non-equilibrium left/right states with normal and tangential slopes
 * Outputs:
 *   S1 = int_0^dt F dt, S2 = int_0^{dt/2} F dt  (second-order f)
 *   Wt, Wtt  Euler time derivatives of W0
 *   NEh = NE(dt/2), NEf = NE(dt) non-equilibrium part of the interface state
 * returns 0, or OC_E_NONPHYSICAL if a state has rho<=0 or p<=0          */
typedef struct {
    double W0[4], W0n[4], W0t[4], W0nn[4], W0nt[4], W0tt[4];
    double Wl[4], Wln[4], Wlt[4], Wr[4], Wrn[4], Wrt[4];
} oc_point_in;
typedef struct { double S1[4], S2[4], Wt[4], Wtt[4], NEh[4], NEf[4], tau; } oc_point_out;

static int prim(int D, double gamma, const double *W, double *rho, double *U, double *V, double *p)
{
    *rho = W[0];
    *U = W[1] / W[0];
    *V = (D == 2) ? W[2] / W[0] : 0.0;
    double ke = 0.5 * (*rho) * ((*U) * (*U) + (*V) * (*V));
    *p = (gamma - 1.0) * (W[D + 1] - ke);
    return (*rho > 0.0 && *p > 0.0) ? 0 : OC_E_NONPHYSICAL;
}

int oc_gks_point(const oc_problem *P, int D, const oc_point_in *in, double dt, oc_point_out *out)
{
    int nv = D + 2;
    double gamma = P->gamma;
    double K = (D == 1) ? (3.0 - gamma) / (gamma - 1.0) : (4.0 - 2.0 * gamma) / (gamma - 1.0);
    double rho, U, V, p, rl, Ul, Vl, pl, rr, Ur, Vr, pr;
    if (prim(D, gamma, in->W0, &rho, &U, &V, &p)) return OC_E_NONPHYSICAL;
    if (prim(D, gamma, in->Wl, &rl, &Ul, &Vl, &pl)) return OC_E_NONPHYSICAL;
    if (prim(D, gamma, in->Wr, &rr, &Ur, &Vr, &pr)) return OC_E_NONPHYSICAL;
    double lam = rho / (2.0 * p), laml = rl / (2.0 * pl), lamr = rr / (2.0 * pr);

    /* equilibrium g0: micro slopes a_n, a_t from the derivatives, Eq. (compatibility) for A */
    moments m0; make_moments(U, V, lam, K, 0, &m0);
    double rhs[4], an[4] = {0}, at[4] = {0}, Abar[4];
    for (int k = 0; k < nv; ++k) rhs[k] = in->W0n[k] / rho;
    solve_slope(D, &m0, rhs, an);
    if (D == 2) { for (int k = 0; k < nv; ++k) rhs[k] = in->W0t[k] / rho; solve_slope(D, &m0, rhs, at); }
    double tu[4], tv[4] = {0, 0, 0, 0}, rhsA[4];
    mom_psi_poly(D, &m0, 1, 0, an, tu);
    if (D == 2) mom_psi_poly(D, &m0, 0, 1, at, tv);
    for (int k = 0; k < nv; ++k) rhsA[k] = -(tu[k] + tv[k]);
    solve_slope(D, &m0, rhsA, Abar);

    /* flux moments of the equilibrium part */
    double F0[4], T1[4], T2[4], t2u[4], t2v[4] = {0, 0, 0, 0};
    mom_psi(D, &m0, 1, 0, F0);
    mom_psi_poly(D, &m0, 1, 0, Abar, T1);
    mom_psi_poly(D, &m0, 2, 0, an, t2u);
    if (D == 2) mom_psi_poly(D, &m0, 1, 1, at, t2v);
    for (int k = 0; k < nv; ++k) { F0[k] *= rho; T1[k] *= rho; T2[k] = rho * (t2u[k] + t2v[k]); }

    /* non-equilibrium g_l (u>0) and g_r (u<0) */
    double Fh[4] = {0}, Th[4] = {0}, Wh[4] = {0}, Wsl[4] = {0};
    for (int side = 0; side < 2; ++side) {
        double rs = side ? rr : rl, Us = side ? Ur : Ul, Vs = side ? Vr : Vl, ls = side ? lamr : laml;
        const double *Wn = side ? in->Wrn : in->Wln, *Wtg = side ? in->Wrt : in->Wlt;
        moments mf, mh;
        make_moments(Us, Vs, ls, K, 0, &mf);
        make_moments(Us, Vs, ls, K, side ? -1 : +1, &mh);
        double asn[4] = {0}, ast[4] = {0}, r2[4];
        for (int k = 0; k < nv; ++k) r2[k] = Wn[k] / rs;
        solve_slope(D, &mf, r2, asn);
        if (D == 2) { for (int k = 0; k < nv; ++k) r2[k] = Wtg[k] / rs; solve_slope(D, &mf, r2, ast); }
        double f[4], tn[4], tt[4] = {0, 0, 0, 0}, w[4], wn[4], wt[4] = {0, 0, 0, 0};
        mom_psi(D, &mh, 1, 0, f);
        mom_psi_poly(D, &mh, 2, 0, asn, tn);
        if (D == 2) mom_psi_poly(D, &mh, 1, 1, ast, tt);
        mom_psi(D, &mh, 0, 0, w);
        mom_psi_poly(D, &mh, 1, 0, asn, wn);
        if (D == 2) mom_psi_poly(D, &mh, 0, 1, ast, wt);
        for (int k = 0; k < nv; ++k) {
            Fh[k] += rs * f[k];
            Th[k] += rs * (tn[k] + tt[k]);
            Wh[k] += rs * w[k];
            Wsl[k] += rs * (wn[k] + wt[k]);
        }
    }

    /* Sec. 4: collision time, enhanced by the pressure jump; for viscous flow the
     * first part is mu/p with p the pressure of the equilibrium state at the point */
    double tau = (P->mu > 0.0 ? P->mu / p : P->eps_tau * dt) + P->c_tau * fabs((pl - pr) / (pl + pr)) * dt;
    out->tau = tau;

    /* time integrals of the second-order flux over [0, dt] and [0, dt/2] */
    for (int w = 0; w < 2; ++w) {
        double D_ = (w == 0) ? dt : 0.5 * dt;
        double e = (tau > 0.0) ? exp(-D_ / tau) : 0.0;
        double c1 = D_ - tau * (1.0 - e);
        double c2 = 0.5 * D_ * D_;
        double c3 = -tau * D_;
        double c4 = tau * tau - tau * (D_ + tau) * e;
        double c5 = tau * (1.0 - e);
        double *S = (w == 0) ? out->S1 : out->S2;
        for (int k = 0; k < nv; ++k)
            S[k] = c1 * F0[k] + c2 * T1[k] + c3 * (T2[k] + T1[k]) + c4 * (T2[k] - Th[k]) + c5 * Fh[k];
    }

    /* interface state: Euler time derivatives and the non-equilibrium part */
    double Wy[4] = {0}, Wxy[4] = {0}, Wyy[4] = {0};
    if (D == 2) for (int k = 0; k < nv; ++k) { Wy[k] = in->W0t[k]; Wxy[k] = in->W0nt[k]; Wyy[k] = in->W0tt[k]; }
    oc_euler_time_derivs(D, gamma, in->W0, in->W0n, Wy, in->W0nn, Wxy, Wyy, out->Wt, out->Wtt);
    for (int w = 0; w < 2; ++w) {
        double t = (w == 0) ? 0.5 * dt : dt;
        double e = (tau > 0.0) ? exp(-t / tau) : 0.0;
        double *NE = (w == 0) ? out->NEh : out->NEf;
        for (int k = 0; k < nv; ++k)
            NE[k] = e * ((Wh[k] - t * Wsl[k]) - in->W0[k] - t * out->Wt[k]);
    }
    return OC_OK;
}

/* ------------------------------------------------------------------ */
/* ghost cells: 2 layers, arrays with (nx+4) x (ny+4) entries per plane   */
#define NG 2

static void prim_to_cons(int D, double gamma, const double *q, double *W)
{
    /* q = rho, u, v, p */
    W[0] = q[0];
    W[1] = q[0] * q[1];
    if (D == 2) { W[2] = q[0] * q[2]; W[3] = q[3] / (gamma - 1.0) + 0.5 * q[0] * (q[1] * q[1] + q[2] * q[2]); }
    else W[2] = q[3] / (gamma - 1.0) + 0.5 * q[0] * q[1] * q[1];
}

/* E: extended planes [12][(ny+4)][(nx+4)], interior copied from W.  halo (for
 * BC_HALO x-sides): [side][12][NG][ny], ghost column -1-m (low) or nx+m (high) */
static void fill_ghosts2d(const oc_problem *P, double *E, const double *halo)
{
    int nx = P->nx, ny = P->ny, X = nx + 2 * NG, Y = ny + 2 * NG;
    size_t PL = (size_t)X * Y;
    double inflow_cons[4][4];
    for (int side = 0; side < 4; ++side) prim_to_cons(2, P->gamma, P->inflow[side], inflow_cons[side]);
#define AT(p, j, i) E[(size_t)(p) * PL + (size_t)((j) + NG) * X + ((i) + NG)]
    /* x-ghosts for the real rows */
    for (int j = 0; j < ny; ++j)
        for (int side = 0; side < 2; ++side)
            for (int m = 0; m < NG; ++m) {
                int g = side ? nx + m : -1 - m;
                int bc = P->bc[side];
                for (int p = 0; p < 12; ++p) {
                    int var = p & 3, grp = p >> 2;   /* grp 0 W, 1 W_x, 2 W_y */
                    double v = 0.0;
                    if (bc == BC_PERIODIC) v = AT(p, j, side ? m % nx : ((nx - 1 - m) % nx + nx) % nx);
                    else if (bc == BC_REFLECT) {
                        int src = side ? nx - 1 - m : m;
                        v = AT(p, j, src);
                        int odd = (grp == 0 && var == 1) || (grp == 1 && var != 1) || (grp == 2 && var == 1);
                        if (odd) v = -v;
                    } else if (bc == BC_INFLOW) v = (grp == 0) ? inflow_cons[side][var] : 0.0;
                    else if (bc == BC_HALO) v = halo[(((size_t)side * 12 + p) * NG + m) * ny + j];
                    else { int src = side ? nx - 1 : 0; v = (grp == 1) ? 0.0 : AT(p, j, src); }
                    AT(p, j, g) = v;
                }
            }
    /* y-ghosts for every column, including the x-ghost columns (corners) */
    for (int i = -NG; i < nx + NG; ++i)
        for (int side = 0; side < 2; ++side)
            for (int m = 0; m < NG; ++m) {
                int g = side ? ny + m : -1 - m;
                int bc = P->bc[2 + side];
                for (int p = 0; p < 12; ++p) {
                    int var = p & 3, grp = p >> 2;
                    double v = 0.0;
                    if (bc == BC_PERIODIC) {
                        int src = side ? m % ny : ((ny - 1 - m) % ny + ny) % ny;
                        v = AT(p, src, i);
                    } else if (bc == BC_REFLECT) {
                        int src = side ? ny - 1 - m : m;
                        v = AT(p, src, i);
                        int odd = (grp == 0 && var == 2) || (grp == 1 && var == 2) || (grp == 2 && var != 2);
                        if (odd) v = -v;
                    } else if (bc == BC_INFLOW) v = (grp == 0) ? inflow_cons[2 + side][var] : 0.0;
                    else { int src = side ? ny - 1 : 0; v = (grp == 2) ? 0.0 : AT(p, src, i); }
                    AT(p, g, i) = v;
                }
            }
#undef AT
}

/* Sec. 4: CFL time step */
double oc_cfl_dt(const oc_problem *P, const double *W)
{
    int D = P->dim, nx = P->nx, ny = (D == 2) ? P->ny : 1;
    size_t PL = (size_t)nx * ny;
    double best = INFINITY;
    for (size_t c = 0; c < PL; ++c) {
        double Wc[4];
        for (int k = 0; k < D + 2; ++k) Wc[k] = W[k * PL + c];
        double rho, U, V, p;
        if (prim(D, P->gamma, Wc, &rho, &U, &V, &p)) return -1.0;
        double a = sqrt(P->gamma * p / rho);
        /* viscous flow: the signal speed gains 2 nu / dx (explicit diffusion limit) */
        double nu = P->mu / rho;
        double d = P->dx / (fabs(U) + a + 2.0 * nu / P->dx);
        if (D == 2) { double dy = P->dy / (fabs(V) + a + 2.0 * nu / P->dy); if (dy < d) d = dy; }
        if (d < best) best = d;
    }
    return P->cfl * best;
}

/* ------------------------------------------------------------------ */
/* per-face results of one stage */
typedef struct { double Fb[4], Ft[4], Wm[4], B[4], Wtt[4]; } face_res;

static void face_from_point(int nv, double dt, const double *W0, const oc_point_out *o, double w,
                            face_res *r, int accumulate)
{
    for (int k = 0; k < nv; ++k) {
        double Fb = (4.0 * o->S2[k] - o->S1[k]) / dt;
        double Ft = 4.0 * (o->S1[k] - 2.0 * o->S2[k]) / (dt * dt);
        double Wm = W0[k] + 0.5 * dt * o->Wt[k] + 0.125 * dt * dt * o->Wtt[k] + o->NEh[k];
        double B = W0[k] + dt * o->Wt[k] + dt * dt / 6.0 * o->Wtt[k] + o->NEf[k];
        if (!accumulate) { r->Fb[k] = 0; r->Ft[k] = 0; r->Wm[k] = 0; r->B[k] = 0; r->Wtt[k] = 0; }
        r->Fb[k] += w * Fb; r->Ft[k] += w * Ft; r->Wm[k] += w * Wm; r->B[k] += w * B; r->Wtt[k] += w * o->Wtt[k];
    }
}

/* ------------------------------------------------------------------ */
/* 1D: planes [6][nx]: rho, rhoU, rhoE, then their cell-averaged x-gradients */
static void fill_ghosts1d(const oc_problem *P, const double *W, double *E)
{
    int nx = P->nx, X = nx + 2 * NG;
    double ic[2][3];
    for (int side = 0; side < 2; ++side) {
        double q[4] = {P->inflow[side][0], P->inflow[side][1], 0.0, P->inflow[side][3]};
        prim_to_cons(1, P->gamma, q, ic[side]);
    }
    for (int p = 0; p < 6; ++p) for (int i = 0; i < nx; ++i) E[p * X + i + NG] = W[p * nx + i];
    for (int side = 0; side < 2; ++side)
        for (int m = 0; m < NG; ++m) {
            int g = side ? nx + m : -1 - m;
            for (int p = 0; p < 6; ++p) {
                int var = p % 3, grp = p / 3;
                double v;
                int bc = P->bc[side];
                if (bc == BC_PERIODIC) v = E[p * X + (side ? m : nx - 1 - m) + NG];
                else if (bc == BC_REFLECT) {
                    v = E[p * X + (side ? nx - 1 - m : m) + NG];
                    int odd = (grp == 0 && var == 1) || (grp == 1 && var != 1);
                    if (odd) v = -v;
                } else if (bc == BC_INFLOW) v = (grp == 0) ? ic[side][var] : 0.0;
                else v = (grp == 1) ? 0.0 : E[p * X + (side ? nx - 1 : 0) + NG];
                E[p * X + g + NG] = v;
            }
        }
}

/* Sec. 3.2 allows the reconstruction in characteristic variables.  For the
 * nonlinear reconstruction at a face the stencil data are projected on the
 * eigenvectors of the normal Euler flux Jacobian at the arithmetic mean of the
 * two cells sharing the face: right eigenvectors R as columns (eigenvalues
 * U-c, U (entropy), [U (shear) in 2D], U+c), left eigenvectors = R^{-1} by
 * elimination.  nv = 3 (1D: rho, m, E) or 4 (face frame: rho, m_n, m_t, E). */
static void char_basis(int D, double gamma, const double *Wref, double *R, double *Linv)
{
    int nv = D + 2;
    double rho = Wref[0], U = Wref[1] / rho, V = (D == 2) ? Wref[2] / rho : 0.0;
    double q2 = U * U + V * V;
    double p = (gamma - 1.0) * (Wref[nv - 1] - 0.5 * rho * q2);
    double c = sqrt(gamma * p / rho), H = (Wref[nv - 1] + p) / rho;
    memset(R, 0, sizeof(double) * nv * nv);
    /* column 0: U - c */
    R[0 * nv + 0] = 1.0; R[1 * nv + 0] = U - c; if (D == 2) R[2 * nv + 0] = V; R[(nv - 1) * nv + 0] = H - U * c;
    /* column 1: entropy wave */
    R[0 * nv + 1] = 1.0; R[1 * nv + 1] = U; if (D == 2) R[2 * nv + 1] = V; R[(nv - 1) * nv + 1] = 0.5 * q2;
    if (D == 2) { /* column 2: shear wave */
        R[2 * nv + 2] = 1.0; R[3 * nv + 2] = V;
    }
    /* last column: U + c */
    R[0 * nv + nv - 1] = 1.0; R[1 * nv + nv - 1] = U + c; if (D == 2) R[2 * nv + nv - 1] = V;
    R[(nv - 1) * nv + nv - 1] = H + U * c;
    for (int col = 0; col < nv; ++col) {
        double A[16], b[4];
        memcpy(A, R, sizeof(double) * nv * nv);
        for (int k = 0; k < nv; ++k) b[k] = (k == col) ? 1.0 : 0.0;
        solve_dense(nv, A, b);
        for (int k = 0; k < nv; ++k) Linv[k * nv + col] = b[k];
    }
}

/* exported for the pin tests */
void oc_char_basis(int D, double gamma, const double *Wref, double *R, double *Linv)
{
    char_basis(D, gamma, Wref, R, Linv);
}

/* nonlinear reconstruction of all nv variables of one face row.  Q[k][c] and
 * hQp[k][c]: variable k, stencil cell c (i-1..i+2).  Outputs per variable. */
static void weno_row(const oc_problem *P, int D, double Q[4][4], double hQp[4][4],
                     double *vl, double *sl, double *vr, double *sr)
{
    int nv = D + 2;
    if (P->recon_vars == 0) {
        for (int k = 0; k < nv; ++k) {
            double s[8];
            for (int c = 0; c < 4; ++c) { s[c] = Q[k][c]; s[4 + c] = hQp[k][c]; }
            oc_weno_left_order(recon_order(P), s, P->weno_eps, &vl[k], &sl[k], NULL);
            oc_weno_right_order(recon_order(P), s, P->weno_eps, &vr[k], &sr[k]);
        }
        return;
    }
    double Wref[4], R[16], L[16];
    for (int k = 0; k < nv; ++k) Wref[k] = 0.5 * (Q[k][1] + Q[k][2]);
    char_basis(D, P->gamma, Wref, R, L);
    double cvl[4], csl[4], cvr[4], csr[4];
    for (int m = 0; m < nv; ++m) {
        double s[8];
        for (int c = 0; c < 4; ++c) {
            double a = 0.0, b = 0.0;
            for (int k = 0; k < nv; ++k) { a += L[m * nv + k] * Q[k][c]; b += L[m * nv + k] * hQp[k][c]; }
            s[c] = a; s[4 + c] = b;
        }
        oc_weno_left_order(recon_order(P), s, P->weno_eps, &cvl[m], &csl[m], NULL);
        oc_weno_right_order(recon_order(P), s, P->weno_eps, &cvr[m], &csr[m]);
    }
    for (int k = 0; k < nv; ++k) {
        vl[k] = sl[k] = vr[k] = sr[k] = 0.0;
        for (int m = 0; m < nv; ++m) {
            vl[k] += R[k * nv + m] * cvl[m]; sl[k] += R[k * nv + m] * csl[m];
            vr[k] += R[k * nv + m] * cvr[m]; sr[k] += R[k * nv + m] * csr[m];
        }
    }
}

static int face1d(const oc_problem *P, const double *E, int f, double dt, face_res *r)
{
    int X = P->nx + 2 * NG;
    double h = P->dx;
    oc_point_in in; memset(&in, 0, sizeof(in));
    double Q[4][4], hQp[4][4], vl[4], sl[4], vr[4], sr[4];
    for (int k = 0; k < 3; ++k) {
        double lin[3];
        for (int c = 0; c < 4; ++c) {
            int cell = f - 2 + c;
            Q[k][c] = E[k * X + cell + NG];
            hQp[k][c] = h * E[(3 + k) * X + cell + NG];
        }
        oc_linear_recon_order(recon_order(P), Q[k], hQp[k], lin);
        in.W0[k] = lin[0]; in.W0n[k] = lin[1] / h; in.W0nn[k] = lin[2] / (h * h);
    }
    weno_row(P, 1, Q, hQp, vl, sl, vr, sr);
    for (int k = 0; k < 3; ++k) {
        in.Wl[k] = vl[k]; in.Wln[k] = sl[k] / h;
        in.Wr[k] = vr[k]; in.Wrn[k] = sr[k] / h;
    }
    oc_point_out o;
    if (oc_gks_point(P, 1, &in, dt, &o)) return OC_E_NONPHYSICAL;
    face_from_point(3, dt, in.W0, &o, 1.0, r, 0);
    return OC_OK;
}

static int step1d(const oc_problem *P, double *W, double dt)
{
    int nx = P->nx, X = nx + 2 * NG;
    double dx = P->dx;
    double *E = calloc((size_t)6 * X, sizeof(double));
    double *Ws = malloc((size_t)6 * nx * sizeof(double));
    double *R = malloc((size_t)6 * nx * sizeof(double));
    face_res *fr = malloc((size_t)(nx + 1) * sizeof(face_res));
    int err = 0;
    /* stage 1 */
    fill_ghosts1d(P, W, E);
#pragma omp parallel for reduction(| : err) if (nx >= 4096)
    for (int f = 0; f <= nx; ++f) err |= face1d(P, E, f, dt, &fr[f]);
    if (err) goto done;
    for (int i = 0; i < nx; ++i)
        for (int k = 0; k < 3; ++k) {
            const face_res *L = &fr[i], *Rf = &fr[i + 1];
            Ws[k * nx + i] = W[k * nx + i] - ((0.5 * dt * Rf->Fb[k] + 0.125 * dt * dt * Rf->Ft[k])
                                              - (0.5 * dt * L->Fb[k] + 0.125 * dt * dt * L->Ft[k])) / dx;
            Ws[(3 + k) * nx + i] = (Rf->Wm[k] - L->Wm[k]) / dx;
            R[k * nx + i] = W[k * nx + i] - ((dt * Rf->Fb[k] + dt * dt / 6.0 * Rf->Ft[k])
                                             - (dt * L->Fb[k] + dt * dt / 6.0 * L->Ft[k])) / dx;
            R[(3 + k) * nx + i] = (Rf->B[k] - L->B[k]) / dx;
        }
    /* stage 2 */
    fill_ghosts1d(P, Ws, E);
#pragma omp parallel for reduction(| : err) if (nx >= 4096)
    for (int f = 0; f <= nx; ++f) err |= face1d(P, E, f, dt, &fr[f]);
    if (err) goto done;
    for (int i = 0; i < nx; ++i)
        for (int k = 0; k < 3; ++k) {
            const face_res *L = &fr[i], *Rf = &fr[i + 1];
            W[k * nx + i] = R[k * nx + i] - dt * dt / 3.0 * (Rf->Ft[k] - L->Ft[k]) / dx;
            W[(3 + k) * nx + i] = R[(3 + k) * nx + i] + dt * dt / 3.0 * (Rf->Wtt[k] - L->Wtt[k]) / dx;
        }
done:
    free(E); free(Ws); free(R); free(fr);
    return err ? OC_E_NONPHYSICAL : OC_OK;
}

/* ------------------------------------------------------------------ */
/* 2D.  Normal reconstruction of one row of one face (orientation o: 0 x-face,
 * 1 y-face), in the face frame (momentum components swapped for y-faces). */
typedef struct { double V[4], N[4], NN[4], L[4], R[4], Ln[4], Rn[4]; } row_rec;

/* rotated variable index: frame component k reads physical component */
static int rot_var(int o, int k) { if (o == 0) return k; return (k == 1) ? 2 : (k == 2) ? 1 : k; }

static double ext_at(const oc_problem *P, const double *E, int p, int j, int i)
{
    int X = P->nx + 2 * NG, Y = P->ny + 2 * NG;
    return E[(size_t)p * X * Y + (size_t)(j + NG) * X + (i + NG)];
}

/* cell (c-th of the 4 normal stencil cells) of face f, row r, orientation o */
static void stencil_cell(int o, int f, int r, int c, int *i, int *j)
{
    if (o == 0) { *i = f - 2 + c; *j = r; } else { *i = r; *j = f - 2 + c; }
}

static void row_recon(const oc_problem *P, const double *E, int o, int f, int r, row_rec *out)
{
    double h = (o == 0) ? P->dx : P->dy;
    int gn = (o == 0) ? 1 : 2;   /* normal gradient group */
    double Q[4][4], hQp[4][4], vl[4], sl[4], vr[4], sr[4];
    for (int k = 0; k < 4; ++k) {
        int pv = rot_var(o, k);
        double lin[3];
        for (int c = 0; c < 4; ++c) {
            int i, j; stencil_cell(o, f, r, c, &i, &j);
            Q[k][c] = ext_at(P, E, pv, j, i);
            hQp[k][c] = h * ext_at(P, E, 4 * gn + pv, j, i);
        }
        oc_linear_recon_order(recon_order(P), Q[k], hQp[k], lin);
        out->V[k] = lin[0]; out->N[k] = lin[1] / h; out->NN[k] = lin[2] / (h * h);
    }
    weno_row(P, 2, Q, hQp, vl, sl, vr, sr);
    for (int k = 0; k < 4; ++k) {
        out->L[k] = vl[k]; out->Ln[k] = sl[k] / h;
        out->R[k] = vr[k]; out->Rn[k] = sr[k] / h;
    }
}

/* Tangential profiles along a face.  A polynomial p(eta) in eta = (y - y_j)/h_t
 * is fixed by its means over unit segments centred at integer offsets from
 * row j.  SEGFIT5 maps the five means (rows j-2..j+2) to the coefficients of
 * the quartic, SEGFIT3 the three means (rows j-1..j+1) to those of the
 * quadratic.  CAND5[k] maps the means of rows j-2+k..j+k to the quadratic on
 * those three segments (k = 0, 1, 2); CAND3[k] maps rows j-1+k..j+k to the
 * linear polynomial on those two segments (k = 0, 1).                       */
static double SEGFIT5[5][5], SEGFIT3[3][3], CAND5[3][3][3], CAND3[2][2][2];
static int SEGFIT_READY = 0;

/* coefficient map of the degree-(n-1) polynomial whose means over the unit
 * segments centred at off[0..n-1] are given: map[m][r] */
static void seg_map(int n, const int *off, double *map)
{
    for (int col = 0; col < n; ++col) {
        double A[25], b[5];
        for (int r = 0; r < n; ++r) {
            double lo = off[r] - 0.5, hi = off[r] + 0.5;
            for (int m = 0; m < n; ++m) A[r * n + m] = (ipow(hi, m + 1) - ipow(lo, m + 1)) / (m + 1);
            b[r] = (r == col) ? 1.0 : 0.0;
        }
        solve_dense(n, A, b);
        for (int m = 0; m < n; ++m) map[m * n + col] = b[m];
    }
}

static void build_segfit(void)
{
    if (SEGFIT_READY) return;
    const int o5[5] = {-2, -1, 0, 1, 2}, o3[3] = {-1, 0, 1};
    seg_map(5, o5, &SEGFIT5[0][0]);
    seg_map(3, o3, &SEGFIT3[0][0]);
    for (int k = 0; k < 3; ++k) { int o[3] = {k - 2, k - 1, k}; seg_map(3, o, &CAND5[k][0][0]); }
    for (int k = 0; k < 2; ++k) { int o[2] = {k - 1, k}; seg_map(2, o, &CAND3[k][0][0]); }
    SEGFIT_READY = 1;
}

/* value, first and second derivative (per unit eta) at eta of the profile
 * through the segment means v[0..n-1] (rows j-n/2 .. j+n/2) */
static void seg_profile(int n, const double *v, double eta, double *p, double *dp, double *d2p)
{
    double c[5] = {0, 0, 0, 0, 0};
    for (int m = 0; m < n; ++m)
        for (int r = 0; r < n; ++r) c[m] += (n == 5 ? SEGFIT5[m][r] : SEGFIT3[m][r]) * v[r];
    double a = 0.0, b = 0.0, cc = 0.0;
    for (int m = 0; m < n; ++m) a += c[m] * ipow(eta, m);
    for (int m = 1; m < n; ++m) b += m * c[m] * ipow(eta, m - 1);
    for (int m = 2; m < n; ++m) cc += m * (m - 1) * c[m] * ipow(eta, m - 2);
    *p = a; *dp = b; *d2p = cc;
}

/* exported for the pin tests: out = (p, dp/deta, d2p/deta2) at eta of the
 * profile through n = 5 or 3 segment means */
void oc_seg_profile(int n, const double *v, double eta, double out[3])
{
    build_segfit();
    seg_profile(n, v, eta, &out[0], &out[1], &out[2]);
}

/* Nonlinear point value along a face (2D reading).  WENO-Z in the form of
 * Sec. 3.3 over the n segment means v[0..n-1] (n = 5: rows j-2..j+2, three
 * quadratic candidates; n = 3: rows j-1..j+1, two linear candidates):
 *   q_k(eta)   candidate through its consecutive segments,
 *   d_k(eta)   linear weights with sum_k d_k q_k(eta) = full-stencil
 *              polynomial at eta for all data (fixed by the outermost
 *              segments, which only one candidate contains; the middle
 *              weight closes sum d_k = 1),
 *   beta_k     Eq. (smooth-indicator) of q_k over the central segment,
 *   Z          |beta_first - beta_last| (WENO-Z global reference),
 *   alpha_k    d_k (1 + Z/(beta_k + eps)),  omega_k = alpha_k / sum alpha.
 * val = sum omega_k q_k(eta); dval = sum omega_k q_k'(eta) (per unit eta).  */
void oc_tang_weno(int n, const double *v, double eta, double eps, double *val, double *dval, double *omega)
{
    build_segfit();
    int nc = n / 2 + 1, deg = n / 2;
    double q[3], dq[3], beta[3], d[3];
    for (int k = 0; k < nc; ++k) {
        double c[MAXDEG + 1] = {0, 0, 0, 0, 0};
        for (int m = 0; m <= deg; ++m)
            for (int r = 0; r <= deg; ++r)
                c[m] += (n == 5 ? CAND5[k][m][r] : CAND3[k][m][r]) * v[k + r];
        q[k] = 0.0; dq[k] = 0.0;
        for (int m = 0; m <= deg; ++m) q[k] += c[m] * ipow(eta, m);
        for (int m = 1; m <= deg; ++m) dq[k] += m * c[m] * ipow(eta, m - 1);
        beta[k] = poly_beta(deg, c);
    }
    /* weight of the first and of the last segment mean at eta in the full
     * polynomial and in the one candidate that contains that segment */
    double wf0 = 0.0, wfl = 0.0, wc0 = 0.0, wcl = 0.0;
    for (int m = 0; m < n; ++m) {
        wf0 += (n == 5 ? SEGFIT5[m][0] : SEGFIT3[m][0]) * ipow(eta, m);
        wfl += (n == 5 ? SEGFIT5[m][n - 1] : SEGFIT3[m][n - 1]) * ipow(eta, m);
    }
    for (int m = 0; m <= deg; ++m) {
        wc0 += (n == 5 ? CAND5[0][m][0] : CAND3[0][m][0]) * ipow(eta, m);
        wcl += (n == 5 ? CAND5[nc - 1][m][deg] : CAND3[nc - 1][m][deg]) * ipow(eta, m);
    }
    d[0] = wf0 / wc0;
    d[nc - 1] = wfl / wcl;
    if (nc == 3) d[1] = 1.0 - d[0] - d[2];
    double Z = fabs(beta[0] - beta[nc - 1]);
    double alpha[3], asum = 0.0;
    for (int k = 0; k < nc; ++k) { alpha[k] = d[k] * (1.0 + Z / (beta[k] + eps)); asum += alpha[k]; }
    double a = 0.0, b = 0.0;
    for (int k = 0; k < nc; ++k) {
        double w = alpha[k] / asum;
        a += w * q[k]; b += w * dq[k];
        if (omega) omega[k] = w;
    }
    *val = a; *dval = b;
}

/* face segment: rows m = -2..+2 around it (rr[0..4]) -> two Gauss points ->
 * Gauss-averaged result (in the face frame) */
static int face_segment(const oc_problem *P, const row_rec *const rr[5], int o, double dt, face_res *res)
{
    double ht = (o == 0) ? P->dy : P->dx;
    const double g = 1.0 / (2.0 * sqrt(3.0));
    for (int gp = 0; gp < 2; ++gp) {
        double eta = gp ? g : -g;
        oc_point_in in;
        for (int k = 0; k < 4; ++k) {
            double v5[5], n5[5], v3[3], p, dp, d2p, w, dw;
            for (int r = 0; r < 5; ++r) { v5[r] = rr[r]->V[k]; n5[r] = rr[r]->N[k]; }
            /* equilibrium: nonlinear value, linear tangential derivatives */
            seg_profile(5, v5, eta, &p, &dp, &d2p);
            oc_tang_weno(5, v5, eta, P->weno_eps, &w, &dw, NULL);
            in.W0[k] = w; in.W0t[k] = dp / ht; in.W0tt[k] = d2p / (ht * ht);
            /* normal derivative and its tangential derivative */
            seg_profile(5, n5, eta, &p, &dp, &d2p);
            in.W0n[k] = p; in.W0nt[k] = dp / ht;
            in.W0nn[k] = rr[2]->NN[k];
            /* non-equilibrium states: nonlinear value and tangential slope
             * from rows j-1..j+1, normal derivative from the quadratic */
            for (int r = 0; r < 3; ++r) v3[r] = rr[r + 1]->L[k];
            oc_tang_weno(3, v3, eta, P->weno_eps, &w, &dw, NULL);
            in.Wl[k] = w; in.Wlt[k] = dw / ht;
            for (int r = 0; r < 3; ++r) v3[r] = rr[r + 1]->Ln[k];
            seg_profile(3, v3, eta, &p, &dp, &d2p);
            in.Wln[k] = p;
            for (int r = 0; r < 3; ++r) v3[r] = rr[r + 1]->R[k];
            oc_tang_weno(3, v3, eta, P->weno_eps, &w, &dw, NULL);
            in.Wr[k] = w; in.Wrt[k] = dw / ht;
            for (int r = 0; r < 3; ++r) v3[r] = rr[r + 1]->Rn[k];
            seg_profile(3, v3, eta, &p, &dp, &d2p);
            in.Wrn[k] = p;
        }
        oc_point_out out;
        if (oc_gks_point(P, 2, &in, dt, &out)) return OC_E_NONPHYSICAL;
        face_from_point(4, dt, in.W0, &out, 0.5, res, gp);
    }
    return OC_OK;
}

/* one stage of face work over both orientations; results in physical frame.
 * fx: (nx+1) x ny x-faces [j*(nx+1)+f]; fy: nx x (ny+1) y-faces [f*nx+i]   */
static int faces2d(const oc_problem *P, const double *E, double dt, face_res *fx, face_res *fy)
{
    int nx = P->nx, ny = P->ny, err = 0;
    for (int o = 0; o < 2; ++o) {
        int nf = (o == 0) ? nx + 1 : ny + 1;     /* faces along the normal */
        int nr = (o == 0) ? ny : nx;             /* rows along the tangent */
        row_rec *rr = malloc((size_t)nf * (nr + 4) * sizeof(row_rec));
#pragma omp parallel for collapse(2) if (nf * nr >= 1024)
        for (int r = -2; r <= nr + 1; ++r)
            for (int f = 0; f < nf; ++f) row_recon(P, E, o, f, r, &rr[(size_t)(r + 2) * nf + f]);
#pragma omp parallel for collapse(2) reduction(| : err) if (nf * nr >= 1024)
        for (int r = 0; r < nr; ++r)
            for (int f = 0; f < nf; ++f) {
                face_res res;
                const row_rec *rows[5];
                for (int m = 0; m < 5; ++m) rows[m] = &rr[(size_t)(r + m) * nf + f];
                err |= face_segment(P, rows, o, dt, &res);
                face_res *dst = (o == 0) ? &fx[(size_t)r * (nx + 1) + f] : &fy[(size_t)f * nx + r];
                for (int k = 0; k < 4; ++k) {
                    int pv = rot_var(o, k);
                    dst->Fb[pv] = res.Fb[k]; dst->Ft[pv] = res.Ft[k]; dst->Wm[pv] = res.Wm[k];
                    dst->B[pv] = res.B[k]; dst->Wtt[pv] = res.Wtt[k];
                }
            }
        free(rr);
    }
    return err ? OC_E_NONPHYSICAL : OC_OK;
}

/* caller-supplied ghost columns of BC_HALO sides: called before each stage with
 * the state that stage reads (12 planes of nx*ny) and the halo array to fill */
typedef void (*oc_exchange_fn)(int stage, const double *state, double *halo, void *ctx);

static int step2d_ex(const oc_problem *P, double *W, double dt, oc_exchange_fn fn, void *ctx)
{
    int nx = P->nx, ny = P->ny, X = nx + 2 * NG, Y = ny + 2 * NG;
    size_t PL = (size_t)nx * ny, EPL = (size_t)X * Y;
    double dx = P->dx, dy = P->dy;
    double *E = calloc(12 * EPL, sizeof(double));
    double *Ws = malloc(12 * PL * sizeof(double));
    double *R = malloc(12 * PL * sizeof(double));
    face_res *fx = malloc((size_t)(nx + 1) * ny * sizeof(face_res));
    face_res *fy = malloc((size_t)nx * (ny + 1) * sizeof(face_res));
    double *halo = fn ? calloc((size_t)2 * 12 * NG * ny, sizeof(double)) : NULL;
    int err = 0;
    for (int stage = 0; stage < 2 && !err; ++stage) {
        const double *S = stage ? Ws : W;
        for (int p = 0; p < 12; ++p)
            for (int j = 0; j < ny; ++j)
                memcpy(&E[p * EPL + (size_t)(j + NG) * X + NG], &S[p * PL + (size_t)j * nx], nx * sizeof(double));
        if (fn) fn(stage, S, halo, ctx);
        fill_ghosts2d(P, E, halo);
        err = faces2d(P, E, dt, fx, fy);
        if (err) break;
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                for (int k = 0; k < 4; ++k) {
                    size_t c = (size_t)j * nx + i;
                    const face_res *xl = &fx[(size_t)j * (nx + 1) + i], *xr = &fx[(size_t)j * (nx + 1) + i + 1];
                    const face_res *yl = &fy[(size_t)j * nx + i], *yr = &fy[(size_t)(j + 1) * nx + i];
                    if (stage == 0) {
                        Ws[k * PL + c] = W[k * PL + c]
                            - ((0.5 * dt * xr->Fb[k] + 0.125 * dt * dt * xr->Ft[k]) - (0.5 * dt * xl->Fb[k] + 0.125 * dt * dt * xl->Ft[k])) / dx
                            - ((0.5 * dt * yr->Fb[k] + 0.125 * dt * dt * yr->Ft[k]) - (0.5 * dt * yl->Fb[k] + 0.125 * dt * dt * yl->Ft[k])) / dy;
                        Ws[(4 + k) * PL + c] = (xr->Wm[k] - xl->Wm[k]) / dx;
                        Ws[(8 + k) * PL + c] = (yr->Wm[k] - yl->Wm[k]) / dy;
                        R[k * PL + c] = W[k * PL + c]
                            - ((dt * xr->Fb[k] + dt * dt / 6.0 * xr->Ft[k]) - (dt * xl->Fb[k] + dt * dt / 6.0 * xl->Ft[k])) / dx
                            - ((dt * yr->Fb[k] + dt * dt / 6.0 * yr->Ft[k]) - (dt * yl->Fb[k] + dt * dt / 6.0 * yl->Ft[k])) / dy;
                        R[(4 + k) * PL + c] = (xr->B[k] - xl->B[k]) / dx;
                        R[(8 + k) * PL + c] = (yr->B[k] - yl->B[k]) / dy;
                    } else {
                        W[k * PL + c] = R[k * PL + c] - dt * dt / 3.0 * ((xr->Ft[k] - xl->Ft[k]) / dx + (yr->Ft[k] - yl->Ft[k]) / dy);
                        W[(4 + k) * PL + c] = R[(4 + k) * PL + c] + dt * dt / 3.0 * (xr->Wtt[k] - xl->Wtt[k]) / dx;
                        W[(8 + k) * PL + c] = R[(8 + k) * PL + c] + dt * dt / 3.0 * (yr->Wtt[k] - yl->Wtt[k]) / dy;
                    }
                }
    }
    free(E); free(Ws); free(R); free(fx); free(fy); free(halo);
    return err;
}

static int step2d(const oc_problem *P, double *W, double dt) { return step2d_ex(P, W, dt, NULL, NULL); }

/* one S2O4 step of a subdomain whose x-sides may be BC_HALO (its neighbours'
 * columns, supplied through fn before each stage); dt is the caller's (the
 * minimum of the subdomains' CFL bounds) */
int oc_step2d_halo(const oc_problem *P, double *W, double dt, oc_exchange_fn fn, void *ctx)
{
    if (P->dim != 2) return OC_E_INVAL;
    build_coef();
    build_segfit();
    return step2d_ex(P, W, dt, fn, ctx) ? OC_E_NONPHYSICAL : OC_OK;
}

/* ------------------------------------------------------------------ */
/* time loop: advance nsteps (or until t_end when t_end > 0).  W holds the
 * planes (1D: 6 x nx, 2D: 12 x ny x nx).  t and steps are updated.       */
int oc_run(const oc_problem *P, double *W, int nsteps, double t_end, double *t, long *steps, double *last_dt)
{
    if (!P || !W || P->nx < 1 || (P->dim == 2 && P->ny < 1) || (P->dim != 1 && P->dim != 2)) return OC_E_INVAL;
    build_coef();
    build_segfit();
    for (int s = 0; s < nsteps; ++s) {
        if (t_end > 0.0 && *t >= t_end) break;
        double dt = oc_cfl_dt(P, W);
        if (!(dt > 0.0)) return OC_E_NONPHYSICAL;
        if (t_end > 0.0 && *t + dt > t_end) dt = t_end - *t;
        int err = (P->dim == 1) ? step1d(P, W, dt) : step2d(P, W, dt);
        if (err) return err;
        *t += dt;
        *steps += 1;
        if (last_dt) *last_dt = dt;
    }
    return OC_OK;
}

/* number of OpenMP threads of the oracle's loops (0: leave the default) */
void oc_set_threads(int n)
{
    if (n > 0) omp_set_num_threads(n);
}

/* one step with a given dt (used by the accuracy tests with dt = C dx^2) */
int oc_step_dt(const oc_problem *P, double *W, double dt)
{
    build_coef();
    build_segfit();
    return (P->dim == 1) ? step1d(P, W, dt) : step2d(P, W, dt);
}

int oc_run_fixed_dt(const oc_problem *P, double *W, int nsteps, double dt)
{
    build_coef();
    build_segfit();
    for (int s = 0; s < nsteps; ++s) {
        int err = oc_step_dt(P, W, dt);
        if (err) return err;
    }
    return OC_OK;
}

/* one stage-1 face evaluation for the pin tests (1D) */
int oc_face1d_debug(const oc_problem *P, const double *W, int f, double dt, double *out /* 5*3 */)
{
    build_coef();
    int X = P->nx + 2 * NG;
    double *E = calloc((size_t)6 * X, sizeof(double));
    fill_ghosts1d(P, W, E);
    face_res r;
    int err = face1d(P, E, f, dt, &r);
    for (int k = 0; k < 3; ++k) { out[k] = r.Fb[k]; out[3 + k] = r.Ft[k]; out[6 + k] = r.Wm[k]; out[9 + k] = r.B[k]; out[12 + k] = r.Wtt[k]; }
    free(E);
    return err;
}

/* point-level entry for the pin tests */
int oc_gks_point_flat(const oc_problem *P, int D, const double *in /* 12*4 */, double dt, double *out /* 6*4 + 1 */)
{
    oc_point_in pi;
    memcpy(&pi, in, sizeof(pi));
    oc_point_out po;
    int err = oc_gks_point(P, D, &pi, dt, &po);
    memcpy(out, &po, sizeof(po));
    return err;
}
