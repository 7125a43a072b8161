// cgks_records.cuh -- the arithmetic of one face-row record (the record
// kernel of cgks_records.cu runs it once per face row of a grid): the stencil
// cells with the boundary conditions applied on the fly (x-boundaries first,
// then y, so the corners match the oracle's ghost layers), the linear compact
// reconstruction (Sec. 3.2, Eq. recons-8th-val) and the nonlinear WENO-Z left
// and right states with their slopes (Sec. 3.3), in conservative or
// characteristic variables.
#pragma once
#include "cgks_device.cuh"
#include "cgks_internal.h"

namespace cgks {

// plane p of ghost cell (i, j) from the value v of its source cell: kx, ky are
// map_axis's transform kinds along x and y (x first, then y)
__device__ __forceinline__ double bc_value(const GridDev& G, double v, int i, int j, int kx, int ky, int p)
{
    if (kx == 1) { if (p == 1 || p == 4 || p == 6 || p == 7 || p == 9) v = -v; }
    else if (kx == 2) v = p < 4 ? G.inflow[i < 0 ? 0 : 1][p] : 0.0;
    else if (kx == 3) { if (p >= 4 && p < 8) v = 0.0; }
    if (ky == 1) { if (p == 2 || p == 6 || p == 8 || p == 9 || p == 11) v = -v; }
    else if (ky == 2) v = p < 4 ? G.inflow[j < 0 ? 2 : 3][p] : 0.0;
    else if (ky == 3) { if (p >= 8) v = 0.0; }
    return v;
}

// plane p of cell (i, j) with the boundary conditions applied outside the grid
__device__ __forceinline__ double cell_value(const GridDev& G, const double* __restrict__ src, size_t PL, int i, int j,
                                             int p)
{
    int kx, ky;
    const int si = map_axis(i, G.nx, G.bc[0], G.bc[1], kx);
    const int sj = map_axis(j, G.ny, G.bc[2], G.bc[3], ky);
    if (!CGKS_IN_BOUNDS(si >= 0 && si < G.nx && sj >= 0 && sj < G.ny && p >= 0 && p < 12, G.ctrl)) return 0.0;
    return bc_value(G, __ldg(src + (size_t)p * PL + (size_t)sj * G.nx + si), i, j, kx, ky, p);
}

// geometry of record r of a grid: orientation, stencil start cell and step,
// frame of the variables, global record index
struct RowRef {
    bool xo, inner;
    int i0, j0, di, dj;     // stencil cell c is (i0 + c di, j0 + c dj)
    int gn;                 // first plane of the normal gradient
    double h, ih;
    double* base;           // record array of this orientation
    size_t stride;          // distance between (field, variable) slices
    size_t idx;             // index of this record inside a slice
};

__device__ __forceinline__ RowRef row_ref(const GridDev& G, int r)
{
    RowRef q;
    const int nx = G.nx, ny = G.ny;
    const int nrx = (nx + 1) * (ny + 4);
    q.xo = r < nrx;
    if (q.xo) {
        const int f = r % (nx + 1), j = r / (nx + 1) - 2;
        q.inner = (j >= -1) && (j <= ny);
        q.i0 = f - 2; q.j0 = j; q.di = 1; q.dj = 0;
        q.gn = 4; q.h = G.dx; q.ih = G.inv_dx;
        q.base = G.recx; q.stride = (size_t)(ny + 4) * (nx + 1); q.idx = (size_t)r;
    } else {
        const int rr = r - nrx;
        const int g = rr % (ny + 1), i = rr / (ny + 1) - 2;
        q.inner = (i >= -1) && (i <= nx);
        q.i0 = i; q.j0 = g - 2; q.di = 0; q.dj = 1;
        q.gn = 8; q.h = G.dy; q.ih = G.inv_dy;
        q.base = G.recy; q.stride = (size_t)(nx + 4) * (ny + 1); q.idx = (size_t)rr;
    }
    return q;
}

// Coefficient table of the register-form reconstruction, one block per order
// (index 0: the 8th-order scheme, 1: the 6th-order variant); copied to shared
// memory by each CTA.
struct ReconTab { double v[2][RK_N]; };

constexpr ReconTab make_recon_tab()
{
    ReconTab t{};
    for (int o = 0; o < 2; ++o) {
        double* k = t.v[o];
        const bool six = (o == 1);
        k[RK_ONE] = 1.0; k[RK_NZERO] = -0.0;
        if (six) {
            k[RK_LV + 0] = 1.0 / 60.0; k[RK_LV + 1] = 29.0 / 60.0; k[RK_LV + 2] = 0.0; k[RK_LV + 3] = 0.2;
            k[RK_LS + 0] = 2.25; k[RK_LS + 1] = 1.0 / 36.0; k[RK_LS + 2] = 0.0; k[RK_LS + 3] = -2.0 / 3.0;
            k[RK_LC + 0] = 0.25; k[RK_LC + 1] = 0.0; k[RK_LC + 2] = -1.5;
        } else {
            k[RK_LV + 0] = 25.0 / 420.0; k[RK_LV + 1] = 185.0 / 420.0; k[RK_LV + 2] = 6.0 / 420.0;
            k[RK_LV + 3] = 102.0 / 420.0;
            k[RK_LS + 0] = 270.0 / 108.0; k[RK_LS + 1] = 14.0 / 108.0; k[RK_LS + 2] = -3.0 / 108.0;
            k[RK_LS + 3] = -99.0 / 108.0;
            k[RK_LC + 0] = 1.0; k[RK_LC + 1] = -0.25; k[RK_LC + 2] = -2.25;
        }
        const double e0[3] = {16.0 / 3.0, -38.0 / 3.0, 25.0 / 3.0};
        const double e1[6] = {801.0 / 80.0, -2443.0 / 80.0, 761.0 / 80.0, 23627.0 / 960.0, -7769.0 / 480.0,
                              3443.0 / 960.0};
        const double e2[6] = {1641.0 / 80.0, 2401.0 / 80.0, -5523.0 / 80.0, 12683.0 / 960.0, -25169.0 / 480.0,
                              56387.0 / 960.0};
        const double e3[3] = {4.0 / 3.0, -5.0 / 3.0, 4.0 / 3.0};
        const double e4[3] = {10.0 / 3.0, -11.0 / 3.0, 4.0 / 3.0};
        const double e5[10] = {4405.0 / 28.0, 4405.0 / 7.0, -110433.0 / 140.0, -21717.0 / 140.0, 93707.0 / 140.0,
                               -226333.0 / 140.0, -48901.0 / 140.0, 209917.0 / 210.0, 17063.0 / 42.0, 5153.0 / 105.0};
        const double e6[10] = {265067.0 / 140.0, 11104.0 / 7.0, -160551.0 / 140.0, -592783.0 / 140.0, 9529.0 / 28.0,
                               -65327.0 / 140.0, -252323.0 / 140.0, 38131.0 / 210.0, 52763.0 / 42.0, 251276.0 / 105.0};
        for (int i = 0; i < 3; ++i) { k[RK_E0 + i] = e0[i]; k[RK_E3 + i] = e3[i]; k[RK_E4 + i] = e4[i]; }
        for (int i = 0; i < 6; ++i) { k[RK_E1 + i] = e1[i]; k[RK_E2 + i] = e2[i]; }
        for (int i = 0; i < 10; ++i) { k[RK_E5 + i] = e5[i]; k[RK_E6 + i] = e6[i]; }
        k[RK_Z + 0] = 3.0; k[RK_Z + 1] = -2.0;
        // Sec. 3.3 linear weights d^8 (the 6th-order variant: d^6)
        const double w8[7] = {3.0 / 98.0, 5.0 / 98.0, 4.0 / 49.0, 7.0 / 98.0, 7.0 / 98.0, 17.0 / 49.0, 17.0 / 49.0};
        const double w6[7] = {3.0 / 70.0, 5.0 / 70.0, 8.0 / 70.0, 7.0 / 70.0, 7.0 / 70.0, 20.0 / 70.0, 20.0 / 70.0};
        const double* w = six ? w6 : w8;
        for (int i = 0; i < 7; ++i) k[RK_W + i] = w[i];
        const double d0 = w[0], d2w = w[2], d5 = w[5], d6 = w[6];
        k[RK_Q0 + 0] = d0 * 7.0 / 6.0; k[RK_Q0 + 1] = -(d0 * 2.0 / 3.0);
        k[RK_Q13 + 0] = 1.0 / 6.0; k[RK_Q13 + 1] = 1.0 / 3.0;
        k[RK_Q2 + 0] = d2w * 0.25; k[RK_Q2 + 1] = d2w * 19.0 / 24.0; k[RK_Q2 + 2] = -(d2w * 13.0 / 24.0);
        k[RK_Q4 + 0] = 2.0 / 3.0; k[RK_Q4 + 1] = -1.0 / 6.0;
        k[RK_Q5 + 0] = d5 * 0.1; k[RK_Q5 + 1] = d5 * 0.7; k[RK_Q5 + 2] = -(d5 / 3.0); k[RK_Q5 + 3] = d5 / 30.0;
        k[RK_Q6 + 0] = d6 * 29.0 / 30.0; k[RK_Q6 + 1] = d6 / 3.0; k[RK_Q6 + 2] = -(d6 * 0.7);
        k[RK_Q6 + 3] = -(d6 * 0.1);
        k[RK_S0 + 0] = d0 * 3.0; k[RK_S0 + 1] = -(d0 * 2.0);
        k[RK_S2 + 0] = d2w * 0.875; k[RK_S2 + 1] = d2w * 0.375; k[RK_S2 + 2] = -(d2w * 0.25);
        k[RK_S5 + 0] = d5 * 0.5; k[RK_S5 + 1] = d5 * 1.5; k[RK_S5 + 2] = -(d5 * 1.5); k[RK_S5 + 3] = d5 * 0.5;
        k[RK_S6 + 0] = d6 * 1.5; k[RK_S6 + 1] = d6 * 0.5; k[RK_S6 + 2] = d6 * 0.5; k[RK_S6 + 3] = -(d6 * 1.5);
    }
    return t;
}


// The arithmetic of one record in conservative variables: variable k from its
// four stencil cells (values Q, h times the normal gradients S), written through
// out(field, k, value); the WENO-Z fields only where `inner` (the rows the
// non-equilibrium states are needed on).
template <int ORDER, class Out>
__device__ __forceinline__ void cons_record(const RegK& r, const double Q[4], const double S[4], double ih,
                                            double weno_eps, bool inner, int k, Out out)
{
    double v, hvx, h2vxx;
    linear_recon_rk<ORDER>(r, Q[0], Q[1], Q[2], Q[3], S[0], S[1], S[2], S[3], v, hvx, h2vxx);
    out(RV, k, v);
    out(RN, k, r.mul(hvx, ih));
    out(RNN, k, r.mul(r.mul(h2vxx, ih), ih));
    if (inner) {
        double vl, sl, vr, sr;
        weno_pair_rk(r, Q[0], Q[1], Q[2], Q[3], S[0], S[1], S[2], S[3], weno_eps, vl, sl, vr, sr);
        out(RL, k, vl);
        out(RR, k, vr);
        out(RLN, k, r.mul(sl, ih));
        out(RRN, k, r.mul(sr, ih));
    }
}

// The arithmetic of one record in characteristic variables: all four variables
// from the stencil cells' values Qa[var][cell] and h times normal gradients
// Sa[var][cell] (face frame), written through out(field, k, value).
template <int ORDER, class Out>
__device__ __forceinline__ void char_record(const RegK& r, double gamma, const double Qa[4][4], const double Sa[4][4],
                                            double ih, double weno_eps, bool inner, Out out)
{
    double Wref[4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) Wref[kk] = 0.5 * (Qa[kk][1] + Qa[kk][2]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double v, hvx, h2vxx;
        linear_recon_rk<ORDER>(r, Qa[k][0], Qa[k][1], Qa[k][2], Qa[k][3], Sa[k][0], Sa[k][1], Sa[k][2], Sa[k][3], v,
                               hvx, h2vxx);
        out(RV, k, v);
        out(RN, k, r.mul(hvx, ih));
        out(RNN, k, r.mul(r.mul(h2vxx, ih), ih));
    }
    if (!inner) return;
    // project on the left eigenvectors of the normal flux Jacobian at the
    // mean of the two cells sharing the face, WENO-Z per field, map back
    CharState cs;
    char_state(Wref, gamma, cs);
    double cvl[4], csl[4], cvr[4], csr[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        double l[4], Q[4], S[4];
        char_left_row(cs, m, l);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            Q[c] = l[0] * Qa[0][c] + l[1] * Qa[1][c] + l[2] * Qa[2][c] + l[3] * Qa[3][c];
            S[c] = l[0] * Sa[0][c] + l[1] * Sa[1][c] + l[2] * Sa[2][c] + l[3] * Sa[3][c];
        }
        weno_pair_rk(r, Q[0], Q[1], Q[2], Q[3], S[0], S[1], S[2], S[3], weno_eps, cvl[m], csl[m], cvr[m], csr[m]);
        csl[m] = r.mul(csl[m], ih);
        csr[m] = r.mul(csr[m], ih);
    }
    double o4[4];
    char_to_cons(cs, cvl, o4);
#pragma unroll
    for (int k = 0; k < 4; ++k) out(RL, k, o4[k]);
    char_to_cons(cs, cvr, o4);
#pragma unroll
    for (int k = 0; k < 4; ++k) out(RR, k, o4[k]);
    char_to_cons(cs, csl, o4);
#pragma unroll
    for (int k = 0; k < 4; ++k) out(RLN, k, o4[k]);
    char_to_cons(cs, csr, o4);
#pragma unroll
    for (int k = 0; k < 4; ++k) out(RRN, k, o4[k]);
}

// Conservative variables: variable k of face row `row`.
template <int ORDER>
__device__ __forceinline__ void cons_row(const RegK& r, const GridDev& G, const double* __restrict__ src, size_t PL,
                                         int row, int k)
{
    const RowRef q = row_ref(G, row);
    if (!CGKS_IN_BOUNDS(q.idx < q.stride, G.ctrl)) return;
    const int pv = q.xo ? k : ((k == 1) ? 2 : (k == 2) ? 1 : k);   // face frame: normal momentum first
    double Q[4], S[4];
    const int i3 = q.i0 + 3 * q.di, j3 = q.j0 + 3 * q.dj;
    if (q.i0 >= 0 && q.j0 >= 0 && i3 < G.nx && j3 < G.ny) {
        // stencil inside the grid: no boundary mapping
        const double* v = src + (size_t)pv * PL + (size_t)q.j0 * G.nx + q.i0;
        const double* d = src + (size_t)(q.gn + pv) * PL + (size_t)q.j0 * G.nx + q.i0;
        const size_t step = q.di ? 1 : (size_t)G.nx;
#pragma unroll
        for (int c = 0; c < 4; ++c) { Q[c] = __ldg(v + c * step); S[c] = r.mul(q.h, __ldg(d + c * step)); }
    } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int i = q.i0 + c * q.di, j = q.j0 + c * q.dj;
            Q[c] = cell_value(G, src, PL, i, j, pv);
            S[c] = r.mul(q.h, cell_value(G, src, PL, i, j, q.gn + pv));
        }
    }
    double* o = q.base + q.idx;
    const size_t st = q.stride;
    cons_record<ORDER>(r, Q, S, q.ih, G.weno_eps, q.inner, k,
                       [&](int f, int kk, double x) { o[(f * 4 + kk) * st] = x; });
}

// Characteristic variables: all four variables of face row `row`.
template <int ORDER>
__device__ __forceinline__ void char_row(const RegK& r, const GridDev& G, const double* __restrict__ src, size_t PL,
                                         int row)
{
    const RowRef q = row_ref(G, row);
    if (!CGKS_IN_BOUNDS(q.idx < q.stride, G.ctrl)) return;
    double Qa[4][4], Sa[4][4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const int pk = q.xo ? kk : ((kk == 1) ? 2 : (kk == 2) ? 1 : kk);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int i = q.i0 + c * q.di, j = q.j0 + c * q.dj;
            Qa[kk][c] = cell_value(G, src, PL, i, j, pk);
            Sa[kk][c] = r.mul(q.h, cell_value(G, src, PL, i, j, q.gn + pk));
        }
    }
    double* o = q.base + q.idx;
    const size_t st = q.stride;
    char_record<ORDER>(r, G.gamma, Qa, Sa, q.ih, G.weno_eps, q.inner,
                       [&](int f, int kk, double x) { o[(f * 4 + kk) * st] = x; });
}


}  // namespace cgks
