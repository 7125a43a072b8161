// cgks_stage.cuh -- the fused per-stage kernel of the two-stage fourth-order
// compact GKS (Sec. 2.2, Eq. step-hyper-1; Sec. 3.1, Eq. compact-deriv-1).
//
// One CTA owns a TX x TY tile of cells of one grid and runs, in shared memory:
//   phase 0  stage the tile plus a two-cell halo of all 12 planes (boundary
//            conditions applied in the loader: periodic, reflecting, inflow,
//            outflow; x-boundaries first, then y, corners included)
//   phase 1  normal reconstruction of every face row the tile needs: linear
//            8th-order values/derivatives (Sec. 3.2) and, for the rows within
//            one of a segment, the nonlinear WENO-Z left/right states with
//            slopes (Sec. 3.3); one record per (face, row), shared by the five
//            face segments that use it
//   phase 2  per face segment, at two Gauss points: WENO-Z point values along
//            the face over rows j-2..j+2 (equilibrium) and j-1..j+1
//            (non-equilibrium states, with their tangential slopes); tangential
//            derivatives of the equilibrium state and normal derivatives from
//            the quartic / quadratic through the same line averages; the
//            gas-kinetic evaluation at each point, Gauss average
//   phase 3  per cell: S2O4 update of cell averages by the fluxes and of the
//            cell-averaged gradients by the Gauss theorem on interface states
// Stage 1 writes W* and R = W^n + dt L + dt^2/6 L_t (and the gradient
// counterparts); stage 2 turns R into W^{n+1} in place and reduces the CFL
// bound of the new state for the next step.
// The kernel is persistent: CTAs stride over a flattened tile queue that may
// span many grids of different sizes (each with its own dt in its Ctrl).
#pragma once
#include "cgks_device.cuh"
#include "cgks_internal.h"
#include "../../include/cgks.h"

namespace cgks {

constexpr int kThreads = 256;

// fields of a face-row record
enum { RV = 0, RN = 1, RNN = 2, RL = 3, RR = 4, RLN = 5, RRN = 6, NREC = 7 };

template <int STAGE> struct FaceQ { static constexpr int n = (STAGE == 1) ? 16 : 8; };

template <int TX, int TY, int STAGE>
struct StageLayout {
    static constexpr int BX = TX + 4, BY = TY + 4;
    static constexpr int NF = FaceQ<STAGE>::n;
    static constexpr int n_cells = 12 * BY * BX;
    static constexpr int n_rx = 4 * NREC * (TY + 4) * (TX + 1);
    static constexpr int n_ry = 4 * NREC * (TX + 4) * (TY + 1);
    static constexpr int n_fx = NF * TY * (TX + 1);
    static constexpr int n_fy = NF * (TY + 1) * TX;
    static constexpr size_t bytes = sizeof(double) * (size_t)(n_cells + n_rx + n_ry + n_fx + n_fy);
};

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

// The face rows around one face segment (records of rows j-2..j+2 of one
// face) and the reconstruction along the face at one Gauss point eta: the
// WENO-Z point values (equilibrium over five rows, non-equilibrium slopes over
// three) are computed once per segment for both points and carried in W0, sL,
// sR; tangential derivatives of the equilibrium state and normal derivatives
// come from the quartic / quadratic through the same line averages.
struct SegmentRows {
    const double* rec;
    int nrec, r0, rstride;
    double eta, iht, weps;
    double W0[4], sL[4], sR[4];   // WENO-Z values at this point, non-equilibrium slopes

    __device__ __forceinline__ double at(int f, int k, int off) const { return rec[(f * 4 + k) * nrec + r0 + off * rstride]; }

    __device__ __forceinline__ void eq_value(double W[4]) const
    {
#pragma unroll
        for (int k = 0; k < 4; ++k) W[k] = W0[k];
    }

    // quartic with segment means m_{j-2..j+2}: coefficients c1..c4 of eta^1..eta^4
    __device__ __forceinline__ static void quartic(double mm, double m, double m0, double p, double pp,
                                                   double& c1, double& c2, double& c3, double& c4)
    {
        const double S1 = p + m, S2 = pp + mm, A1 = p - m, A2 = pp - mm;
        c1 = (34.0 * A1 - 5.0 * A2) * (1.0 / 48.0);
        c3 = (A2 - 2.0 * A1) * (1.0 / 12.0);
        c2 = (12.0 * S1 - S2 - 22.0 * m0) * (1.0 / 16.0);
        c4 = (S2 - 4.0 * S1 + 6.0 * m0) * (1.0 / 24.0);
    }

    __device__ __forceinline__ void eq_derivs(double W0n[4], double W0t[4], double W0nn[4], double W0nt[4],
                                              double W0tt[4]) const
    {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            double c1, c2, c3, c4;
            quartic(at(RV, k, -2), at(RV, k, -1), at(RV, k, 0), at(RV, k, 1), at(RV, k, 2), c1, c2, c3, c4);
            W0t[k] = (c1 + 0.25 * c3 + eta * (2.0 * c2 + c4 * (1.0 / 3.0))) * iht;
            W0tt[k] = (2.0 * c2 + c4 + 6.0 * eta * c3) * iht * iht;
            const double N0 = at(RN, k, 0);
            quartic(at(RN, k, -2), at(RN, k, -1), N0, at(RN, k, 1), at(RN, k, 2), c1, c2, c3, c4);
            W0n[k] = N0 - c4 * (1.0 / 180.0) + eta * (c1 + c3 * (1.0 / 12.0));
            W0nt[k] = (c1 + 0.25 * c3 + eta * (2.0 * c2 + c4 * (1.0 / 3.0))) * iht;
            W0nn[k] = at(RNN, k, 0);
        }
    }

    __device__ __forceinline__ void ne_value(int side, double W[4], double Wt[4]) const
    {
        const int f = side ? RR : RL;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const double sl = side ? sR[k] : sL[k];
            W[k] = at(f, k, 0) + eta * sl;
            Wt[k] = sl * iht;
        }
    }

    __device__ __forceinline__ void ne_normal(int side, double Wn[4]) const
    {
        const int f = side ? RRN : RLN;
#pragma unroll
        for (int k = 0; k < 4; ++k) Wn[k] = at(f, k, 0) + eta * 0.5 * (at(f, k, 1) - at(f, k, -1));
    }
};

template <int TX, int TY, int STAGE>
__global__ void __launch_bounds__(kThreads, 1)
stage_kernel(const GridDev* __restrict__ grids, const TileRef* __restrict__ tiles, int ntiles)
{
    using L = StageLayout<TX, TY, STAGE>;
    constexpr int BX = L::BX, BY = L::BY, NF = L::NF;
    extern __shared__ double smem[];
    double* sc = smem;                  // [12][BY][BX]
    double* rx = sc + L::n_cells;       // [28][TY+4][TX+1]
    double* ry = rx + L::n_rx;          // [28][TX+4][TY+1]
    double* fx = ry + L::n_ry;          // [NF][TY][TX+1]
    double* fy = fx + L::n_fx;          // [NF][TY+1][TX]
    __shared__ double s_dt;
    __shared__ int s_skip, s_par;
    const int tid = threadIdx.x;
    constexpr double gq = 0.28867513459481287;   // 1/(2 sqrt 3): Gauss points at +-gq

    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();
        const TileRef tr = tiles[tile];
        const GridDev& G = grids[tr.grid];
        if (tid == 0) {
            const Ctrl* C = G.ctrl;
            s_skip = C->done;
            s_dt = C->dt;
            s_par = C->par;
        }
        __syncthreads();
        if (s_skip) continue;
        const int nx = G.nx, ny = G.ny, x0 = tr.x0, y0 = tr.y0;
        const double dt = s_dt;
        const int par = s_par;
        const bool dim1 = (G.dim == 1);
        const double* __restrict__ src = (STAGE == 1) ? G.buf[par] : G.ws;
        const size_t PL = (size_t)nx * ny;

        // ---------------- phase 0: halo tile with boundary conditions
        for (int idx = tid; idx < BX * BY; idx += kThreads) {
            const int ii = idx % BX, jj = idx / BX;
            int kx, ky;
            const int sj = map_axis(y0 - 2 + jj, ny, G.bc[2], G.bc[3], ky);
            const int si = map_axis(x0 - 2 + ii, nx, G.bc[0], G.bc[1], kx);
            const size_t off = (size_t)sj * nx + si;
            double v[12];
#pragma unroll
            for (int p = 0; p < 12; ++p) v[p] = __ldg(src + p * PL + off);
            // x-boundary transform
            if (kx == 1) { v[1] = -v[1]; v[4] = -v[4]; v[6] = -v[6]; v[7] = -v[7]; v[9] = -v[9]; }
            else if (kx == 2) {
                const double* q = G.inflow[(x0 - 2 + ii < 0) ? 0 : 1];
#pragma unroll
                for (int p = 0; p < 4; ++p) { v[p] = q[p]; v[4 + p] = 0.0; v[8 + p] = 0.0; }
            } else if (kx == 3) { v[4] = v[5] = v[6] = v[7] = 0.0; }
            // y-boundary transform
            if (ky == 1) { v[2] = -v[2]; v[6] = -v[6]; v[8] = -v[8]; v[9] = -v[9]; v[11] = -v[11]; }
            else if (ky == 2) {
                const double* q = G.inflow[(y0 - 2 + jj < 0) ? 2 : 3];
#pragma unroll
                for (int p = 0; p < 4; ++p) { v[p] = q[p]; v[4 + p] = 0.0; v[8 + p] = 0.0; }
            } else if (ky == 3) { v[8] = v[9] = v[10] = v[11] = 0.0; }
#pragma unroll
            for (int p = 0; p < 12; ++p) sc[(p * BY + jj) * BX + ii] = v[p];
        }
        __syncthreads();

        // ---------------- phase 1: normal reconstruction per (face, row, variable)
        // items are (variable, record) pairs so the 256 threads finish together
        const double eps = G.weno_eps;
        constexpr int NRX = (TX + 1) * (TY + 4), NRY = (TX + 4) * (TY + 1), NR = NRX + NRY;
        // the heavy items (inner rows: linear + WENO-Z) are dealt out first, then the
        // light ones (the outer row on each side: linear only), so that no thread gets
        // more than its share of heavy items
        constexpr int NIX = (TX + 1) * (TY + 2), NIY = (TY + 1) * (TX + 2), NI = NIX + NIY;
        constexpr int NOX = (TX + 1) * 2, NOY = (TY + 1) * 2, NO = NOX + NOY;
        static_assert(NI + NO == NR, "record count");
        for (int it = tid; it < 4 * NR; it += kThreads) {
            int k, a, rl;          // variable, face index along the tile, row index of the record
            bool xo;
            if (it < 4 * NI) {
                k = it / NI;
                int r = it - k * NI;
                xo = r < NIX;
                if (!xo) r -= NIX;
                const int nf = xo ? TX + 1 : TY + 1;
                a = r % nf; rl = 1 + r / nf;
            } else {
                const int r2 = it - 4 * NI;
                k = r2 / NO;
                int r = r2 - k * NO;
                xo = r < NOX;
                if (!xo) r -= NOX;
                const int nf = xo ? TX + 1 : TY + 1;
                a = r % nf; rl = (r / nf) ? (xo ? TY + 3 : TX + 3) : 0;
            }
            int box_i, box_j, step_i, step_j, ridx, nrec, pv, gn;
            double h, ih;
            double* rec;
            bool valid, inner;
            if (xo) {
                const int fl = a;                                       // row y0-2+rl
                valid = (x0 + fl <= nx) && (y0 - 2 + rl <= ny + 1);
                inner = (rl >= 1) && (rl <= TY + 2);
                box_i = fl; box_j = rl; step_i = 1; step_j = 0;
                h = G.dx; ih = G.inv_dx; gn = 4;
                pv = k;
                rec = rx; nrec = (TY + 4) * (TX + 1); ridx = rl * (TX + 1) + fl;
            } else {
                const int gl = a;                                       // column x0-2+rl
                valid = !dim1 && (y0 + gl <= ny) && (x0 - 2 + rl <= nx + 1);
                inner = (rl >= 1) && (rl <= TX + 2);
                box_i = rl; box_j = gl; step_i = 0; step_j = 1;
                h = G.dy; ih = G.inv_dy; gn = 8;
                pv = (k == 1) ? 2 : (k == 2) ? 1 : k;                  // face frame: normal momentum first
                rec = ry; nrec = (TX + 4) * (TY + 1); ridx = rl * (TY + 1) + gl;
            }
            if (!valid) {
#pragma unroll
                for (int f = 0; f < NREC; ++f) rec[(f * 4 + k) * nrec + ridx] = 0.0;
                continue;
            }
            double Q[4], S[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int bi = box_i + c * step_i, bj = box_j + c * step_j;
                Q[c] = sc[(pv * BY + bj) * BX + bi];
                S[c] = h * sc[((gn + pv) * BY + bj) * BX + bi];
            }
            double v, hvx, h2vxx;
            linear_recon(Q[0], Q[1], Q[2], Q[3], S[0], S[1], S[2], S[3], v, hvx, h2vxx);
            rec[(RV * 4 + k) * nrec + ridx] = v;
            rec[(RN * 4 + k) * nrec + ridx] = hvx * ih;
            rec[(RNN * 4 + k) * nrec + ridx] = h2vxx * ih * ih;
            if (inner) {
                if (G.recon_vars) {
                    // characteristic field k: project the stencil on the k-th left eigenvector
                    // at the mean of the two cells sharing the face
                    double Wref[4], Qa[4][4], Sa[4][4], l[4];
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const int pk = xo ? kk : ((kk == 1) ? 2 : (kk == 2) ? 1 : kk);
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const int bi = box_i + c * step_i, bj = box_j + c * step_j;
                            Qa[kk][c] = sc[(pk * BY + bj) * BX + bi];
                            Sa[kk][c] = h * sc[((gn + pk) * BY + bj) * BX + bi];
                        }
                        Wref[kk] = 0.5 * (Qa[kk][1] + Qa[kk][2]);
                    }
                    CharState cs;
                    char_state(Wref, G.gamma, cs);
                    char_left_row(cs, k, l);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        Q[c] = l[0] * Qa[0][c] + l[1] * Qa[1][c] + l[2] * Qa[2][c] + l[3] * Qa[3][c];
                        S[c] = l[0] * Sa[0][c] + l[1] * Sa[1][c] + l[2] * Sa[2][c] + l[3] * Sa[3][c];
                    }
                }
                double vl, sl, vr, sr;
                weno_pair(Q[0], Q[1], Q[2], Q[3], S[0], S[1], S[2], S[3], eps, vl, sl, vr, sr);
                rec[(RL * 4 + k) * nrec + ridx] = vl;
                rec[(RR * 4 + k) * nrec + ridx] = vr;
                rec[(RLN * 4 + k) * nrec + ridx] = sl * ih;
                rec[(RRN * 4 + k) * nrec + ridx] = sr * ih;
            }
        }
        __syncthreads();
        if (G.recon_vars) {
            // back to conservative variables, one record per thread
            for (int item = tid; item < NR; item += kThreads) {
                const bool xo = item < NR - NRY;
                int box_i, box_j, step_i, step_j, ridx, nrec;
                double* rec;
                bool valid, inner;
                if (xo) {
                    const int fl = item % (TX + 1), rl = item / (TX + 1);
                    valid = (x0 + fl <= nx) && (y0 - 2 + rl <= ny + 1);
                    inner = (rl >= 1) && (rl <= TY + 2);
                    box_i = fl; box_j = rl; step_i = 1; step_j = 0;
                    rec = rx; nrec = (TY + 4) * (TX + 1); ridx = rl * (TX + 1) + fl;
                } else {
                    const int itm = item - NRX;
                    const int gl = itm % (TY + 1), rl = itm / (TY + 1);
                    valid = !dim1 && (y0 + gl <= ny) && (x0 - 2 + rl <= nx + 1);
                    inner = (rl >= 1) && (rl <= TX + 2);
                    box_i = rl; box_j = gl; step_i = 0; step_j = 1;
                    rec = ry; nrec = (TX + 4) * (TY + 1); ridx = rl * (TY + 1) + gl;
                }
                if (!valid || !inner) continue;
                double Wref[4];
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const int pk = xo ? kk : ((kk == 1) ? 2 : (kk == 2) ? 1 : kk);
                    const double a = sc[(pk * BY + box_j + step_j) * BX + box_i + step_i];
                    const double b = sc[(pk * BY + box_j + 2 * step_j) * BX + box_i + 2 * step_i];
                    Wref[kk] = 0.5 * (a + b);
                }
                CharState cs;
                char_state(Wref, G.gamma, cs);
#pragma unroll
                for (int f = RL; f <= RRN; ++f) {
                    double w[4], o[4];
#pragma unroll
                    for (int m = 0; m < 4; ++m) w[m] = rec[(f * 4 + m) * nrec + ridx];
                    char_to_cons(cs, w, o);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) rec[(f * 4 + kk) * nrec + ridx] = o[kk];
                }
            }
            __syncthreads();
        }

        // ---------------- phase 2: face segments, two Gauss points each
        Params P;
        P.gamma = G.gamma; P.K = G.K; P.eps_tau = G.eps_tau; P.c_tau = G.c_tau; P.dt = dt; P.mu = G.mu;
        P.idt = __drcp_rn(dt); P.inv_K2 = __drcp_rn(G.K + 2.0); P.inv_gm1 = __drcp_rn(G.gamma - 1.0);
        P.K2inv2 = 2.0 * P.inv_K2; P.Kheat = 0.5 * (G.K + 4.0);
        bool bad = false;
        constexpr int NSX = (TX + 1) * TY, NSY = TX * (TY + 1);
        for (int item = tid; item < NSX + NSY; item += kThreads) {
            const bool xo = item < NSX;
            const double* rec;
            int nrec, r0, rstride;
            double ht;
            double* out;
            int nout, oidx;
            bool valid;
            if (xo) {
                const int fl = item % (TX + 1), jl = item / (TX + 1);
                valid = (x0 + fl <= nx) && (y0 + jl < ny);
                rec = rx; nrec = (TY + 4) * (TX + 1); r0 = (jl + 2) * (TX + 1) + fl; rstride = TX + 1;
                ht = G.dy; out = fx; nout = TY * (TX + 1); oidx = jl * (TX + 1) + fl;
            } else {
                const int it = item - NSX;
                const int il = it % TX, gl = it / TX;
                valid = !dim1 && (y0 + gl <= ny) && (x0 + il < nx);
                rec = ry; nrec = (TX + 4) * (TY + 1); r0 = (il + 2) * (TY + 1) + gl; rstride = TY + 1;
                ht = G.dx; out = fy; nout = (TY + 1) * TX; oidx = gl * TX + il;
            }
            if (!valid) {
#pragma unroll
                for (int q = 0; q < NF; ++q) out[q * nout + oidx] = 0.0;
                continue;
            }
            const double iht = xo ? G.inv_dy : G.inv_dx;
            const double weps = G.weno_eps;
            double acc[NF];
#pragma unroll
            for (int q = 0; q < NF; ++q) acc[q] = 0.0;
            // the nonlinear values along the face: both Gauss points at once
            double W0m[4], W0p[4], sL[4], sR[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                auto R = [&](int f, int off) { return rec[(f * 4 + k) * nrec + r0 + off * rstride]; };
                tang_weno5_pair(R(RV, -2), R(RV, -1), R(RV, 0), R(RV, 1), R(RV, 2), gq, weps, W0m[k], W0p[k]);
                sL[k] = tang_weno3_slope(R(RL, -1), R(RL, 0), R(RL, 1), weps);
                sR[k] = tang_weno3_slope(R(RR, -1), R(RR, 0), R(RR, 1), weps);
            }
#pragma unroll 1
            for (int gp = 0; gp < 2; ++gp) {
                const double eta = gp ? gq : -gq;
                const SegmentRows src{rec, nrec, r0, rstride, eta, iht, weps,
                                      {gp ? W0p[0] : W0m[0], gp ? W0p[1] : W0m[1], gp ? W0p[2] : W0m[2],
                                       gp ? W0p[3] : W0m[3]},
                                      {sL[0], sL[1], sL[2], sL[3]}, {sR[0], sR[1], sR[2], sR[3]}};
                double Fb[4], Ft[4], Wm[4], Wb[4], Wtt[4];
                bad |= !gks_point<STAGE>(src, P, Fb, Ft, Wm, Wb, Wtt);
                if (STAGE == 1) {
                    const double c1a = 0.25 * dt, c1b = dt * dt * (1.0 / 16.0);       // half of (dt/2, dt^2/8)
                    const double c2a = 0.5 * dt, c2b = dt * dt * (1.0 / 12.0);        // half of (dt, dt^2/6)
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        acc[k] += c1a * Fb[k] + c1b * Ft[k];
                        acc[4 + k] += c2a * Fb[k] + c2b * Ft[k];
                        acc[8 + k] += 0.5 * Wm[k];
                        acc[12 + k] += 0.5 * Wb[k];
                    }
                } else {
                    const double c3 = dt * dt * (1.0 / 6.0);                           // half of dt^2/3
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        acc[k] += c3 * Ft[k];
                        acc[4 + k] += c3 * Wtt[k];
                    }
                }
            }
            // back to the physical frame (y-faces: swap momentum components)
#pragma unroll
            for (int q = 0; q < NF; q += 4) {
                const int k1 = xo ? 1 : 2, k2 = xo ? 2 : 1;
                out[(q + 0) * nout + oidx] = acc[q + 0];
                out[(q + k1) * nout + oidx] = acc[q + 1];
                out[(q + k2) * nout + oidx] = acc[q + 2];
                out[(q + 3) * nout + oidx] = acc[q + 3];
            }
        }
        if (bad) atomicOr(&G.ctrl->status, (int)CGKS_E_NONPHYSICAL);
        __syncthreads();

        // ---------------- phase 3: cell update
        double* __restrict__ rbuf = G.buf[par ^ 1];
        const double idx_ = G.inv_dx, idy_ = G.inv_dy;
        double dtmin = INFINITY;
        bool bad2 = false;
        for (int item = tid; item < TX * TY; item += kThreads) {
            const int il = item % TX, jl = item / TX;
            const int i = x0 + il, j = y0 + jl;
            if (i >= nx || j >= ny) continue;
            const size_t off = (size_t)j * nx + i;
            const int xl = jl * (TX + 1) + il, xr = xl + 1;
            const int yb = jl * TX + il, yt = yb + TX;
            constexpr int nfx = TY * (TX + 1), nfy = (TY + 1) * TX;
            auto FX = [&](int q, int at) { return fx[q * nfx + at]; };
            auto FY = [&](int q, int at) { return dim1 ? 0.0 : fy[q * nfy + at]; };
            if (STAGE == 1) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const double W = sc[(k * BY + jl + 2) * BX + il + 2];
                    G.ws[k * PL + off] = W - (FX(k, xr) - FX(k, xl)) * idx_ - (FY(k, yt) - FY(k, yb)) * idy_;
                    G.ws[(4 + k) * PL + off] = (FX(8 + k, xr) - FX(8 + k, xl)) * idx_;
                    G.ws[(8 + k) * PL + off] = (FY(8 + k, yt) - FY(8 + k, yb)) * idy_;
                    rbuf[k * PL + off] = W - (FX(4 + k, xr) - FX(4 + k, xl)) * idx_ - (FY(4 + k, yt) - FY(4 + k, yb)) * idy_;
                    rbuf[(4 + k) * PL + off] = (FX(12 + k, xr) - FX(12 + k, xl)) * idx_;
                    rbuf[(8 + k) * PL + off] = (FY(12 + k, yt) - FY(12 + k, yb)) * idy_;
                }
            } else {
                double Wn[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const double R = rbuf[k * PL + off];
                    Wn[k] = R - (FX(k, xr) - FX(k, xl)) * idx_ - (FY(k, yt) - FY(k, yb)) * idy_;
                    rbuf[k * PL + off] = Wn[k];
                    rbuf[(4 + k) * PL + off] += (FX(4 + k, xr) - FX(4 + k, xl)) * idx_;
                    rbuf[(8 + k) * PL + off] += (FY(4 + k, yt) - FY(4 + k, yb)) * idy_;
                }
                // CFL bound of the new state (Sec. 4)
                const double ir = 1.0 / Wn[0];
                const double U = Wn[1] * ir, V = Wn[2] * ir;
                const double p = (G.gamma - 1.0) * (Wn[3] - 0.5 * (Wn[1] * U + Wn[2] * V));
                const bool ok = (Wn[0] > 0.0) && (p > 0.0);
                bad2 |= !ok;
                const double c = sqrt(G.gamma * p * ir);
                const double nu = G.mu * ir;
                double d = G.dx / (fabs(U) + c + 2.0 * nu * G.inv_dx);
                if (!dim1) d = fmin(d, G.dy / (fabs(V) + c + 2.0 * nu * G.inv_dy));
                if (ok) dtmin = fmin(dtmin, d);
            }
        }
        if (STAGE == 2) {
            if (bad2) atomicOr(&G.ctrl->status, (int)CGKS_E_NONPHYSICAL);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dtmin = fmin(dtmin, __shfl_xor_sync(0xffffffffu, dtmin, o));
            if ((tid & 31) == 0 && dtmin < INFINITY)
                atomicMin(&G.ctrl->dtmin_bits, (unsigned long long)__double_as_longlong(dtmin));
        }
    }
}

template <int TX, int TY, int STAGE>
cudaError_t launch_stage_t(const GridDev* grids, const TileRef* tiles, int ntiles, int nblocks, cudaStream_t st)
{
    using L = StageLayout<TX, TY, STAGE>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(stage_kernel<TX, TY, STAGE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    if (ntiles <= 0) return cudaSuccess;
    stage_kernel<TX, TY, STAGE><<<nblocks, kThreads, L::bytes, st>>>(grids, tiles, ntiles);
    return cudaGetLastError();
}

// The launcher and shared-memory size of one tile shape (one translation unit
// per shape, so the shapes compile in parallel).
#define CGKS_STAGE_INSTANCE(TX, TY)                                                                         \
    static_assert(StageLayout<TX, TY, 1>::bytes + 64 <= 227 * 1024, "stage-1 tile exceeds shared memory");  \
    cudaError_t launch_stage_##TX##x##TY(int stage, const GridDev* grids, const TileRef* tiles, int ntiles,  \
                                         int nblocks, cudaStream_t st)                                      \
    {                                                                                                       \
        return stage == 1 ? launch_stage_t<TX, TY, 1>(grids, tiles, ntiles, nblocks, st)                    \
                          : launch_stage_t<TX, TY, 2>(grids, tiles, ntiles, nblocks, st);                   \
    }                                                                                                       \
    size_t smem_##TX##x##TY(int stage)                                                                      \
    {                                                                                                       \
        return stage == 1 ? StageLayout<TX, TY, 1>::bytes : StageLayout<TX, TY, 2>::bytes;                  \
    }

}  // namespace cgks
