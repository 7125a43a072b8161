// cgks_stage.cuh -- the per-stage flux kernel of the two-stage fourth-order
// compact GKS (Sec. 2.2, Eq. step-hyper-1).  It runs after the record kernel
// (cgks_records.cu), which did the normal reconstruction of every face row of
// the grid once, and before the update kernel (cgks_update.cu), which applies
// the face results to the cells.
//
// One CTA owns a TX x TY tile of cells of one grid and runs, in shared memory:
//   phase 1  stage the face-row records the tile needs (its faces on its rows
//            and two rows either side) with asynchronous copies
//   phase 2  per face segment the tile owns (the x- and y-faces on the low side
//            of its cells, plus the grid's last face where the tile ends on the
//            grid's edge, so every face is evaluated once), at two Gauss points:
//            WENO-Z point values along the face over rows j-2..j+2
//            (equilibrium) and j-1..j+1 (non-equilibrium states, with their
//            tangential slopes); tangential derivatives of the equilibrium state
//            and normal derivatives from the quartic / quadratic through the same
//            line averages (their Gauss-point-independent parts once per
//            segment); the gas-kinetic evaluation at each point; the Gauss
//            average, weighted by the stage's time factors, written to the face
//            results (stage 1: the W* and R flux combinations and the interface
//            states W(dt/2), W(dt); stage 2: dt^2/3 F_t and dt^2/3 W_tt)
// Coefficients (fixed, and the tile's grid and dt) come from the shared-memory
// table of cgks_flux.cuh; all arithmetic is in the register-only DFMA forms.
// The kernel is persistent: CTAs stride over a flattened tile queue that may
// span many grids of different sizes (each with its own dt in its Ctrl).
#pragma once
#include "cgks_device.cuh"
#include "cgks_flux.cuh"
#include "cgks_internal.h"
#include "../../include/cgks.h"

#include <mutex>

namespace cgks {

constexpr int kThreads = 128;

static __constant__ FluxFixed kFluxFixed = make_flux_fixed();

template <int STAGE> struct FaceQ { static constexpr int n = (STAGE == 1) ? 16 : 8; };

// Face-row records of one orientation in shared memory: T own rows of F faces.
// Group A (RV, RN: 8 planes) on rows -2..T+1, group B (RL, RR, RLN, RRN: 16
// planes) on rows -1..T, group C (RNN: 4 planes) on rows 0..T-1 -- the rows each
// field is read on.
template <int T, int F>
struct RecGroups {
    static constexpr int pa = (T + 4) * F, pb = (T + 2) * F, pc = T * F;
    static constexpr int n = 8 * pa + 16 * pb + 4 * pc;
};

// field f, variable k, row `off` relative to the row of r0 = row * F + face
__device__ __forceinline__ double rec_at(const double* rec, int pa, int pb, int pc, int r0, int F, int f, int k,
                                         int off)
{
    if (f == RV || f == RN) return rec[(f * 4 + k) * pa + r0 + (off + 2) * F];
    if (f == RNN) return rec[8 * pa + 16 * pb + k * pc + r0 + off * F];
    return rec[8 * pa + ((f - RL) * 4 + k) * pb + r0 + (off + 1) * F];
}

template <int TX, int TY, int STAGE>
struct StageLayout {
    static constexpr int NF = FaceQ<STAGE>::n;
    static constexpr int n_rx = RecGroups<TY, TX + 1>::n;
    static constexpr int n_ry = RecGroups<TX, TY + 1>::n;
    // where it fits, a per-thread slice of 32 doubles holds the Gauss-point-independent
    // parts of the tangential / normal derivatives of one segment (shared by its two points)
    static constexpr int n_dc_full = 32 * kThreads;
    static constexpr bool share =
        kStageCtasPerSm * (sizeof(double) * (size_t)(n_rx + n_ry + n_dc_full) + 2048) <= 228 * 1024;
    static constexpr int n_dc = share ? n_dc_full : 0;
    static constexpr size_t bytes = sizeof(double) * (size_t)(n_rx + n_ry + n_dc);
};

// The face rows around one face segment (records of rows j-2..j+2 of one
// face) and the reconstruction along the face at one Gauss point eta: the
// WENO-Z point values (equilibrium over five rows, non-equilibrium slopes over
// three) are computed once per segment for both points and carried in W0, sL,
// sR; tangential derivatives of the equilibrium state and normal derivatives
// come from the quartic / quadratic through the same line averages.
template <bool SHARE>
struct SegmentRows {
    RegK r;
    const double* rec;
    int pa, pb, pc, r0, rstride;
    double eta, iht;
    double W0[4], sL[4], sR[4];   // WENO-Z values at this point, non-equilibrium slopes
    const double* dc;             // SHARE: this thread's slice of the segment's derivative parts

    __device__ __forceinline__ double at(int f, int k, int off) const
    {
        return rec_at(rec, pa, pb, pc, r0, rstride, f, k, off);
    }

    __device__ __forceinline__ void eq_value(double W[4]) const
    {
#pragma unroll
        for (int k = 0; k < 4; ++k) W[k] = W0[k];
    }

    // The quartic through the segment means m_{j-2..j+2} (m0 the centre row), written
    // with S1 = m_1 + m_-1, S2 = m_2 + m_-2, A1 = m_1 - m_-1, A2 = m_2 - m_-2:
    //   p(eta)   = m0 - (S2 - 4 S1 + 6 m0)/4320 + eta (50 A1 - 7 A2)/72 + O(eta^2 - 1/12)
    //   p'(eta)  = (8 A1 - A2)/12 + eta (13 S1 - S2 - 24 m0)/9 + O(eta^2 - 1/12)
    //   p''(eta) = (16 S1 - S2 - 30 m0)/12 + eta (A2 - 2 A1)/2 + O(eta^2 - 1/12)
    // (exact at the Gauss points eta = +-1/(2 sqrt 3), where eta^2 = 1/12)
    __device__ __forceinline__ void eq_derivs(double W0n[4], double W0t[4], double W0nn[4], double W0nt[4],
                                              double W0tt[4]) const
    {
        const double iht2 = r.mul(iht, iht);
        if constexpr (SHARE) {
            // the parts computed once per segment by seg_deriv_parts: value + eta * slope
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                auto P = [&](int j) { return dc[(8 * k + j) * kThreads]; };
                W0t[k] = r.mul(fma(eta, P(1), P(0)), iht);
                W0tt[k] = r.mul(fma(eta, P(3), P(2)), iht2);
                W0n[k] = fma(eta, P(5), P(4));
                W0nt[k] = r.mul(fma(eta, P(7), P(6)), iht);
                W0nn[k] = at(RNN, k, 0);
            }
            return;
        }
        auto dp = [&](double m0, double S1, double S2, double A1, double A2) {   // p'(eta) / h_t
            return r.mul(fma(eta, r.kfma(FK_S1T, S1, r.kfma(FK_S2T, S2, r.kmul(FK_M0T, m0))),
                             r.kfma(FK_A1T, A1, r.kmul(FK_A2T, A2))), iht);
        };
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            {
                const double m0 = at(RV, k, 0), mp = at(RV, k, 1), mm = at(RV, k, -1);
                const double m2p = at(RV, k, 2), m2m = at(RV, k, -2);
                const double S1 = r.add(mp, mm), S2 = r.add(m2p, m2m), A1 = r.sub(mp, mm), A2 = r.sub(m2p, m2m);
                W0t[k] = dp(m0, S1, S2, A1, A2);
                W0tt[k] = r.mul(fma(eta, r.kfma(FK_HALF, A2, -A1),
                                    r.kfma(FK_S1TT, S1, r.kfma(FK_S2TT, S2, r.kmul(FK_M0TT, m0)))), iht2);
            }
            {
                const double m0 = at(RN, k, 0), mp = at(RN, k, 1), mm = at(RN, k, -1);
                const double m2p = at(RN, k, 2), m2m = at(RN, k, -2);
                const double S1 = r.add(mp, mm), S2 = r.add(m2p, m2m), A1 = r.sub(mp, mm), A2 = r.sub(m2p, m2m);
                W0n[k] = fma(eta, r.kfma(FK_A1N, A1, r.kmul(FK_A2N, A2)),
                             r.kfma(FK_M0N, m0, r.kfma(FK_S1N, S1, r.kmul(FK_S2N, S2))));
                W0nt[k] = dp(m0, S1, S2, A1, A2);
            }
            W0nn[k] = at(RNN, k, 0);
        }
    }

    // the eta-independent parts of the quartic's derivatives above for variable k
    // (rows m_{-2..2} of the values and of the normal derivatives), stored at dc
    __device__ __forceinline__ static void seg_deriv_parts(const RegK& r, double* dc, double m2m, double mm, double m0,
                                                           double mp, double m2p, double n2m, double nm, double n0,
                                                           double np, double n2p)
    {
        const double S1 = r.add(mp, mm), S2 = r.add(m2p, m2m), A1 = r.sub(mp, mm), A2 = r.sub(m2p, m2m);
        dc[0 * kThreads] = r.kfma(FK_A1T, A1, r.kmul(FK_A2T, A2));
        dc[1 * kThreads] = r.kfma(FK_S1T, S1, r.kfma(FK_S2T, S2, r.kmul(FK_M0T, m0)));
        dc[2 * kThreads] = r.kfma(FK_S1TT, S1, r.kfma(FK_S2TT, S2, r.kmul(FK_M0TT, m0)));
        dc[3 * kThreads] = r.kfma(FK_HALF, A2, -A1);
        const double T1 = r.add(np, nm), T2 = r.add(n2p, n2m), B1 = r.sub(np, nm), B2 = r.sub(n2p, n2m);
        dc[4 * kThreads] = r.kfma(FK_M0N, n0, r.kfma(FK_S1N, T1, r.kmul(FK_S2N, T2)));
        dc[5 * kThreads] = r.kfma(FK_A1N, B1, r.kmul(FK_A2N, B2));
        dc[6 * kThreads] = r.kfma(FK_A1T, B1, r.kmul(FK_A2T, B2));
        dc[7 * kThreads] = r.kfma(FK_S1T, T1, r.kfma(FK_S2T, T2, r.kmul(FK_M0T, n0)));
    }

    __device__ __forceinline__ void ne_value(int side, double W[4], double Wt[4]) const
    {
        const int f = side ? RR : RL;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const double sl = side ? sR[k] : sL[k];
            W[k] = fma(eta, sl, at(f, k, 0));
            Wt[k] = r.mul(sl, iht);
        }
    }

    __device__ __forceinline__ void ne_normal(int side, double Wn[4]) const
    {
        const int f = side ? RRN : RLN;
        const double he = r.kmul(FK_HALF, eta);
#pragma unroll
        for (int k = 0; k < 4; ++k) Wn[k] = fma(he, r.sub(at(f, k, 1), at(f, k, -1)), at(f, k, 0));
    }
};

template <int TX, int TY, int STAGE>
__global__ void __launch_bounds__(kThreads, kStageCtasPerSm)
stage_kernel(const GridDev* __restrict__ grids, const TileRef* __restrict__ tiles, int ntiles,
             const int* __restrict__ dcount)
{
    if (dcount) ntiles = *dcount;   // queue length in device memory (a server's patched queue)
    using L = StageLayout<TX, TY, STAGE>;
    constexpr int NF = L::NF;
    extern __shared__ double smem[];
    double* rx = smem;                  // x-face records, RecGroups<TY, TX+1>
    double* ry = rx + L::n_rx;          // y-face records, RecGroups<TX, TY+1>
    double* dc = ry + L::n_ry + threadIdx.x;   // [32][kThreads] when L::share
    __shared__ double s_fk[FK_N];       // coefficient table (fixed part, then the tile's grid and dt)
    __shared__ int s_skip;
    const int tid = threadIdx.x;
    constexpr double gq = 0.28867513459481287;   // 1/(2 sqrt 3): Gauss points at +-gq
    for (int i = tid; i < FK_NFIX; i += kThreads) s_fk[i] = kFluxFixed.v[i];
    if (tid < 32) s_fk[FK_EXP2 + tid] = exp2((double)tid * (1.0 / 32.0));
    __syncthreads();
    const RegK r{s_fk, ((volatile const double*)s_fk)[FK_ONE], ((volatile const double*)s_fk)[FK_NZERO]};

    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        __syncthreads();
        const TileRef tr = tiles[tile];
        const GridDev& G = grids[tr.grid];
        if (tid == 0) {
            const Ctrl* C = G.ctrl;
            s_skip = C->done;
            if (!C->done) flux_table_tile(s_fk, G, C->dt);
        }
        __syncthreads();
        if (s_skip) continue;
        const int nx = G.nx, ny = G.ny, x0 = tr.x0, y0 = tr.y0;
        const bool dim1 = (G.dim == 1);

        // ---------------- phase 1: the tile's face-row records (the record kernel
        // wrote them for every face row of the grid): x-faces x0..x0+TX on rows
        // y0-2..y0+TY+1, y-faces y0..y0+TY on columns x0-2..x0+TX+1, each field on
        // the rows it is read on; rows beyond the grid's last ghost row are zero
        // and unused.  Asynchronous 8-byte copies, zero-filled where invalid.
        {
            const size_t sx = (size_t)(ny + 4) * (nx + 1), sy = (size_t)(nx + 4) * (ny + 1);
            const unsigned sbx = (unsigned)__cvta_generic_to_shared(rx), sby = (unsigned)__cvta_generic_to_shared(ry);
            // group g of one orientation: plane p of the group is global plane p0 + p, its
            // local row q is record row base + q (records carry two ghost rows first)
            auto stage = [&](unsigned sbase, int sofs, int np, int plane, int F, int p0, const double* g, size_t gs,
                             int gfaces, int row0, int face0, int nface_max, int row_max, bool on) {
                const int n = np * plane;
                for (int idx = tid; idx < n; idx += kThreads) {
                    const int p = idx / plane, rem = idx - p * plane;
                    const int q = rem / F, fc = rem - q * F;
                    const bool valid = on && (face0 + fc <= nface_max) && (row0 + q <= row_max);
                    const double* src = valid ? g + (size_t)(p0 + p) * gs + (size_t)(row0 + q) * gfaces + face0 + fc
                                              : G.recx;
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(sbase + 8u * (unsigned)(sofs + idx)),
                                 "l"(src), "r"(valid ? 8 : 0) : "memory");
                }
            };
            using RX = RecGroups<TY, TX + 1>;
            using RY = RecGroups<TX, TY + 1>;
            // x-faces: record rows y0 + 2 + (own row); group A starts two rows earlier, B one
            stage(sbx, 0, 8, RX::pa, TX + 1, 0, G.recx, sx, nx + 1, y0, x0, nx, ny + 3, true);
            stage(sbx, 8 * RX::pa, 16, RX::pb, TX + 1, 4 * RL, G.recx, sx, nx + 1, y0 + 1, x0, nx, ny + 3, true);
            stage(sbx, 8 * RX::pa + 16 * RX::pb, 4, RX::pc, TX + 1, 4 * RNN, G.recx, sx, nx + 1, y0 + 2, x0, nx, ny + 3,
                  true);
            stage(sby, 0, 8, RY::pa, TY + 1, 0, G.recy, sy, ny + 1, x0, y0, ny, nx + 3, !dim1);
            stage(sby, 8 * RY::pa, 16, RY::pb, TY + 1, 4 * RL, G.recy, sy, ny + 1, x0 + 1, y0, ny, nx + 3, !dim1);
            stage(sby, 8 * RY::pa + 16 * RY::pb, 4, RY::pc, TY + 1, 4 * RNN, G.recy, sy, ny + 1, x0 + 2, y0, ny, nx + 3,
                  !dim1);
            asm volatile("cp.async.wait_all;" ::: "memory");
        }
        __syncthreads();

        // ---------------- phase 2: face segments, two Gauss points each
        bool bad = false;
        // the tile's own faces: x-faces x0..x0+TX-1 and y-faces y0..y0+TY-1 of its
        // cells, plus the last face of the grid where the tile ends on the grid's
        // edge; every face is evaluated by exactly one tile
        const int xe = (x0 + TX == nx) ? TY : 0, ye = (!dim1 && y0 + TY == ny) ? TX : 0;
        const int nseg = (dim1 ? TX * TY : 2 * TX * TY) + xe + ye;
        const size_t nfx = (size_t)ny * (nx + 1), nfy = (size_t)(ny + 1) * nx;
        for (int item = tid; item < nseg; item += kThreads) {
            int fl, jl, il, gl;
            bool xo;
            if (item < TX * TY) { xo = true; fl = item % TX; jl = item / TX; }
            else if (!dim1 && item < 2 * TX * TY) { xo = false; const int it = item - TX * TY; il = it % TX; gl = it / TX; }
            else {
                const int it = item - (dim1 ? TX * TY : 2 * TX * TY);
                if (it < xe) { xo = true; fl = TX; jl = it; }
                else { xo = false; il = it - xe; gl = TY; }
            }
            const double* rec;
            int pa, pb, pc, r0, rstride;
            double* out;
            size_t ostride, oidx;
            if (xo) {
                if (!((x0 + fl <= nx) && (y0 + jl < ny))) continue;
                rec = rx; pa = RecGroups<TY, TX + 1>::pa; pb = RecGroups<TY, TX + 1>::pb; pc = RecGroups<TY, TX + 1>::pc;
                r0 = jl * (TX + 1) + fl; rstride = TX + 1;
                out = G.facex; ostride = nfx; oidx = (size_t)(y0 + jl) * (nx + 1) + x0 + fl;
            } else {
                if (!((y0 + gl <= ny) && (x0 + il < nx))) continue;
                rec = ry; pa = RecGroups<TX, TY + 1>::pa; pb = RecGroups<TX, TY + 1>::pb; pc = RecGroups<TX, TY + 1>::pc;
                r0 = il * (TY + 1) + gl; rstride = TY + 1;
                out = G.facey; ostride = nfy; oidx = (size_t)(y0 + gl) * nx + x0 + il;
            }
            const double iht = r.k(xo ? FK_IDY : FK_IDX);
            const double weps = r.k(FK_WEPS);
            double acc[NF];
#pragma unroll
            for (int q = 0; q < NF; ++q) acc[q] = 0.0;
            // the nonlinear values along the face: both Gauss points at once
            double W0m[4], W0p[4], sL[4], sR[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                auto R = [&](int f, int off) { return rec_at(rec, pa, pb, pc, r0, rstride, f, k, off); };
                const double m2m = R(RV, -2), mm = R(RV, -1), m0 = R(RV, 0), mp = R(RV, 1), m2p = R(RV, 2);
                tang_weno5_pair(r, m2m, mm, m0, mp, m2p, weps, W0m[k], W0p[k]);
                if constexpr (L::share)
                    SegmentRows<true>::seg_deriv_parts(r, dc + 8 * k * kThreads, m2m, mm, m0, mp, m2p, R(RN, -2),
                                                       R(RN, -1), R(RN, 0), R(RN, 1), R(RN, 2));
                tang_weno3_slopes(r, R(RL, -1), R(RL, 0), R(RL, 1), R(RR, -1), R(RR, 0), R(RR, 1), weps, sL[k],
                                  sR[k]);
            }
#pragma unroll 1
            for (int gp = 0; gp < 2; ++gp) {
                const double eta = gp ? gq : -gq;
                const SegmentRows<L::share> src{r, rec, pa, pb, pc, r0, rstride, eta, iht,
                                                {gp ? W0p[0] : W0m[0], gp ? W0p[1] : W0m[1], gp ? W0p[2] : W0m[2],
                                                 gp ? W0p[3] : W0m[3]},
                                                {sL[0], sL[1], sL[2], sL[3]}, {sR[0], sR[1], sR[2], sR[3]}, dc};
                double Fb[4], Ft[4], Wm[4], Wb[4], Wtt[4];
                bad |= !gks_point<STAGE>(r, src, Fb, Ft, Wm, Wb, Wtt);
                // Gauss average (weight 1/2 per point) times the stage's time factors
                if (STAGE == 1) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        acc[k] = r.kfma(FK_W1B, Ft[k], r.kfma(FK_W1A, Fb[k], acc[k]));
                        acc[4 + k] = r.kfma(FK_W2B, Ft[k], r.kfma(FK_W2A, Fb[k], acc[4 + k]));
                        acc[8 + k] = r.kfma(FK_HALF, Wm[k], acc[8 + k]);
                        acc[12 + k] = r.kfma(FK_HALF, Wb[k], acc[12 + k]);
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        acc[k] = r.kfma(FK_W3, Ft[k], acc[k]);
                        acc[4 + k] = r.kfma(FK_W3, Wtt[k], acc[4 + k]);
                    }
                }
            }
            // back to the physical frame (y-faces: swap momentum components)
#pragma unroll
            for (int q = 0; q < NF; q += 4) {
                const int k1 = xo ? 1 : 2, k2 = xo ? 2 : 1;
                out[(q + 0) * ostride + oidx] = acc[q + 0];
                out[(q + k1) * ostride + oidx] = acc[q + 1];
                out[(q + k2) * ostride + oidx] = acc[q + 2];
                out[(q + 3) * ostride + oidx] = acc[q + 3];
            }
        }
        if (bad) atomicOr(&G.ctrl->status, (int)CGKS_E_NONPHYSICAL);
    }
}

// The kernel's attributes (more than 48 KB of dynamic shared memory, the
// largest carveout) belong to one device's context: they are set once per
// device, thread-safely, before the first launch on that device.
template <int TX, int TY, int STAGE>
cudaError_t configure_stage_t()
{
    using L = StageLayout<TX, TY, STAGE>;
    static std::once_flag once[kMaxDevices];
    static cudaError_t status[kMaxDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::call_once(once[dev], [dev] {
        cudaError_t r = cudaFuncSetAttribute(stage_kernel<TX, TY, STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)L::bytes);
        // the largest shared-memory carveout, so that two CTAs fit where the shape allows
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(stage_kernel<TX, TY, STAGE>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared);
        status[dev] = r;
    });
    return status[dev];
}

template <int TX, int TY, int STAGE>
cudaError_t launch_stage_t(const GridDev* grids, const TileRef* tiles, int ntiles, int nblocks, cudaStream_t st,
                           const int* dcount)
{
    using L = StageLayout<TX, TY, STAGE>;
    cudaError_t e = configure_stage_t<TX, TY, STAGE>();
    if (e != cudaSuccess) return e;
    if (ntiles <= 0 || nblocks <= 0) return cudaSuccess;
    stage_kernel<TX, TY, STAGE><<<nblocks, kThreads, L::bytes, st>>>(grids, tiles, ntiles, dcount);
    return cudaGetLastError();
}

// The launcher and shared-memory size of one tile shape (one translation unit
// per shape, so the shapes compile in parallel).
#define CGKS_STAGE_INSTANCE(TX, TY)                                                                         \
    static_assert(StageLayout<TX, TY, 1>::bytes + 64 <= 227 * 1024, "stage-1 tile exceeds shared memory");  \
    cudaError_t launch_stage_##TX##x##TY(int stage, const GridDev* grids, const TileRef* tiles, int ntiles,  \
                                         int nblocks, cudaStream_t st, const int* dcount)                   \
    {                                                                                                       \
        return stage == 1 ? launch_stage_t<TX, TY, 1>(grids, tiles, ntiles, nblocks, st, dcount)            \
                          : launch_stage_t<TX, TY, 2>(grids, tiles, ntiles, nblocks, st, dcount);           \
    }                                                                                                       \
    size_t smem_##TX##x##TY(int stage)                                                                      \
    {                                                                                                       \
        return stage == 1 ? StageLayout<TX, TY, 1>::bytes : StageLayout<TX, TY, 2>::bytes;                  \
    }

}  // namespace cgks
