// cgks_segment.cuh -- the per-face-segment arithmetic of the flux kernel
// (cgks_stage.cuh): the layout of a tile's face-row records in shared memory,
// the reconstruction along a face at a Gauss point (SegmentRows) and one
// segment's two Gauss points with their Gauss average (segment_results).
#pragma once
#include "cgks_device.cuh"
#include "cgks_flux.cuh"
#include "cgks_internal.h"

namespace cgks {

constexpr int kThreads = 128;

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
    // (S1 = mp + mm and A1 = mp - mm come from the caller, which shares them with the WENO-Z values)
    __device__ __forceinline__ static void seg_deriv_parts(const RegK& r, double* dc, double m2m, double S1, double A1,
                                                           double m0, double m2p, double n2m, double nm, double n0,
                                                           double np, double n2p)
    {
        const double S2 = r.add(m2p, m2m), A2 = r.sub(m2p, m2m);
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

// One face segment of the flux kernel: the nonlinear point values along the face
// at both Gauss points, then the gas-kinetic evaluation at each point, Gauss-
// averaged (weight 1/2) with the stage's time factors into acc (face frame;
// stage 1: the W* and R flux combinations and the interface states W(dt/2),
// W(dt); stage 2: dt^2/3 F_t and dt^2/3 W_tt).  rec, pa, pb, pc, r0, rstride
// locate the segment's face rows in the tile's records; dc is this thread's
// slice for the Gauss-point-independent derivative parts (SHARE).  PARK: the
// first point's sums are stored at park[q * park_stride] (the segment's own
// output slots) while the second point is evaluated, and read back after it,
// which frees their registers (the same values, the same bits).  Returns
// false if a state was non-physical.
template <int STAGE, bool SHARE, bool PARK = false>
__device__ __forceinline__ bool segment_results(const RegK& r, const double* rec, int pa, int pb, int pc, int r0,
                                                int rstride, double iht, double* dc, double acc[FaceQ<STAGE>::n],
                                                double* park = nullptr, size_t park_stride = 0)
{
    constexpr int NF = FaceQ<STAGE>::n;
    constexpr double gq = 0.28867513459481287;   // 1/(2 sqrt 3): Gauss points at +-gq
    const double weps = r.k(FK_WEPS), weps4 = r.k(FK_WEPS4);
    bool bad = false;
#pragma unroll
    for (int q = 0; q < NF; ++q) acc[q] = 0.0;
    // the nonlinear values along the face: both Gauss points at once
    double W0m[4], W0p[4], sL[4], sR[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        auto R = [&](int f, int off) { return rec_at(rec, pa, pb, pc, r0, rstride, f, k, off); };
        const double m2m = R(RV, -2), mm = R(RV, -1), m0 = R(RV, 0), mp = R(RV, 1), m2p = R(RV, 2);
        const double S1 = r.add(mp, mm), A1 = r.sub(mp, mm);
        tang_weno5_pair(r, m2m, mm, m0, mp, m2p, A1, S1, weps4, W0m[k], W0p[k]);
        if constexpr (SHARE)
            SegmentRows<true>::seg_deriv_parts(r, dc + 8 * k * kThreads, m2m, S1, A1, m0, m2p, R(RN, -2), R(RN, -1),
                                               R(RN, 0), R(RN, 1), R(RN, 2));
        tang_weno3_slopes(r, R(RL, -1), R(RL, 0), R(RL, 1), R(RR, -1), R(RR, 0), R(RR, 1), weps, sL[k], sR[k]);
    }
#pragma unroll 1
    for (int gp = 0; gp < 2; ++gp) {
        const double eta = gp ? gq : -gq;
        const SegmentRows<SHARE> src{r, rec, pa, pb, pc, r0, rstride, eta, iht,
                                     {gp ? W0p[0] : W0m[0], gp ? W0p[1] : W0m[1], gp ? W0p[2] : W0m[2],
                                      gp ? W0p[3] : W0m[3]},
                                     {sL[0], sL[1], sL[2], sL[3]}, {sR[0], sR[1], sR[2], sR[3]}, dc};
        double Fb[4], Ft[4], Wm[4], Wb[4], Wtt[4];
        bad |= !gks_point<STAGE>(r, src, Fb, Ft, Wm, Wb, Wtt);
        if (PARK && gp == 1) {
#pragma unroll
            for (int q = 0; q < NF; ++q) acc[q] = park[q * park_stride];
        }
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
        if (PARK && gp == 0) {
#pragma unroll
            for (int q = 0; q < NF; ++q) park[q * park_stride] = acc[q];
        }
    }
    return !bad;
}

}  // namespace cgks
