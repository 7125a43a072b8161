// cgks_fused.cuh -- both stages of one two-stage fourth-order step (Sec. 2.2,
// Eq. step-hyper-1) for one TX x TY tile, with the intermediate state W* kept
// in shared memory: the temporal fusion of the two stages.  The fused kernel
// (cgks_fused.cu) runs it per tile; a host build runs the same phases (one
// caller thread per phase) to check the layout against the three-kernel step.
//
// Stage 2 of the tile's faces needs W* on the tile widened by two cells on each
// side (the normal stencils reach cells i-2..i+1 of a face, the tangential ones
// rows j-2..j+2), so stage 1 runs on that widened region: its records, face
// segments and cell updates are recomputed by every tile that needs them.  On a
// periodic axis the region is computed in unwrapped coordinates (a ghost cell
// is the same arithmetic on the same inputs as the cell it wraps to); on the
// other axes W* of a ghost cell is the boundary condition applied to the
// region's own cells, as the three-kernel step applies it to W* in memory.
// Every record, segment and update is the three-kernel step's arithmetic
// (cons_record / char_record, segment_results, update_cell_core), so the
// results are the same bits.
//
//   phase 1  stage-1 records of the region's faces (from W^n in global memory)
//   phase 2  stage-1 face segments of the region's cells
//   phase 3  stage-1 update of the region's cells: W* to shared memory, R (the
//            tile's own cells) to buf[par^1]
//   phase 4  stage-2 records of the tile's faces (from W* in shared memory)
//   phase 5  stage-2 face segments of the tile's cells (each tile evaluates
//            both faces of its cells: a face between two tiles is evaluated twice)
//   phase 6  stage-2 update of the tile's cells, W^{n+1} to buf[par^1], CFL bound
#pragma once
#include "cgks_records.cuh"
#include "cgks_segment.cuh"
#include "cgks_update.cuh"

namespace cgks {

constexpr int kFusedThreads = 256;
constexpr int kFusedTX = 16, kFusedTY = 8;

constexpr int cmax(int a, int b) { return a > b ? a : b; }

template <int TX, int TY>
struct FusedLayout {
    static constexpr int EX = TX + 4, EY = TY + 4;   // the widened region of W*
    // stage 1: records of x-faces x0-2..x0+TX+2 on the region's rows, y-faces likewise
    using R1X = RecGroups<EY, EX + 1>;
    using R1Y = RecGroups<EX, EY + 1>;
    static constexpr int n1x = (EX + 1) * EY, n1y = (EY + 1) * EX;   // stage-1 face segments
    // stage 2: records of the tile's faces
    using R2X = RecGroups<TY, TX + 1>;
    using R2Y = RecGroups<TX, TY + 1>;
    static constexpr int n2x = (TX + 1) * TY, n2y = (TY + 1) * TX;   // stage-2 face segments
    static constexpr int nws = 12 * EX * EY;                          // W* of the region
    // region P: stage-1 records; after phase 2, W* and the stage-2 records
    static constexpr int nP = cmax(R1X::n + R1Y::n, nws + R2X::n + R2Y::n);
    // region Q: stage-1 face results (16 per segment); after phase 3, stage-2 ones (8)
    static constexpr int nQ = cmax(16 * (n1x + n1y), 8 * (n2x + n2y));
    static constexpr size_t bytes = sizeof(double) * (size_t)(nP + nQ);
};

template <int TX, int TY>
struct FusedTile {
    using L = FusedLayout<TX, TY>;
    static constexpr int EX = L::EX, EY = L::EY;
    const GridDev& G;
    double* P;         // L::nP doubles of shared memory
    double* Q;         // L::nQ doubles
    RegK rf;           // flux table (the tile's grid and dt)
    RegK rr;           // reconstruction table of the grid's order
    int x0, y0, par;
    bool perx, pery;

    __device__ __forceinline__ int nx() const { return G.nx; }
    __device__ __forceinline__ int ny() const { return G.ny; }
    // a cell of the region whose stage-1 update the tile computes: on a periodic axis
    // any (unwrapped) coordinate, otherwise a cell of the grid
    __device__ __forceinline__ bool computed(int i, int j) const
    {
        return (perx || (i >= 0 && i < G.nx)) && (pery || (j >= 0 && j < G.ny));
    }
    __device__ __forceinline__ static int wrap(int i, int n) { const int m = i % n; return m < 0 ? m + n : m; }

    // ---------------- phase 1: the stage-1 record of (orientation, face, row[, variable])
    // written into the RecGroups slots of that row (group A: values and normal
    // derivatives, B: non-equilibrium states and slopes, C: second normal derivative)
    template <class Rec>
    __device__ __forceinline__ static void put(double* rec, int F, int fc, int qa, int rowsA, int f, int k, double v)
    {
        // qa: the row's slot in group A (group B slots start one row later, C two)
        if (f == RV || f == RN) {
            rec[(f * 4 + k) * Rec::pa + qa * F + fc] = v;
        } else if (f == RNN) {
            const int qc = qa - 2;
            if (qc >= 0 && qc < rowsA - 4) rec[8 * Rec::pa + 16 * Rec::pb + k * Rec::pc + qc * F + fc] = v;
        } else {
            const int qb = qa - 1;
            if (qb >= 0 && qb < rowsA - 2) rec[8 * Rec::pa + ((f - RL) * 4 + k) * Rec::pb + qb * F + fc] = v;
        }
    }

    __device__ void records1(int tid, int nth) const
    {
        using RX = typename L::R1X;
        using RY = typename L::R1Y;
        double* recx = P;
        double* recy = P + RX::n;
        const bool cv = G.recon_vars != 0;
        const int nv = cv ? 1 : 4;
        // x-faces: EX+1 faces x (EY+4) rows; y-faces: EY+1 faces x (EX+4) columns
        const int nxr = (EX + 1) * (EY + 4), nyr = (EY + 1) * (EX + 4);
        const double* __restrict__ src = G.buf[par];
        const size_t PL = (size_t)G.nx * G.ny;
        for (int item = tid; item < nv * (nxr + nyr); item += nth) {
            const int k = item / (nxr + nyr);
            const int it = item - k * (nxr + nyr);
            const bool xo = it < nxr;
            const int F = xo ? EX + 1 : EY + 1, rowsA = xo ? EY + 4 : EX + 4;
            const int fc = (xo ? it : it - nxr) % F, qa = (xo ? it : it - nxr) / F;
            // global face index along the normal and row index along the face
            const int f = (xo ? x0 : y0) - 2 + fc, j = (xo ? y0 : x0) - 4 + qa;
            const bool pn = xo ? perx : pery, pt = xo ? pery : perx;
            const int nn = xo ? G.nx : G.ny, nt = xo ? G.ny : G.nx;
            double* rec = xo ? recx : recy;
            auto out = [&](int fld, int kk, double v) {
                if (xo) put<RX>(rec, F, fc, qa, rowsA, fld, kk, v);
                else put<RY>(rec, F, fc, qa, rowsA, fld, kk, v);
            };
            // rows beyond the grid's two ghost rows (non-periodic) and faces outside the grid
            // are read by no segment the tile evaluates: zero
            const bool valid = (pn || (f >= 0 && f <= nn)) && (pt || (j >= -2 && j <= nt + 1));
            if (!valid) {
                for (int fld = 0; fld < NREC; ++fld)
                    for (int kk = (cv ? 0 : k); kk < (cv ? 4 : k + 1); ++kk) out(fld, kk, 0.0);
                continue;
            }
            // the non-equilibrium fields on group B's rows (rows -1..n on a non-periodic axis)
            const bool inner = (qa >= 1 && qa <= rowsA - 2) && (pt || (j >= -1 && j <= nt));
            if (!inner) {
                for (int fld = RL; fld <= RRN; ++fld)
                    for (int kk = (cv ? 0 : k); kk < (cv ? 4 : k + 1); ++kk) out(fld, kk, 0.0);
            }
            const int gn = xo ? 4 : 8;
            const double h = xo ? G.dx : G.dy, ih = xo ? G.inv_dx : G.inv_dy;
            auto cell = [&](int c, int p) {
                return xo ? cell_value(G, src, PL, f - 2 + c, j, p) : cell_value(G, src, PL, j, f - 2 + c, p);
            };
            if (!cv) {
                const int pv = xo ? k : ((k == 1) ? 2 : (k == 2) ? 1 : k);
                double Qv[4], S[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) { Qv[c] = cell(c, pv); S[c] = rr.mul(h, cell(c, gn + pv)); }
                if (G.order == 6) cons_record<6>(rr, Qv, S, ih, G.weno_eps, inner, k, out);
                else cons_record<8>(rr, Qv, S, ih, G.weno_eps, inner, k, out);
            } else {
                double Qa[4][4], Sa[4][4];
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const int pk = xo ? kk : ((kk == 1) ? 2 : (kk == 2) ? 1 : kk);
#pragma unroll
                    for (int c = 0; c < 4; ++c) { Qa[kk][c] = cell(c, pk); Sa[kk][c] = rr.mul(h, cell(c, gn + pk)); }
                }
                if (G.order == 6) char_record<6>(rr, G.gamma, Qa, Sa, ih, G.weno_eps, inner, out);
                else char_record<8>(rr, G.gamma, Qa, Sa, ih, G.weno_eps, inner, out);
            }
        }
    }

    // ---------------- phase 2: the stage-1 face segments the region's cells need;
    // results in the physical frame at Q[q * (n1x + n1y) + segment]
    __device__ bool flux1(int tid, int nth) const
    {
        using RX = typename L::R1X;
        using RY = typename L::R1Y;
        constexpr int NS = L::n1x + L::n1y;
        bool bad = false;
        for (int item = tid; item < NS; item += nth) {
            const bool xo = item < L::n1x;
            int fc, q, r0, rstride, pa, pb, pc;
            const double* rec;
            bool need;
            if (xo) {
                // x-face x0-2+fc on row y0-2+q; its cells fc-1 and fc of the region
                fc = item % (EX + 1); q = item / (EX + 1);
                const int f = x0 - 2 + fc, j = y0 - 2 + q;
                need = (fc >= 1 && computed(f - 1, j)) || (fc <= EX - 1 && computed(f, j));
                rec = P; pa = RX::pa; pb = RX::pb; pc = RX::pc; rstride = EX + 1; r0 = q * rstride + fc;
            } else {
                const int it = item - L::n1x;
                fc = it % (EY + 1); q = it / (EY + 1);
                const int g = y0 - 2 + fc, i = x0 - 2 + q;
                need = (fc >= 1 && computed(i, g - 1)) || (fc <= EY - 1 && computed(i, g));
                rec = P + RX::n; pa = RY::pa; pb = RY::pb; pc = RY::pc; rstride = EY + 1; r0 = q * rstride + fc;
            }
            if (!need) continue;
            if (!CGKS_IN_BOUNDS(r0 >= 0 && r0 + 4 * rstride < pa && r0 + 2 * rstride < pb && r0 < pc, G.ctrl)) continue;
            double acc[16];
            bad |= !segment_results<1, false>(rf, rec, pa, pb, pc, r0, rstride, rf.k(xo ? FK_IDY : FK_IDX), nullptr,
                                              acc);
#pragma unroll
            for (int qq = 0; qq < 16; qq += 4) {
                const int k1 = xo ? 1 : 2, k2 = xo ? 2 : 1;
                Q[(qq + 0) * NS + item] = acc[qq + 0];
                Q[(qq + k1) * NS + item] = acc[qq + 1];
                Q[(qq + k2) * NS + item] = acc[qq + 2];
                Q[(qq + 3) * NS + item] = acc[qq + 3];
            }
        }
        return !bad;
    }

    // ---------------- phase 3: stage-1 update of the region's computed cells
    __device__ void update1(int tid, int nth) const
    {
        constexpr int NS = L::n1x + L::n1y;
        double* ws = P;   // 12 planes of EX x EY
        double dtmin = 0.0;
        bool bad = false;
        for (int c = tid; c < EX * EY; c += nth) {
            const int lx = c % EX, ly = c / EX;
            const int i = x0 - 2 + lx, j = y0 - 2 + ly;
            if (!computed(i, j)) continue;
            const int wi = perx ? wrap(i, G.nx) : i, wj = pery ? wrap(j, G.ny) : j;
            const size_t off = (size_t)wj * G.nx + wi;
            const bool own = lx >= 2 && lx < TX + 2 && ly >= 2 && ly < TY + 2 && i < G.nx && j < G.ny;
            double* __restrict__ rbuf = G.buf[par ^ 1];
            const size_t PL = (size_t)G.nx * G.ny;
            update_cell_core<1>(
                G, par, off, [&](int q, int side) { return Q[q * NS + ly * (EX + 1) + lx + side]; },
                [&](int q, int side) { return Q[q * NS + L::n1x + lx * (EY + 1) + ly + side]; },
                [&](int p, double v) { ws[p * EX * EY + c] = v; },
                [&](int p, double v) {
                    if (own) rbuf[p * PL + off] = v;
                },
                dtmin, bad);
        }
    }

    // W* of cell (i, j) of the grid (unwrapped on periodic axes) from the region,
    // with the boundary conditions applied on the other axes
    __device__ __forceinline__ double wstar(int i, int j, int p) const
    {
        int kx = 0, ky = 0, si = i, sj = j;
        if (!perx) si = map_axis(i, G.nx, G.bc[0], G.bc[1], kx);
        if (!pery) sj = map_axis(j, G.ny, G.bc[2], G.bc[3], ky);
        const int lx = si - (x0 - 2), ly = sj - (y0 - 2);
        if (!CGKS_IN_BOUNDS(lx >= 0 && lx < EX && ly >= 0 && ly < EY && p >= 0 && p < 12, G.ctrl)) return 0.0;
        return bc_value(G, P[p * EX * EY + ly * EX + lx], i, j, kx, ky, p);
    }

    // ---------------- phase 4: stage-2 records of the tile's faces, from W*
    __device__ void records2(int tid, int nth) const
    {
        using RX = typename L::R2X;
        using RY = typename L::R2Y;
        double* recx = P + L::nws;
        double* recy = recx + RX::n;
        const bool cv = G.recon_vars != 0;
        const int nv = cv ? 1 : 4;
        const int nxr = (TX + 1) * (TY + 4), nyr = (TY + 1) * (TX + 4);
        for (int item = tid; item < nv * (nxr + nyr); item += nth) {
            const int k = item / (nxr + nyr);
            const int it = item - k * (nxr + nyr);
            const bool xo = it < nxr;
            const int F = xo ? TX + 1 : TY + 1, rowsA = xo ? TY + 4 : TX + 4;
            const int fc = (xo ? it : it - nxr) % F, qa = (xo ? it : it - nxr) / F;
            const int f = (xo ? x0 : y0) + fc, j = (xo ? y0 : x0) - 2 + qa;
            const bool pt = xo ? pery : perx;
            const int nn = xo ? G.nx : G.ny, nt = xo ? G.ny : G.nx;
            double* rec = xo ? recx : recy;
            auto out = [&](int fld, int kk, double v) {
                if (xo) put<RX>(rec, F, fc, qa, rowsA, fld, kk, v);
                else put<RY>(rec, F, fc, qa, rowsA, fld, kk, v);
            };
            // faces of the tile's cells only (the grid's last face where the tile ends on
            // its edge), rows up to the two ghost rows of a non-periodic axis
            const bool valid = (f <= nn) && (pt || (j >= -2 && j <= nt + 1));
            if (!valid) {
                for (int fld = 0; fld < NREC; ++fld)
                    for (int kk = (cv ? 0 : k); kk < (cv ? 4 : k + 1); ++kk) out(fld, kk, 0.0);
                continue;
            }
            const bool inner = (qa >= 1 && qa <= rowsA - 2) && (pt || (j >= -1 && j <= nt));
            if (!inner) {
                for (int fld = RL; fld <= RRN; ++fld)
                    for (int kk = (cv ? 0 : k); kk < (cv ? 4 : k + 1); ++kk) out(fld, kk, 0.0);
            }
            const int gn = xo ? 4 : 8;
            const double h = xo ? G.dx : G.dy, ih = xo ? G.inv_dx : G.inv_dy;
            auto cell = [&](int c, int p) { return xo ? wstar(f - 2 + c, j, p) : wstar(j, f - 2 + c, p); };
            if (!cv) {
                const int pv = xo ? k : ((k == 1) ? 2 : (k == 2) ? 1 : k);
                double Qv[4], S[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) { Qv[c] = cell(c, pv); S[c] = rr.mul(h, cell(c, gn + pv)); }
                if (G.order == 6) cons_record<6>(rr, Qv, S, ih, G.weno_eps, inner, k, out);
                else cons_record<8>(rr, Qv, S, ih, G.weno_eps, inner, k, out);
            } else {
                double Qa[4][4], Sa[4][4];
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const int pk = xo ? kk : ((kk == 1) ? 2 : (kk == 2) ? 1 : kk);
#pragma unroll
                    for (int c = 0; c < 4; ++c) { Qa[kk][c] = cell(c, pk); Sa[kk][c] = rr.mul(h, cell(c, gn + pk)); }
                }
                if (G.order == 6) char_record<6>(rr, G.gamma, Qa, Sa, ih, G.weno_eps, inner, out);
                else char_record<8>(rr, G.gamma, Qa, Sa, ih, G.weno_eps, inner, out);
            }
        }
    }

    // ---------------- phase 5: stage-2 segments of the tile's faces; results at
    // Q[q * (n2x + n2y) + segment] in the physical frame
    __device__ bool flux2(int tid, int nth) const
    {
        using RX = typename L::R2X;
        using RY = typename L::R2Y;
        constexpr int NS = L::n2x + L::n2y;
        bool bad = false;
        for (int item = tid; item < NS; item += nth) {
            const bool xo = item < L::n2x;
            int r0, rstride, pa, pb, pc;
            const double* rec;
            bool need;
            if (xo) {
                const int fc = item % (TX + 1), q = item / (TX + 1);
                need = (x0 + fc <= G.nx) && (y0 + q < G.ny);
                rec = P + L::nws; pa = RX::pa; pb = RX::pb; pc = RX::pc; rstride = TX + 1; r0 = q * rstride + fc;
            } else {
                const int it = item - L::n2x;
                const int gc = it % (TY + 1), q = it / (TY + 1);
                need = (y0 + gc <= G.ny) && (x0 + q < G.nx);
                rec = P + L::nws + RX::n; pa = RY::pa; pb = RY::pb; pc = RY::pc; rstride = TY + 1;
                r0 = q * rstride + gc;
            }
            if (!need) continue;
            if (!CGKS_IN_BOUNDS(r0 >= 0 && r0 + 4 * rstride < pa && r0 + 2 * rstride < pb && r0 < pc, G.ctrl)) continue;
            double acc[8];
            bad |= !segment_results<2, false>(rf, rec, pa, pb, pc, r0, rstride, rf.k(xo ? FK_IDY : FK_IDX), nullptr,
                                              acc);
#pragma unroll
            for (int qq = 0; qq < 8; qq += 4) {
                const int k1 = xo ? 1 : 2, k2 = xo ? 2 : 1;
                Q[(qq + 0) * NS + item] = acc[qq + 0];
                Q[(qq + k1) * NS + item] = acc[qq + 1];
                Q[(qq + k2) * NS + item] = acc[qq + 2];
                Q[(qq + 3) * NS + item] = acc[qq + 3];
            }
        }
        return !bad;
    }

    // ---------------- phase 6: stage-2 update of the tile's cells
    __device__ void update2(int tid, int nth, double& dtmin, bool& bad) const
    {
        constexpr int NS = L::n2x + L::n2y;
        for (int c = tid; c < TX * TY; c += nth) {
            const int lx = c % TX, ly = c / TX;
            const int i = x0 + lx, j = y0 + ly;
            if (i >= G.nx || j >= G.ny) continue;
            const size_t off = (size_t)j * G.nx + i;
            update_cell_core<2>(
                G, par, off, [&](int q, int side) { return Q[q * NS + ly * (TX + 1) + lx + side]; },
                [&](int q, int side) { return Q[q * NS + L::n2x + lx * (TY + 1) + ly + side]; },
                [&](int, double) {}, [&](int, double) {}, dtmin, bad);
        }
    }
};

}  // namespace cgks
