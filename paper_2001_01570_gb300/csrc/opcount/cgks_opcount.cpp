// cgks_opcount.cpp -- host count of the FP64 operations of one time step of
// the CUDA kernels' own formulas, and host runs of one step of those formulas
// in the three-kernel and the fused arrangement (libcgks_opcount; not part of
// the solver).
//
// The device arithmetic of the record, flux and update kernels
// (cgks_records.cuh, cgks_segment.cuh / cgks_flux.cuh, cgks_update.cuh) is
// compiled here for the host with every FP64 value of type Real, whose
// operations tally themselves: add, subtract and multiply count 1, a fused
// multiply-add 2, and a divide, square root, reciprocal, exponential or erfc
// 1 each, however the GPU expands them (the kernels' Tang exponential, table
// erfc and Newton reciprocal count as one operation).  RegK's register forms
// count as the operation they stand for.  The code below runs one step of a
// 2D grid the way the kernels do -- every face row's record, every face
// segment of every 8x16 tile (each face once), every cell's update, both
// stages -- and reports the tally of each of the six launches.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <utility>
#include <vector>

#include "../../../include/cgks.h"

namespace cgks_oc {

enum Kind { K_ADD, K_MUL, K_FMA, K_DIV, K_SQRT, K_RCP, K_EXP, K_ERFC, K_N };
inline unsigned long long g_tally[K_N];

inline void count(Kind k)
{
    ++g_tally[k];
}

struct Real {
    double v;
    constexpr Real() : v(0.0) {}
    constexpr Real(double x) : v(x) {}
    constexpr Real(const Real& o) = default;
    Real(const volatile Real& o) : v(o.v) {}
    constexpr Real& operator=(const Real& o) = default;
    explicit constexpr operator double() const { return v; }
    explicit constexpr operator int() const { return (int)v; }
};

#define CGKS_OC_COUNT(k) \
    if (!std::is_constant_evaluated()) count(k)
constexpr Real operator+(Real a, Real b) { CGKS_OC_COUNT(K_ADD); return Real(a.v + b.v); }
constexpr Real operator-(Real a, Real b) { CGKS_OC_COUNT(K_ADD); return Real(a.v - b.v); }
constexpr Real operator*(Real a, Real b) { CGKS_OC_COUNT(K_MUL); return Real(a.v * b.v); }
constexpr Real operator/(Real a, Real b) { CGKS_OC_COUNT(K_DIV); return Real(a.v / b.v); }
constexpr Real operator-(Real a) { return Real(-a.v); }   // a sign change is free in an FP64 instruction
constexpr Real operator+(Real a) { return a; }
inline Real& operator+=(Real& a, Real b) { a = a + b; return a; }
inline Real& operator-=(Real& a, Real b) { a = a - b; return a; }
inline Real& operator*=(Real& a, Real b) { a = a * b; return a; }
constexpr bool operator<(Real a, Real b) { return a.v < b.v; }
constexpr bool operator>(Real a, Real b) { return a.v > b.v; }
constexpr bool operator<=(Real a, Real b) { return a.v <= b.v; }
constexpr bool operator>=(Real a, Real b) { return a.v >= b.v; }
constexpr bool operator==(Real a, Real b) { return a.v == b.v; }
constexpr bool operator!=(Real a, Real b) { return a.v != b.v; }
inline Real fma(Real a, Real b, Real c) { count(K_FMA); return Real(std::fma(a.v, b.v, c.v)); }
inline Real fabs(Real a) { return Real(std::fabs(a.v)); }
inline Real fmin(Real a, Real b) { return Real(std::fmin(a.v, b.v)); }
inline Real fmax(Real a, Real b) { return Real(std::fmax(a.v, b.v)); }
inline Real sqrt(Real a) { count(K_SQRT); return Real(std::sqrt(a.v)); }
inline Real rsqrt(Real a) { count(K_SQRT); return Real(1.0 / std::sqrt(a.v)); }
inline Real exp2(Real a) { count(K_EXP); return Real(std::exp2(a.v)); }
inline bool isinf(Real a) { return std::isinf(a.v); }
inline bool isnan(Real a) { return std::isnan(a.v); }

}  // namespace cgks_oc

using cgks_oc::Real;

// the CUDA device functions the included formulas call, for Real on the host
inline Real cgks_opcount_rcp(Real x) { cgks_oc::count(cgks_oc::K_RCP); return Real(1.0 / x.v); }
inline Real cgks_opcount_exp(Real x) { cgks_oc::count(cgks_oc::K_EXP); return Real(std::exp(x.v)); }
inline Real cgks_opcount_erfc(Real x) { cgks_oc::count(cgks_oc::K_ERFC); return Real(std::erfc(x.v)); }
inline Real __drcp_rn(Real x) { cgks_oc::count(cgks_oc::K_RCP); return Real(1.0 / x.v); }
inline Real __ddiv_rn(Real a, Real b) { return a / b; }
inline Real __dmul_rn(Real a, Real b) { return a * b; }
inline Real __dadd_rn(Real a, Real b) { return a + b; }
inline Real __dsub_rn(Real a, Real b) { return a - b; }
inline Real __dsqrt_rn(Real a) { return cgks_oc::sqrt(a); }
inline long long __double_as_longlong(Real x) { long long b; memcpy(&b, &x.v, 8); return b; }
inline Real __longlong_as_double(long long b) { double x; memcpy(&x, &b, 8); return Real(x); }
template <class T> inline T __ldg(const T* p) { return *p; }
inline int min(int a, int b) { return a < b ? a : b; }
inline int max(int a, int b) { return a > b ? a : b; }

#define CGKS_OPCOUNT_HOST 1
#define double Real
#include "../cgks_internal.h"
#include "../cgks_records.cuh"
#include "../cgks_segment.cuh"
#include "../cgks_update.cuh"
#include "../cgks_fused.cuh"
#undef double

namespace {

using namespace cgks;

struct Grid {
    GridDev G;
    std::vector<Real> planes, records, faces;
    Ctrl ctrl;
};

// the x- and y-face records of one TX x TY tile in the shared-memory layout of
// the flux kernel (cgks_stage.cuh, phase 1), zero outside the grid
template <int TX, int TY>
void stage_tile(const GridDev& G, int x0, int y0, std::vector<Real>& rx, std::vector<Real>& ry)
{
    using RX = RecGroups<TY, TX + 1>;
    using RY = RecGroups<TX, TY + 1>;
    const int nx = G.nx, ny = G.ny;
    const size_t sx = (size_t)(ny + 4) * (nx + 1), sy = (size_t)(nx + 4) * (ny + 1);
    rx.assign(RX::n, Real(0.0));
    ry.assign(RY::n, Real(0.0));
    auto stage = [&](std::vector<Real>& dst, int sofs, int np, int plane, int F, int p0, const Real* g, size_t gs,
                     int gfaces, int row0, int face0, int nface_max, int row_max) {
        for (int idx = 0; idx < np * plane; ++idx) {
            const int p = idx / plane, rem = idx - p * plane;
            const int q = rem / F, fc = rem - q * F;
            const bool valid = (face0 + fc <= nface_max) && (row0 + q <= row_max);
            dst[sofs + idx] = valid ? g[(size_t)(p0 + p) * gs + (size_t)(row0 + q) * gfaces + face0 + fc] : Real(0.0);
        }
    };
    stage(rx, 0, 8, RX::pa, TX + 1, 0, G.recx, sx, nx + 1, y0, x0, nx, ny + 3);
    stage(rx, 8 * RX::pa, 16, RX::pb, TX + 1, 4 * RL, G.recx, sx, nx + 1, y0 + 1, x0, nx, ny + 3);
    stage(rx, 8 * RX::pa + 16 * RX::pb, 4, RX::pc, TX + 1, 4 * RNN, G.recx, sx, nx + 1, y0 + 2, x0, nx, ny + 3);
    stage(ry, 0, 8, RY::pa, TY + 1, 0, G.recy, sy, ny + 1, x0, y0, ny, nx + 3);
    stage(ry, 8 * RY::pa, 16, RY::pb, TY + 1, 4 * RL, G.recy, sy, ny + 1, x0 + 1, y0, ny, nx + 3);
    stage(ry, 8 * RY::pa + 16 * RY::pb, 4, RY::pc, TY + 1, 4 * RNN, G.recy, sy, ny + 1, x0 + 2, y0, ny, nx + 3);
}

// the face segments of one tile (cgks_stage.cuh, phase 2)
template <int TX, int TY, int STAGE>
bool tile_segments(const RegK& r, const GridDev& G, int x0, int y0, const std::vector<Real>& rx,
                   const std::vector<Real>& ry, std::vector<Real>& dc)
{
    constexpr int NF = FaceQ<STAGE>::n;
    const int nx = G.nx, ny = G.ny;
    const int xe = (x0 + TX == nx) ? TY : 0, ye = (y0 + TY == ny) ? TX : 0;
    const int nseg = 2 * TX * TY + xe + ye;
    const size_t nfx = (size_t)ny * (nx + 1), nfy = (size_t)(ny + 1) * nx;
    bool ok = true;
    for (int item = 0; item < nseg; ++item) {
        int fl = 0, jl = 0, il = 0, gl = 0;
        bool xo;
        if (item < TX * TY) { xo = true; fl = item % TX; jl = item / TX; }
        else if (item < 2 * TX * TY) { xo = false; const int it = item - TX * TY; il = it % TX; gl = it / TX; }
        else {
            const int it = item - 2 * TX * TY;
            if (it < xe) { xo = true; fl = TX; jl = it; }
            else { xo = false; il = it - xe; gl = TY; }
        }
        const Real* rec;
        int pa, pb, pc, r0, rstride;
        Real* out;
        size_t ostride, oidx;
        if (xo) {
            if (!((x0 + fl <= nx) && (y0 + jl < ny))) continue;
            rec = rx.data(); pa = RecGroups<TY, TX + 1>::pa; pb = RecGroups<TY, TX + 1>::pb; pc = RecGroups<TY, TX + 1>::pc;
            r0 = jl * (TX + 1) + fl; rstride = TX + 1;
            out = G.facex; ostride = nfx; oidx = (size_t)(y0 + jl) * (nx + 1) + x0 + fl;
        } else {
            if (!((y0 + gl <= ny) && (x0 + il < nx))) continue;
            rec = ry.data(); pa = RecGroups<TX, TY + 1>::pa; pb = RecGroups<TX, TY + 1>::pb; pc = RecGroups<TX, TY + 1>::pc;
            r0 = il * (TY + 1) + gl; rstride = TY + 1;
            out = G.facey; ostride = nfy; oidx = (size_t)(y0 + gl) * nx + x0 + il;
        }
        const Real iht = r.k(xo ? FK_IDY : FK_IDX);
        Real acc[NF];
        ok &= segment_results<STAGE, true>(r, rec, pa, pb, pc, r0, rstride, iht, dc.data(), acc);
        for (int q = 0; q < NF; q += 4) {
            const int k1 = xo ? 1 : 2, k2 = xo ? 2 : 1;
            out[(q + 0) * ostride + oidx] = acc[q + 0];
            out[(q + k1) * ostride + oidx] = acc[q + 1];
            out[(q + k2) * ostride + oidx] = acc[q + 2];
            out[(q + 3) * ostride + oidx] = acc[q + 3];
        }
    }
    return ok;
}

void snapshot(unsigned long long* dst)
{
    for (int k = 0; k < cgks_oc::K_N; ++k) dst[k] = cgks_oc::g_tally[k];
}

// One step of a 2D grid on the host: the grid's buffers, dt from the CFL bound
// of the state, the coefficient tables as the kernels build them.
struct HostStep {
    Grid g;
    size_t PL = 0;
    ReconTab rt;
    std::vector<Real> fk;
    RegK rrec{}, rflux{};

    // 0, or -1 for a problem not covered (1D), -2 for a non-physical initial state
    int setup(const cgks_problem* prob, const double* planes)
    {
        if (!prob || prob->dim != 2) return -1;
        const int nx = prob->nx, ny = prob->ny;
        PL = (size_t)nx * ny;
        g.planes.assign(36 * PL, Real(0.0));
        for (size_t i = 0; i < 12 * PL; ++i) g.planes[i] = Real(planes[i]);
        g.records.assign(record_doubles(nx, ny, 2), Real(0.0));
        g.faces.assign(face_doubles(nx, ny, 2), Real(0.0));
        GridDev& G = g.G;
        memset((void*)&G, 0, sizeof(G));
        memset((void*)&g.ctrl, 0, sizeof(g.ctrl));
        G.buf[0] = g.planes.data();
        G.buf[1] = g.planes.data() + 12 * PL;
        G.ws = g.planes.data() + 24 * PL;
        G.ctrl = &g.ctrl;
        G.recx = g.records.data();
        G.recy = g.records.data() + (size_t)28 * (nx + 1) * (ny + 4);
        G.facex = g.faces.data();
        G.facey = g.faces.data() + (size_t)16 * (nx + 1) * ny;
        G.nx = nx;
        G.ny = ny;
        G.dim = 2;
        for (int k = 0; k < 4; ++k) G.bc[k] = prob->bc[k];
        G.dx = Real((prob->x1 - prob->x0) / nx);
        G.dy = Real((prob->y1 - prob->y0) / ny);
        G.inv_dx = Real(1.0 / G.dx.v);
        G.inv_dy = Real(1.0 / G.dy.v);
        G.gamma = Real(prob->gamma);
        G.K = Real((4.0 - 2.0 * prob->gamma) / (prob->gamma - 1.0));
        G.cfl = Real(prob->cfl);
        G.eps_tau = Real(prob->eps_tau);
        G.c_tau = Real(prob->c_tau);
        G.weno_eps = Real(prob->weno_eps);
        G.mu = Real(prob->mu);
        G.recon_vars = prob->recon_vars ? 1 : 0;
        G.order = prob->order == 6 ? 6 : 8;
        for (int side = 0; side < 4; ++side) {
            const double* q = prob->inflow[side];
            G.inflow[side][0] = Real(q[0]);
            G.inflow[side][1] = Real(q[0] * q[1]);
            G.inflow[side][2] = Real(q[0] * q[2]);
            G.inflow[side][3] = Real(q[3] / (prob->gamma - 1.0) + 0.5 * q[0] * (q[1] * q[1] + q[2] * q[2]));
        }
        // dt from the CFL bound of the state (not part of the counted launches)
        double dmin = INFINITY;
        for (size_t c = 0; c < PL; ++c) {
            Real d;
            if (!cfl_cell_bound(G, G.buf[0][c], G.buf[0][PL + c], G.buf[0][2 * PL + c], G.buf[0][3 * PL + c], false,
                                &d))
                return -2;
            dmin = std::min(dmin, d.v);
        }
        const Real dt = Real(prob->cfl * dmin);
        rt = make_recon_tab();
        const int ob = G.order == 6 ? 1 : 0;
        rrec = RegK{rt.v[ob], rt.v[ob][RK_ONE], rt.v[ob][RK_NZERO]};
        fk.assign(FK_N, Real(0.0));
        const FluxFixed ff = make_flux_fixed();
        for (int i = 0; i < FK_NFIX; ++i) fk[i] = ff.v[i];
        for (int j = 0; j < 32; ++j) fk[FK_EXP2 + j] = Real(std::exp2(j / 32.0));
        flux_table_tile(fk.data(), G, dt);
        rflux = RegK{fk.data(), fk[FK_ONE], fk[FK_NZERO]};
        return 0;
    }

    // the three-kernel step (records, flux over 8 x 16 tiles, update per stage);
    // out (may be NULL): the counts of the six launches
    bool unfused(unsigned long long* out)
    {
        GridDev& G = g.G;
        const int nx = G.nx, ny = G.ny;
        std::vector<Real> rx, ry, dc(32 * kThreads, Real(0.0));
        const int nrec = record_rows(nx, ny, 2);
        bool ok = true;
        unsigned long long scratch[3 * cgks_oc::K_N];
        for (int stage = 1; stage <= 2; ++stage) {
            unsigned long long* o = out ? out + (size_t)(stage - 1) * 3 * cgks_oc::K_N : scratch;
            const Real* src = stage == 1 ? G.buf[0] : G.ws;
            // records
            memset(cgks_oc::g_tally, 0, sizeof(cgks_oc::g_tally));
            if (G.recon_vars) {
                for (int item = 0; item < nrec; ++item) {
                    if (G.order == 6) char_row<6>(rrec, G, src, PL, item);
                    else char_row<8>(rrec, G, src, PL, item);
                }
            } else {
                for (int item = 0; item < 4 * nrec; ++item) {
                    const int k = item / nrec;
                    if (G.order == 6) cons_row<6>(rrec, G, src, PL, item - k * nrec, k);
                    else cons_row<8>(rrec, G, src, PL, item - k * nrec, k);
                }
            }
            snapshot(o);
            // face segments, 8 x 16 tiles (the 2D default)
            unsigned long long before[cgks_oc::K_N];
            memset(cgks_oc::g_tally, 0, sizeof(cgks_oc::g_tally));
            for (int y0 = 0; y0 < ny; y0 += 16)
                for (int x0 = 0; x0 < nx; x0 += 8) {
                    snapshot(before);
                    stage_tile<8, 16>(G, x0, y0, rx, ry);   // copies, not counted
                    for (int k = 0; k < cgks_oc::K_N; ++k) cgks_oc::g_tally[k] = before[k];
                    ok &= stage == 1 ? tile_segments<8, 16, 1>(rflux, G, x0, y0, rx, ry, dc)
                                     : tile_segments<8, 16, 2>(rflux, G, x0, y0, rx, ry, dc);
                }
            snapshot(o + cgks_oc::K_N);
            // cell updates
            memset(cgks_oc::g_tally, 0, sizeof(cgks_oc::g_tally));
            Real dtmin = Real(INFINITY);
            bool bad = false;
            for (long long cell = 0; cell < (long long)PL; ++cell) {
                if (stage == 1) update_cell<1>(G, 0, cell, dtmin, bad);
                else update_cell<2>(G, 0, cell, dtmin, bad);
            }
            snapshot(o + 2 * cgks_oc::K_N);
            ok &= !bad;
        }
        return ok;
    }

    // the fused step (cgks_fused.cuh): per 16 x 8 tile its six phases, each run by
    // one caller thread over all of the phase's items
    bool fused()
    {
        GridDev& G = g.G;
        using L = FusedLayout<kFusedTX, kFusedTY>;
        std::vector<Real> P(L::nP, Real(0.0)), Q(L::nQ, Real(0.0));
        const RegK rr = rrec;
        bool ok = true;
        Real dtmin = Real(INFINITY);
        for (int y0 = 0; y0 < G.ny; y0 += kFusedTY)
            for (int x0 = 0; x0 < G.nx; x0 += kFusedTX) {
                const FusedTile<kFusedTX, kFusedTY> T{G, P.data(), Q.data(), rflux, rr, x0, y0, 0,
                                                       G.bc[0] == CGKS_BC_PERIODIC, G.bc[2] == CGKS_BC_PERIODIC};
                bool bad = false;
                T.records1(0, 1);
                bad |= !T.flux1(0, 1);
                T.update1(0, 1);
                T.records2(0, 1);
                bad |= !T.flux2(0, 1);
                T.update2(0, 1, dtmin, bad);
                ok &= !bad;
            }
        return ok;
    }
};

}  // namespace

extern "C" {

// One S2O4 step of the 2D problem `prob` from the 12 planes `planes` (layout of
// include/cgks.h), counted.  out receives 6 x 8 numbers: for the launches
// records<1>, flux<1>, update<1>, records<2>, flux<2>, update<2> the counts of
// add/sub, mul, fma, div, sqrt/rsqrt, reciprocal, exp, erfc.  Returns 0, or -1
// for a problem this count does not cover (1D, characteristic variables) and
// -2 if a state met was non-physical.
int cgks_opcount_step(const cgks_problem* prob, const double* planes, unsigned long long* out)
{
    if (!prob || prob->dim != 2 || prob->recon_vars != 0) return -1;
    HostStep h;
    const int st = h.setup(prob, planes);
    if (st != 0) return st;
    return h.unfused(out) ? 0 : -2;
}

// One step of the kernels' arithmetic on the host, three-kernel (fused = 0) or
// fused (fused = 1), from `planes` to `out` (12 planes each; dt from the CFL
// bound of `planes`).  Returns 0, -1 for 1D, -2 if a state met was non-physical.
int cgks_host_step(const cgks_problem* prob, const double* planes, int fused, double* out)
{
    HostStep h;
    const int st = h.setup(prob, planes);
    if (st != 0) return st;
    const bool ok = fused ? h.fused() : h.unfused(nullptr);
    const Real* res = h.g.G.buf[1];
    for (size_t i = 0; i < 12 * h.PL; ++i) out[i] = res[i].v;
    return ok ? 0 : -2;
}

}  // extern "C"
