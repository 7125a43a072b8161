// cgks_update.cuh -- the arithmetic of one cell's update in one stage of the
// two-stage fourth-order step (Sec. 2.2, Eq. step-hyper-1; the gradients by the
// Gauss theorem, Sec. 3.1, Eq. compact-deriv-1), run by the update kernel of
// cgks_update.cu.
#pragma once
#include "cgks_internal.h"
#include "../../include/cgks.h"

namespace cgks {

// The arithmetic of one cell's update from the results of its four faces:
// FX(q, side) and FY(q, side) give result q of its low (side 0) and high (side
// 1) x- and y-faces.  Stage 1 reads W from buf[par] at `off` and writes W* and
// its gradients through ws_out(plane, value) and R through r_out(plane, value);
// stage 2 reads R from buf[par^1] at `off`, writes W^{n+1} there, folds the
// cell's CFL bound into dtmin and flags a non-physical state in bad.  The
// operations are written out as explicitly rounded differences and products
// and explicit FMAs (no contraction left to the compiler), so that each kernel
// that inlines it -- the update kernel, the fused step -- gets the same bits.
template <int STAGE, class FXs, class FYs, class WSo, class Ro>
__device__ __forceinline__ void update_cell_core(const GridDev& G, int par, size_t off, FXs FX, FYs FY, WSo ws_out,
                                                 Ro r_out, double& dtmin, bool& bad)
{
    const bool dim1 = (G.dim == 1);
    const size_t PL = (size_t)G.nx * G.ny;
    double* __restrict__ rbuf = G.buf[par ^ 1];
    const double idx_ = G.inv_dx, idy_ = G.inv_dy;
    // high - low of face result q along x and y
    auto dX = [&](int q) { return __dsub_rn(FX(q, 1), FX(q, 0)); };
    auto dY = [&](int q) { return __dsub_rn(FY(q, 1), FY(q, 0)); };
    // a - dX/h_x - dY/h_y
    auto div = [&](double a, int q) { return fma(-dY(q), idy_, fma(-dX(q), idx_, a)); };
    if (STAGE == 1) {
        const double* __restrict__ src = G.buf[par];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const double W = __ldg(src + k * PL + off);
            ws_out(k, div(W, k));
            ws_out(4 + k, __dmul_rn(dX(8 + k), idx_));
            ws_out(8 + k, __dmul_rn(dY(8 + k), idy_));
            r_out(k, div(W, 4 + k));
            r_out(4 + k, __dmul_rn(dX(12 + k), idx_));
            r_out(8 + k, __dmul_rn(dY(12 + k), idy_));
        }
    } else {
        double Wn[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const double R = rbuf[k * PL + off];
            Wn[k] = div(R, k);
            rbuf[k * PL + off] = Wn[k];
            rbuf[(4 + k) * PL + off] = fma(dX(4 + k), idx_, rbuf[(4 + k) * PL + off]);
            rbuf[(8 + k) * PL + off] = fma(dY(4 + k), idy_, rbuf[(8 + k) * PL + off]);
        }
        // CFL bound of the new state (Sec. 4)
        double d;
        if (cfl_cell_bound(G, Wn[0], Wn[1], Wn[2], Wn[3], dim1, &d)) dtmin = fmin(dtmin, d);
        else bad = true;
    }
}

// the update of one cell of the grid from the face results in global memory
template <int STAGE>
__device__ __forceinline__ void update_cell(const GridDev& G, int par, long long cell, double& dtmin, bool& bad)
{
    const int nx = G.nx, ny = G.ny;
    const bool dim1 = (G.dim == 1);
    const size_t PL = (size_t)nx * ny;
    const size_t nfx = (size_t)ny * (nx + 1), nfy = (size_t)(ny + 1) * nx;
    const int i = (int)(cell % nx), j = (int)(cell / nx);
    const size_t off = (size_t)cell;
    const size_t xl = (size_t)j * (nx + 1) + i, xr = xl + 1;
    const size_t yb = (size_t)j * nx + i, yt = yb + nx;
    if (!CGKS_IN_BOUNDS(cell >= 0 && cell < (long long)PL && xr < nfx && (dim1 || yt < nfy), G.ctrl)) return;
    double* __restrict__ rbuf = G.buf[par ^ 1];
    update_cell_core<STAGE>(
        G, par, off, [&](int q, int side) { return __ldg(G.facex + q * nfx + (side ? xr : xl)); },
        [&](int q, int side) { return dim1 ? 0.0 : __ldg(G.facey + q * nfy + (side ? yt : yb)); },
        [&](int p, double v) { G.ws[p * PL + off] = v; }, [&](int p, double v) { rbuf[p * PL + off] = v; }, dtmin,
        bad);
}

}  // namespace cgks
