// cgks_update.cuh -- the arithmetic of one cell's update in one stage of the
// two-stage fourth-order step (Sec. 2.2, Eq. step-hyper-1; the gradients by the
// Gauss theorem, Sec. 3.1, Eq. compact-deriv-1), run by the update kernel of
// cgks_update.cu.
#pragma once
#include "cgks_internal.h"
#include "../../include/cgks.h"

namespace cgks {

// the update of one cell (its four faces' results); stage 2 also folds the
// cell's CFL bound into dtmin and flags a non-physical state in bad
template <int STAGE>
__device__ __forceinline__ void update_cell(const GridDev& G, int par, long long cell, double& dtmin, bool& bad)
{
    const int nx = G.nx, ny = G.ny;
    const bool dim1 = (G.dim == 1);
    const size_t PL = (size_t)nx * ny;
    const size_t nfx = (size_t)ny * (nx + 1), nfy = (size_t)(ny + 1) * nx;
    double* __restrict__ rbuf = G.buf[par ^ 1];
    const double idx_ = G.inv_dx, idy_ = G.inv_dy;
    const int i = (int)(cell % nx), j = (int)(cell / nx);
    const size_t off = (size_t)cell;
    const size_t xl = (size_t)j * (nx + 1) + i, xr = xl + 1;
    const size_t yb = (size_t)j * nx + i, yt = yb + nx;
    if (!CGKS_IN_BOUNDS(cell >= 0 && cell < (long long)PL && xr < nfx && (dim1 || yt < nfy), G.ctrl)) return;
    auto FX = [&](int q, size_t at) { return __ldg(G.facex + q * nfx + at); };
    auto FY = [&](int q, size_t at) { return dim1 ? 0.0 : __ldg(G.facey + q * nfy + at); };
    if (STAGE == 1) {
        const double* __restrict__ src = G.buf[par];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const double W = __ldg(src + k * PL + off);
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
        double d;
        if (cfl_cell_bound(G, Wn[0], Wn[1], Wn[2], Wn[3], dim1, &d)) dtmin = fmin(dtmin, d);
        else bad = true;
    }
}

}  // namespace cgks
