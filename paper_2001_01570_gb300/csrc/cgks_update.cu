// cgks_update.cu -- the cell update of one stage of the two-stage fourth-order
// step (Sec. 2.2, Eq. step-hyper-1) from the face results the flux kernel wrote
// (each face evaluated once): cell averages by the Gauss-averaged fluxes, cell-
// averaged gradients by the Gauss theorem on the interface states (Sec. 3.1,
// Eq. compact-deriv-1).
//   stage 1: W* = W - (dt/2 F + dt^2/8 F_t) differences,  grad* from W(dt/2);
//            R  = W - (dt F + dt^2/6 F_t) differences,    R_grad from W(dt)
//            (the face results already carry the dt factors and the Gauss weights)
//   stage 2: W^{n+1} = R - dt^2/3 F_t* differences, grad^{n+1} = R_grad + dt^2/3
//            differences of W_tt*; then the CFL bound of W^{n+1} for the next step
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

// One CTA per chunk of 256 cells of one grid; CPT cells per thread (256 / CPT
// threads), the cells of a thread 256 / CPT apart so that every pass of the CTA
// reads and writes contiguous cells.
template <int STAGE, int CPT>
__global__ void __launch_bounds__(256 / CPT) update_kernel(const GridDev* __restrict__ grids,
                                                           const TileRef* __restrict__ chunks, int nchunks,
                                                           const int* __restrict__ dcount)
{
    constexpr int NT = 256 / CPT;
    if (dcount) nchunks = *dcount;   // queue length in device memory (a server's patched queue)
    for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const TileRef tr = chunks[ch];
        const GridDev& G = grids[tr.grid];
        const Ctrl* C = G.ctrl;
        if (C->done) continue;                      // uniform over the block (one grid per chunk)
        const int par = C->par;
        const long long PL = (long long)G.nx * G.ny;
        double dtmin = INFINITY;
        bool bad = false;
#pragma unroll
        for (int m = 0; m < CPT; ++m) {
            const long long cell = (long long)tr.x0 + threadIdx.x + m * NT;
            if (cell < PL) update_cell<STAGE>(G, par, cell, dtmin, bad);
        }
        if (STAGE == 2) {
            if (bad) atomicOr(&G.ctrl->status, (int)CGKS_E_NONPHYSICAL);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dtmin = fmin(dtmin, __shfl_xor_sync(0xffffffffu, dtmin, o));
            if ((threadIdx.x & 31) == 0 && dtmin < INFINITY)
                atomicMin(&G.ctrl->dtmin_bits, (unsigned long long)__double_as_longlong(dtmin));
        }
    }
}

std::vector<TileRef> cell_chunks(int nx, int ny, int grid)
{
    const long long cells = (long long)nx * ny;
    std::vector<TileRef> c;
    for (long long s = 0; s < cells; s += 256) c.push_back(TileRef{grid, (int)s, 0, 0});
    return c;
}

cudaError_t launch_update(int stage, const GridDev* grids, const TileRef* chunks, int nchunks, int nblocks,
                          cudaStream_t st, const int* dcount, int cpt)
{
    if (nchunks <= 0 || nblocks <= 0) return cudaSuccess;
#define CGKS_UPDATE_LAUNCH(S, C) update_kernel<S, C><<<nblocks, 256 / C, 0, st>>>(grids, chunks, nchunks, dcount)
    if (stage == 1) {
        if (cpt == 4) CGKS_UPDATE_LAUNCH(1, 4);
        else if (cpt == 2) CGKS_UPDATE_LAUNCH(1, 2);
        else CGKS_UPDATE_LAUNCH(1, 1);
    } else {
        if (cpt == 4) CGKS_UPDATE_LAUNCH(2, 4);
        else if (cpt == 2) CGKS_UPDATE_LAUNCH(2, 2);
        else CGKS_UPDATE_LAUNCH(2, 1);
    }
#undef CGKS_UPDATE_LAUNCH
    return cudaGetLastError();
}

}  // namespace cgks
