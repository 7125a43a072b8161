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
#include "cgks_update.cuh"

namespace cgks {

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
