// cgks_records.cu -- the face-row records of one stage: the normal
// reconstruction of every face row of a grid (linear compact reconstruction,
// Sec. 3.2, Eq. recons-8th-val; nonlinear WENO-Z left and right states with
// their slopes, Sec. 3.3), computed once per row and written to global memory,
// where the flux kernels of all tiles that share the row read it.
//
// A record holds 7 fields x 4 variables (face frame: density, normal momentum,
// tangential momentum, energy): RV, RN, RNN (P7, P7_n, P7_nn) and, for the rows
// the non-equilibrium states are needed on, RL, RR (WENO-Z values) and RLN, RRN
// (their normal slopes).  x-face rows: faces 0..nx, rows -2..ny+1; y-face rows
// (2D): faces 0..ny, columns -2..nx+1.  Ghost cells of the stencils are the
// boundary conditions applied on the fly: x-boundaries first, then y, so the
// corners match the oracle's ghost layers.
#include "cgks_records.cuh"

namespace cgks {

__constant__ ReconTab kReconTab = make_recon_tab();

// CHAR = 0: conservative variables, one (record, variable) per thread;
// CHAR = 1: characteristic variables, one record (all four variables) per thread.
// The reconstruction order is per grid (a uniform branch per chunk).
template <int STAGE, int CHAR>
__global__ void __launch_bounds__(256, CHAR ? 1 : 2) records_kernel(const GridDev* __restrict__ grids,
                                                                    const TileRef* __restrict__ chunks, int nchunks,
                                                                    const int* __restrict__ dcount)
{
    if (dcount) nchunks = *dcount;   // queue length in device memory (a server's patched queue)
    __shared__ double s_tab[2 * RK_N];
    for (int i = threadIdx.x; i < 2 * RK_N; i += blockDim.x) s_tab[i] = kReconTab.v[i / RK_N][i % RK_N];
    __syncthreads();
    const double one = ((volatile const double*)s_tab)[RK_ONE];
    const double nzero = ((volatile const double*)s_tab)[RK_NZERO];
    for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const TileRef tr = chunks[ch];
        const GridDev& G = grids[tr.grid];
        if (G.ctrl->done) continue;
        const double* __restrict__ src = (STAGE == 1) ? G.buf[G.ctrl->par] : G.ws;
        const size_t PL = (size_t)G.nx * G.ny;
        const int nrec = record_rows(G.nx, G.ny, G.dim);
        const int item = tr.x0 + (int)threadIdx.x;
        if (!CHAR) {
            if (item >= 4 * nrec) continue;
            const int k = item / nrec;
            if (G.order == 6) cons_row<6>(RegK{s_tab + RK_N, one, nzero}, G, src, PL, item - k * nrec, k);
            else cons_row<8>(RegK{s_tab, one, nzero}, G, src, PL, item - k * nrec, k);
        } else {
            if (item >= nrec) continue;
            if (G.order == 6) char_row<6>(RegK{s_tab + RK_N, one, nzero}, G, src, PL, item);
            else char_row<8>(RegK{s_tab, one, nzero}, G, src, PL, item);
        }
    }
}

std::vector<TileRef> record_chunks(int nx, int ny, int dim, int recon_vars, int grid)
{
    const long long items = (long long)(recon_vars ? 1 : 4) * record_rows(nx, ny, dim);
    std::vector<TileRef> c;
    for (long long s = 0; s < items; s += 256) c.push_back(TileRef{grid, (int)s, 0, 0});
    return c;
}

cudaError_t launch_records(int stage, int char_vars, const GridDev* grids, const TileRef* chunks, int nchunks,
                           int nblocks, cudaStream_t st, const int* dcount)
{
    if (nchunks <= 0 || nblocks <= 0) return cudaSuccess;
    if (char_vars) {
        if (stage == 1) records_kernel<1, 1><<<nblocks, 256, 0, st>>>(grids, chunks, nchunks, dcount);
        else records_kernel<2, 1><<<nblocks, 256, 0, st>>>(grids, chunks, nchunks, dcount);
    } else {
        if (stage == 1) records_kernel<1, 0><<<nblocks, 256, 0, st>>>(grids, chunks, nchunks, dcount);
        else records_kernel<2, 0><<<nblocks, 256, 0, st>>>(grids, chunks, nchunks, dcount);
    }
    return cudaGetLastError();
}

}  // namespace cgks
