// cgks_fused.cu -- the fused step kernel: both stages of one two-stage
// fourth-order step (Sec. 2.2) per 16 x 8 tile, W* in shared memory
// (cgks_fused.cuh), one launch per step between the step-control kernels.
// Every tile recomputes stage 1 on its tile widened by two cells, so the kernel
// does more FP64 work than the three-kernel step (records, flux and update per
// stage) and is slower on this FP64-bound path; it is kept as the measured
// alternative and gives the same bits.
#include "cgks_fused.cuh"

#include <mutex>

namespace cgks {

static __constant__ FluxFixed kFusedFluxFixed = make_flux_fixed();
static __constant__ ReconTab kFusedReconTab = make_recon_tab();

template <int TX, int TY>
__global__ void __launch_bounds__(kFusedThreads, 1)
fused_step_kernel(const GridDev* __restrict__ grids, const TileRef* __restrict__ tiles, int ntiles)
{
    using L = FusedLayout<TX, TY>;
    extern __shared__ double smem[];
    __shared__ double s_fk[FK_N];
    __shared__ double s_rk[2 * RK_N];
    __shared__ int s_skip;
    const int tid = threadIdx.x;
    for (int i = tid; i < FK_NFIX; i += kFusedThreads) s_fk[i] = kFusedFluxFixed.v[i];
    if (tid < 32) s_fk[FK_EXP2 + tid] = exp2((double)tid * (1.0 / 32.0));
    for (int i = tid; i < 2 * RK_N; i += kFusedThreads) s_rk[i] = kFusedReconTab.v[i / RK_N][i % RK_N];
    __syncthreads();
    const double one = ((volatile const double*)s_fk)[FK_ONE], nzero = ((volatile const double*)s_fk)[FK_NZERO];
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
        const FusedTile<TX, TY> T{G,
                                  smem,
                                  smem + L::nP,
                                  RegK{s_fk, one, nzero},
                                  RegK{s_rk + (G.order == 6 ? RK_N : 0), one, nzero},
                                  tr.x0,
                                  tr.y0,
                                  G.ctrl->par,
                                  G.bc[0] == CGKS_BC_PERIODIC,
                                  G.bc[2] == CGKS_BC_PERIODIC};
        bool bad = false;
        double dtmin = INFINITY;
        T.records1(tid, kFusedThreads);
        __syncthreads();
        bad |= !T.flux1(tid, kFusedThreads);
        __syncthreads();
        T.update1(tid, kFusedThreads);
        __syncthreads();
        T.records2(tid, kFusedThreads);
        __syncthreads();
        bad |= !T.flux2(tid, kFusedThreads);
        __syncthreads();
        T.update2(tid, kFusedThreads, dtmin, bad);
        if (bad) atomicOr(&G.ctrl->status, (int)CGKS_E_NONPHYSICAL);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dtmin = fmin(dtmin, __shfl_xor_sync(0xffffffffu, dtmin, o));
        if ((tid & 31) == 0 && dtmin < INFINITY)
            atomicMin(&G.ctrl->dtmin_bits, (unsigned long long)__double_as_longlong(dtmin));
    }
}

// more than 48 KB of dynamic shared memory: set once per device before the first launch
template <int TX, int TY>
static cudaError_t configure_fused()
{
    static std::once_flag once[kMaxDevices];
    static cudaError_t status[kMaxDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::call_once(once[dev], [dev] {
        status[dev] = cudaFuncSetAttribute(fused_step_kernel<TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)FusedLayout<TX, TY>::bytes);
    });
    return status[dev];
}

static_assert(FusedLayout<kFusedTX, kFusedTY>::bytes + sizeof(double) * (FK_N + 2 * RK_N) + 64 <= 227 * 1024,
              "fused tile exceeds shared memory");

cudaError_t launch_fused_step(const GridDev* grids, const TileRef* tiles, int ntiles, int nblocks, cudaStream_t st)
{
    cudaError_t e = configure_fused<kFusedTX, kFusedTY>();
    if (e != cudaSuccess) return e;
    if (ntiles <= 0 || nblocks <= 0) return cudaSuccess;
    fused_step_kernel<kFusedTX, kFusedTY>
        <<<nblocks, kFusedThreads, FusedLayout<kFusedTX, kFusedTY>::bytes, st>>>(grids, tiles, ntiles);
    return cudaGetLastError();
}

}  // namespace cgks
