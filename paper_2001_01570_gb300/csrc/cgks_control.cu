// cgks_control.cu -- step-control kernels (CFL time step, step begin/end),
// state layout conversions and the stage-kernel dispatcher.
#include "cgks_internal.h"
#include "../../include/cgks.h"
#include <math.h>

namespace cgks {

#define CGKS_DECLARE_TILE(w, h)                                                                          \
    cudaError_t launch_stage_##w##x##h(int, const GridDev*, const TileRef*, int, int, cudaStream_t, const int*); \
    size_t smem_##w##x##h(int);
CGKS_FOR_EACH_TILE(CGKS_DECLARE_TILE)
#undef CGKS_DECLARE_TILE

cudaError_t launch_stage(int shape, int stage, const GridDev* grids, const TileRef* tiles, int ntiles, int nblocks,
                         cudaStream_t st, const int* dcount)
{
    switch (shape) {
#define CGKS_LAUNCH_CASE(w, h) \
    case TILE_##w##x##h: return launch_stage_##w##x##h(stage, grids, tiles, ntiles, nblocks, st, dcount);
    CGKS_FOR_EACH_TILE(CGKS_LAUNCH_CASE)
#undef CGKS_LAUNCH_CASE
    default: return cudaErrorInvalidValue;
    }
}

size_t stage_smem_bytes(int shape, int stage)
{
    switch (shape) {
#define CGKS_SMEM_CASE(w, h) \
    case TILE_##w##x##h: return smem_##w##x##h(stage);
    CGKS_FOR_EACH_TILE(CGKS_SMEM_CASE)
#undef CGKS_SMEM_CASE
    default: return 0;
    }
}

static __device__ __forceinline__ unsigned long long inf_bits() { return 0x7ff0000000000000ull; }

// Start of a step: dt = CFL * (min over cells of dx/(|U|+c+2 nu/dx)) of the current
// state, clipped so that t does not pass t_end; marks grids that are finished.
__global__ void begin_step_kernel(const GridDev* grids, int n)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    Ctrl* C = grids[g].ctrl;
    if (C->done) return;
    if (C->status) { C->done = 1; return; }
    if (C->steps_target >= 0 && C->steps >= C->steps_target) { C->done = 1; return; }
    if (C->t_end > 0.0 && C->t >= C->t_end) { C->done = 1; return; }
    double dt = grids[g].cfl * __longlong_as_double((long long)C->dtmin_bits);
    if (!(dt > 0.0) || isinf(dt)) { C->status |= CGKS_E_NONPHYSICAL; C->done = 1; return; }
    if (C->t_end > 0.0 && C->t + dt > C->t_end) dt = C->t_end - C->t;
    C->dt = dt;
    C->dtmin_bits = inf_bits();
}

// End of a step: the new state becomes current unless a kernel raised an error.
__global__ void end_step_kernel(const GridDev* grids, int n)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    Ctrl* C = grids[g].ctrl;
    if (C->done) return;
    if (C->status) { C->done = 1; return; }
    C->par ^= 1;
    C->t += C->dt;
    C->steps += 1;
}

// CFL bound of the current state (after a state is set).
__global__ void cfl_kernel(const GridDev* grids, int gidx)
{
    const GridDev& G = grids[gidx];
    const size_t PL = (size_t)G.nx * G.ny;
    const double* W = G.buf[G.ctrl->par];
    double dmin = INFINITY;
    bool bad = false;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < PL; c += (size_t)gridDim.x * blockDim.x) {
        double d;
        if (!cfl_cell_bound(G, W[c], W[PL + c], W[2 * PL + c], W[3 * PL + c], G.dim == 1, &d)) { bad = true; continue; }
        dmin = fmin(dmin, d);
    }
    if (bad) atomicOr(&G.ctrl->status, (int)CGKS_E_NONPHYSICAL);
    for (int o = 16; o > 0; o >>= 1) dmin = fmin(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
    if ((threadIdx.x & 31) == 0 && dmin < INFINITY)
        atomicMin(&G.ctrl->dtmin_bits, (unsigned long long)__double_as_longlong(dmin));
}

__global__ void set_ctrl_kernel(Ctrl* c, double t, double t_end, long long steps_target, int reset, long long steps0)
{
    if (reset) {
        c->t = t;
        c->steps = steps0;
        c->status = 0;
        c->done = 0;
        c->par = 0;
        c->dt = 0.0;
        c->dtmin_bits = inf_bits();
    } else if (!c->status) {
        // a new request may continue a solve that was stopped by its step target or t_end
        c->done = 0;
    }
    c->t_end = t_end;
    c->steps_target = steps_target;
}

// a batch call continues every grid of the batch that has no error: no step
// target, no end time
__global__ void batch_resume_kernel(const GridDev* grids, int n)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    Ctrl* c = grids[g].ctrl;
    if (!c->status) c->done = 0;
    c->t_end = 0.0;
    c->steps_target = -1;
}

// 1D planes (rho, rhoU, rhoE, their x-gradients) <-> the internal 2D layout
__global__ void expand1d_kernel(const double* src, double* dst, int nx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx) return;
    const int map[12] = {0, 1, -1, 2, 3, 4, -1, 5, -1, -1, -1, -1};
    for (int p = 0; p < 12; ++p) dst[(size_t)p * nx + i] = map[p] < 0 ? 0.0 : src[(size_t)map[p] * nx + i];
}

__global__ void compress1d_kernel(const double* src, double* dst, int nx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx) return;
    const int map[6] = {0, 1, 3, 4, 5, 7};
    for (int p = 0; p < 6; ++p) dst[(size_t)p * nx + i] = src[(size_t)map[p] * nx + i];
}

cudaError_t launch_begin_step(const GridDev* grids, int n, cudaStream_t st)
{
    begin_step_kernel<<<(n + 127) / 128, 128, 0, st>>>(grids, n);
    return cudaGetLastError();
}

cudaError_t launch_end_step(const GridDev* grids, int n, cudaStream_t st)
{
    end_step_kernel<<<(n + 127) / 128, 128, 0, st>>>(grids, n);
    return cudaGetLastError();
}

cudaError_t launch_cfl(const GridDev* grids, int gidx, const GridDev& host, cudaStream_t st)
{
    const size_t cells = (size_t)host.nx * host.ny;
    int blocks = (int)((cells + 255) / 256);
    if (blocks > 1024) blocks = 1024;
    cfl_kernel<<<blocks, 256, 0, st>>>(grids, gidx);
    return cudaGetLastError();
}

cudaError_t launch_set_ctrl(Ctrl* c, double t, double t_end, long long steps_target, int reset, cudaStream_t st,
                            long long steps0)
{
    set_ctrl_kernel<<<1, 1, 0, st>>>(c, t, t_end, steps_target, reset, steps0);
    return cudaGetLastError();
}

cudaError_t launch_batch_resume(const GridDev* grids, int n, cudaStream_t st)
{
    batch_resume_kernel<<<(n + 127) / 128, 128, 0, st>>>(grids, n);
    return cudaGetLastError();
}

cudaError_t launch_expand1d(const double* src6, double* dst12, int nx, cudaStream_t st)
{
    expand1d_kernel<<<(nx + 255) / 256, 256, 0, st>>>(src6, dst12, nx);
    return cudaGetLastError();
}

cudaError_t launch_compress1d(const double* src12, double* dst6, int nx, cudaStream_t st)
{
    compress1d_kernel<<<(nx + 255) / 256, 256, 0, st>>>(src12, dst6, nx);
    return cudaGetLastError();
}

}  // namespace cgks
