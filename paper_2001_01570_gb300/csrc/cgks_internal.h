// cgks_internal.h -- device-side data structures shared by the kernels and the
// host runtime of libcgks (not part of the public C ABI in include/cgks.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <vector>

namespace cgks {

// Per-grid control block in device memory.  Written only by the step-control
// kernels and the stage kernels, so a sequence of steps (or a CUDA graph of
// them) runs without any host round trip.
struct Ctrl {
    double dt;                        // time step of the step in flight
    double t;                         // simulated time of the state in buf[par]
    double t_end;                     // > 0: clip the last step to reach t_end, then stop
    unsigned long long dtmin_bits;    // min over cells of dx/(|U|+c) (positive double bits)
    int status;                       // CGKS_E_* bits raised by kernels
    int done;                         // 1: no further steps run on this grid
    int par;                          // index of the buffer holding the current state
    int pad;
    long long steps;                  // steps completed
    long long steps_target;           // < 0: unlimited
};

// Per-grid descriptor (read-only for kernels).
struct GridDev {
    double* buf[2];     // current state / next state ping-pong, 12 planes each
    double* ws;         // intermediate state W* (12 planes)
    Ctrl* ctrl;
    int nx, ny, dim, recon_vars;
    int bc[4];
    double dx, dy, inv_dx, inv_dy;
    double gamma, K, cfl, eps_tau, c_tau, weno_eps;
    double mu;          // > 0: viscous collision time mu/p
    double inflow[4][4];   // conservative inflow state per side (x-low, x-high, y-low, y-high)
};

// One unit of work of the stage kernels: a TX x TY tile of one grid.
struct TileRef { int grid, x0, y0, pad; };

// tile shapes compiled into the library.  16x7, 7x16 and 14x8 give 247, 247
// and 246 face segments per tile, i.e. one pass of the 256-thread CTA over the
// heaviest phase (16x8 needs 280: a second pass with a single warp)
// 24x8 trades a second, five-warp pass over the segments for less halo
// recomputation (2.52 instead of 2.65 WENO records per cell).
enum TileShape { TILE_16x8 = 0, TILE_8x16 = 1, TILE_32x4 = 2, TILE_64x1 = 3, TILE_16x7 = 4, TILE_7x16 = 5,
                 TILE_14x8 = 6, TILE_24x8 = 7, TILE_COUNT = 8 };
inline int tile_w(int s) { static const int w[TILE_COUNT] = {16, 8, 32, 64, 16, 7, 14, 24}; return w[s]; }
inline int tile_h(int s) { static const int h[TILE_COUNT] = {8, 16, 4, 1, 7, 16, 8, 8}; return h[s]; }

// launchers (defined in the kernel translation units)
cudaError_t launch_stage(int shape, int stage, const GridDev* grids, const TileRef* tiles, int ntiles,
                         int nblocks, cudaStream_t st);
size_t stage_smem_bytes(int shape, int stage);
cudaError_t launch_begin_step(const GridDev* grids, int ngrids, cudaStream_t st);
cudaError_t launch_end_step(const GridDev* grids, int ngrids, cudaStream_t st);
cudaError_t launch_cfl(const GridDev* grids, int gidx, const GridDev& host, cudaStream_t st);
cudaError_t launch_expand1d(const double* src6, double* dst12, int nx, cudaStream_t st);
cudaError_t launch_compress1d(const double* src12, double* dst6, int nx, cudaStream_t st);
cudaError_t launch_set_ctrl(Ctrl* c, double t, double t_end, long long steps_target, int reset, cudaStream_t st);
cudaError_t launch_batch_resume(const GridDev* grids, int n, cudaStream_t st);

}  // namespace cgks

struct cgks_solver;

namespace cgks {

// A batch of solvers stepped together: device descriptor array, one tile
// queue and one captured step graph per candidate tile shape.
struct BatchPlan {
    std::vector<cgks_solver*> solvers;
    cudaStream_t stream = nullptr;
    int nsm = 1, dim = 2;
    long long cells = 0;
    GridDev* d_grids = nullptr;
    TileRef* d_tiles[TILE_COUNT] = {};
    int ntiles[TILE_COUNT] = {};
    cudaGraphExec_t exec[TILE_COUNT] = {};
    std::vector<int> candidates;
    int chosen = -1, trial_idx = 0;
    float trial_ms[TILE_COUNT] = {};
    int trial_count[TILE_COUNT] = {};
};

cudaError_t make_plan(cgks_solver* const* solvers, int n, cudaStream_t stream, int forced_shape, BatchPlan** out);
cudaError_t run_plan(BatchPlan* bp, int nsteps, long* launches);
void destroy_plan(BatchPlan* bp);

}  // namespace cgks
