// cgks_internal.h -- device-side data structures shared by the kernels and the
// host runtime of libcgks (not part of the public C ABI in include/cgks.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <utility>
#include <vector>

#include "../../include/cgks.h"

namespace cgks {

// devices whose per-device state (kernel attributes, fixed-array addresses) the
// library tracks
constexpr int kMaxDevices = 64;

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

// Ctrl.status bit raised by a build with CGKS_CHECK_BOUNDS when a kernel index
// falls outside its buffer (the access is skipped); the host reports it as a
// CUDA error.  Other builds never set it.
constexpr int kStatusBounds = 1 << 8;

// Per-grid descriptor (read-only for kernels).
struct GridDev {
    double* buf[2];     // current state / next state ping-pong, 12 planes each
    double* ws;         // intermediate state W* (12 planes)
    Ctrl* ctrl;
    int nx, ny, dim, recon_vars;
    int order;          // 8: compact 8th-order reconstruction; 6: the 6th-order variant
    int bc[4];
    double dx, dy, inv_dx, inv_dy;
    double gamma, K, cfl, eps_tau, c_tau, weno_eps;
    double mu;          // > 0: viscous collision time mu/p
    double inflow[4][4];   // conservative inflow state per side (x-low, x-high, y-low, y-high)
    double* recx;       // face-row records of the stage in flight: x-faces [7][4][ny+4][nx+1]
    double* recy;       // y-faces [7][4][nx+4][ny+1] (2D)
    double* facex;      // face results of the stage in flight: x-faces [16][ny][nx+1]
    double* facey;      // y-faces [16][ny+1][nx] (2D)
};

#if defined(__CUDACC__) || defined(CGKS_OPCOUNT_HOST)
// Bounds check of the CGKS_CHECK_BOUNDS build: true if ok; otherwise the grid's
// status records it.  In other builds it is true and the condition is not evaluated.
#if defined(CGKS_CHECK_BOUNDS) && defined(__CUDACC__)
__device__ __forceinline__ bool in_bounds(bool ok, Ctrl* c)
{
    if (!ok) atomicOr(&c->status, kStatusBounds);
    return ok;
}
#define CGKS_IN_BOUNDS(cond, ctrl) ::cgks::in_bounds((cond), (ctrl))
#else
#define CGKS_IN_BOUNDS(cond, ctrl) true
#endif

// CFL bound of one cell, dx/(|U|+c+2 nu/dx) and dy/(|V|+c+2 nu/dy) (Sec. 4; nu =
// mu/rho), written with explicitly rounded operations so that every kernel that
// evaluates it (the stage-2 update of a step, the bound of a state that was set
// or restored) gets the same bits: a restored checkpoint continues exactly as
// the uninterrupted run.  Returns false for rho <= 0 or p <= 0 (or NaN).
__device__ __forceinline__ bool cfl_cell_bound(const GridDev& G, double r, double m, double n, double E, bool dim1,
                                               double* d_out)
{
    const double ir = __ddiv_rn(1.0, r);
    const double U = __dmul_rn(m, ir), V = __dmul_rn(n, ir);
    const double ke = __dmul_rn(0.5, __dadd_rn(__dmul_rn(m, U), __dmul_rn(n, V)));
    const double p = __dmul_rn(__dsub_rn(G.gamma, 1.0), __dsub_rn(E, ke));
    if (!(r > 0.0) || !(p > 0.0)) return false;
    const double c = __dsqrt_rn(__dmul_rn(__dmul_rn(G.gamma, p), ir));
    const double two_nu = __dmul_rn(2.0, __dmul_rn(G.mu, ir));
    double d = __ddiv_rn(G.dx, __dadd_rn(__dadd_rn(fabs(U), c), __dmul_rn(two_nu, G.inv_dx)));
    if (!dim1) d = fmin(d, __ddiv_rn(G.dy, __dadd_rn(__dadd_rn(fabs(V), c), __dmul_rn(two_nu, G.inv_dy))));
    *d_out = d;
    return true;
}
#endif

// face rows with a record: x-faces 0..nx on rows -2..ny+1, y-faces 0..ny on
// columns -2..nx+1 (2D); each record holds 7 fields x 4 variables
__host__ __device__ inline int record_rows(int nx, int ny, int dim)
{
    return (nx + 1) * (ny + 4) + (dim == 2 ? (ny + 1) * (nx + 4) : 0);
}
inline size_t record_doubles(int nx, int ny, int dim) { return (size_t)28 * record_rows(nx, ny, dim); }
// per face up to 16 results (stage 1: two flux combinations, two interface states)
inline size_t face_doubles(int nx, int ny, int dim)
{
    return (size_t)16 * ((size_t)(nx + 1) * ny + (dim == 2 ? (size_t)(ny + 1) * nx : 0));
}

// One unit of work of the stage kernels: a TX x TY tile of one grid.
struct TileRef { int grid, x0, y0, pad; };

// tile shapes compiled into the library, in the public numbering of
// cgks_set_tile_shape.  The flux kernel runs one face segment per thread and a
// tile owns 2 TX TY segments (plus the grid's last faces on its edges), so
// 16x8 (256), 16x16 (512), 24x16 and 32x12 (768) fill whole passes of
// the 256-thread CTA; a tile's records must fit 227 KB of shared memory.
#define CGKS_FOR_EACH_TILE(X) X(16, 8) X(8, 16) X(32, 4) X(64, 1) X(16, 7) X(7, 16) X(14, 8) X(24, 8) \
    X(16, 14) X(20, 11) X(15, 15) X(22, 10) X(18, 12) X(20, 12) X(15, 16) X(17, 14) X(16, 16) X(24, 16) X(32, 12)
#define CGKS_TILE_ENUM(w, h) TILE_##w##x##h,
enum TileShape { CGKS_FOR_EACH_TILE(CGKS_TILE_ENUM) TILE_COUNT };
#undef CGKS_TILE_ENUM
#define CGKS_TILE_W(w, h) w,
#define CGKS_TILE_H(w, h) h,
inline int tile_w(int s) { static const int v[TILE_COUNT] = {CGKS_FOR_EACH_TILE(CGKS_TILE_W)}; return v[s]; }
inline int tile_h(int s) { static const int v[TILE_COUNT] = {CGKS_FOR_EACH_TILE(CGKS_TILE_H)}; return v[s]; }
#undef CGKS_TILE_W
#undef CGKS_TILE_H

// the record kernel's work queue: chunks of 256 (record, variable) items of one
// grid (one record per item in characteristic mode); TileRef.x0 is the first item
std::vector<TileRef> record_chunks(int nx, int ny, int dim, int recon_vars, int grid);
// the update kernel's work queue: chunks of 256 cells of one grid (TileRef.x0
// is the first cell)
std::vector<TileRef> cell_chunks(int nx, int ny, int grid);
// cpt: cells per thread of the update kernel (1, 2 or 4: CTAs of 256, 128 or 64
// threads per chunk of 256 cells)
cudaError_t launch_update(int stage, const GridDev* grids, const TileRef* chunks, int nchunks, int nblocks,
                          cudaStream_t st, const int* dcount = nullptr, int cpt = 1);
// persistent grid of the update kernel: up to 8 resident CTAs per SM
inline int update_blocks(int nchunks, int nsm, int cpt = 1)
{
    const int cap = 8 * cpt * nsm;
    return nchunks < cap ? nchunks : cap;
}
// flux kernel: two resident CTAs of 128 threads per SM (one stages its tile
// while the other computes)
constexpr int kStageCtasPerSm = 2;
inline int stage_blocks(int ntiles, int nsm)
{
    return ntiles < kStageCtasPerSm * nsm ? ntiles : kStageCtasPerSm * nsm;
}

// persistent grid of the record kernel: its resident CTAs (two per SM with
// conservative variables, one with characteristic ones), at most one per chunk
inline int record_blocks(int nchunks, int nsm, int char_vars)
{
    const int cap = (char_vars ? 1 : 2) * nsm;
    return nchunks < cap ? nchunks : cap;
}

// launchers (defined in the kernel translation units).  The persistent kernels
// stride over a work queue of `n` entries; a non-NULL `dcount` points to an int
// in device memory that holds the queue's current length instead (read when the
// kernel starts), so that a captured graph keeps working while a server patches
// its queues between replays.
cudaError_t launch_records(int stage, int char_vars, const GridDev* grids, const TileRef* chunks, int nchunks,
                           int nblocks, cudaStream_t st, const int* dcount = nullptr);
cudaError_t launch_stage(int shape, int stage, const GridDev* grids, const TileRef* tiles, int ntiles,
                         int nblocks, cudaStream_t st, const int* dcount = nullptr);
size_t stage_smem_bytes(int shape, int stage);
// the fused step (cgks_fused.cu): both stages of a step in one launch over 16 x 8
// tiles (make_tiles with TILE_16x8), one CTA of 256 threads per SM
cudaError_t launch_fused_step(const GridDev* grids, const TileRef* tiles, int ntiles, int nblocks, cudaStream_t st);
cudaError_t launch_begin_step(const GridDev* grids, int ngrids, cudaStream_t st);
cudaError_t launch_end_step(const GridDev* grids, int ngrids, cudaStream_t st);
cudaError_t launch_cfl(const GridDev* grids, int gidx, const GridDev& host, cudaStream_t st);
cudaError_t launch_expand1d(const double* src6, double* dst12, int nx, cudaStream_t st);
cudaError_t launch_compress1d(const double* src12, double* dst6, int nx, cudaStream_t st);
// reset != 0: the control block starts a solve at time t with `steps0` steps
// already taken (0 for a new solve, the checkpoint's count on a restore)
cudaError_t launch_set_ctrl(Ctrl* c, double t, double t_end, long long steps_target, int reset, cudaStream_t st,
                            long long steps0 = 0);
cudaError_t launch_batch_resume(const GridDev* grids, int n, cudaStream_t st);

}  // namespace cgks

// A solver: one grid's device planes, control block, descriptor and queues
// (the object behind the opaque cgks_solver of the C ABI).
struct cgks_solver {
    cgks_problem prob;
    size_t device_bytes = 0;
    int nx = 0, ny = 0;
    int device = 0;
    int nsm = 1;
    cudaStream_t stream = nullptr;
    double* d_planes = nullptr;   // 3 x 12 planes: buf0, buf1, ws
    double* d_records = nullptr;  // face-row records of the stage in flight
    cgks::TileRef* d_rchunks = nullptr; // record-kernel work queue
    int nrchunks = 0;
    double* d_faces = nullptr;    // face results of the stage in flight
    cgks::TileRef* d_cchunks = nullptr; // update-kernel work queue
    int ncchunks = 0;
    double* d_stage1d = nullptr;  // 6-plane staging for dim 1
    cgks::Ctrl* d_ctrl = nullptr;
    cgks::GridDev host_desc;
    cgks::GridDev* d_desc = nullptr;
    cgks::TileRef* d_tiles = nullptr;
    int ntiles = 0;
    int shape = cgks::TILE_16x8;
    cgks::TileRef* d_ftiles = nullptr;  // 16 x 8 tiles of the fused step (made at its first call)
    int nftiles = 0;
};

namespace cgks {

// the descriptor of a grid of problem p whose buffers start at the given
// device addresses (planes: 3 x 12 planes of nx*ny)
void fill_grid_desc(const cgks_problem& p, double* planes, double* records, double* faces, Ctrl* ctrl, GridDev& G);
// device bytes of one grid's planes, records and face results
size_t grid_device_bytes(const cgks_problem& p);
// argument checks of a problem (CGKS_OK or CGKS_E_INVAL with the detail in
// cgks_last_error)
cgks_status validate_problem(const cgks_problem* p);

// ---------------------------------------------------------------------------
// The batched engine: many grids of any size advance together, one persistent
// launch per kernel and stage over flattened work queues of all of them,
// replayed as a CUDA graph.  Grids sit in slots of a descriptor table; an
// empty slot points to a control block marked done.  The queues and their
// lengths live in device memory and may be rewritten between replays (on the
// engine's stream), so one captured graph per candidate serves every
// composition of the slots.  A candidate is a tile shape of the flux kernel
// (the face segments per thread follow from it) and a cells-per-thread count
// of the update kernel; the tuner times each candidate on the first steps
// (shapes first, then cells per thread with the best shape) and keeps the
// fastest; no candidate changes a result.
struct BatchCand { int shape, cpt; };

class BatchEngine {
public:
    // nslots: size of the descriptor table; forced_shape >= 0 fixes the tile
    // shape (no tuning of the shape)
    static cudaError_t create(int nslots, int dim, cudaStream_t stream, int forced_shape, BatchEngine** out);
    ~BatchEngine();

    // Set the grids of the slots (slot index, descriptor); the others become
    // empty.  Rebuilds the queues and enqueues their upload on the stream, so
    // the next replay sees the new composition.
    cudaError_t set_members(const std::vector<std::pair<int, GridDev>>& members);
    // Enqueue nsteps steps.  While the tuner runs it times candidates (one
    // tuning step per call synchronises the stream).
    cudaError_t run(int nsteps, long* launches, bool tune = true);
    // Enqueue one replay of candidate `cand` for `nsteps` steps, bracketed by
    // the events (either may be NULL): the server times its rounds with them.
    cudaError_t replay(int cand, int nsteps, cudaEvent_t before, cudaEvent_t after, long* launches);
    // Enqueue a copy of every slot's control block into dst (nslots entries).
    cudaError_t snapshot(Ctrl* dst);
    // The tuner's current choice, or -1 while candidates are still timed.
    int chosen() const { return chosen_; }
    // the candidate the next step runs, and the tuner's record of its time
    int next_candidate() const;
    void record_time(int cand, double ms_per_cell_step);
    const BatchCand& candidate(int k) const { return cands_[k]; }
    int ncandidates() const { return (int)cands_.size(); }
    long long member_cells() const { return cells_; }
    int launches_per_step() const { return launches_per_step_; }
    long captures() const { return captures_; }
    cudaStream_t stream() const { return stream_; }
    const GridDev* device_table() const { return d_grids_; }

private:
    BatchEngine() = default;
    cudaError_t ensure_capacity(int k, size_t n);
    cudaError_t capture(int cand);
    int nslots_ = 0, dim_ = 2, nsm_ = 1;
    cudaStream_t stream_ = nullptr;
    GridDev* d_grids_ = nullptr;
    Ctrl* d_dummy_ = nullptr;
    // device queues: [0, TILE_COUNT) tiles per shape, then records (2), cells
    static constexpr int kQ = TILE_COUNT + 3;
    TileRef* d_q_[kQ] = {};
    size_t cap_[kQ] = {};
    int* d_counts_ = nullptr;
    // pinned staging of the uploads, reused once the previous upload finished
    char* h_stage_ = nullptr;
    size_t stage_cap_ = 0;
    cudaEvent_t stage_done_ = nullptr;
    std::vector<BatchCand> cands_;
    std::vector<cudaGraphExec_t> exec_;
    std::vector<double> trial_;
    int chosen_ = -1, tune_phase_ = 0, trial_next_ = 0;
    long long cells_ = 0;
    int launches_per_step_ = 0;
    long captures_ = 0;
};

}  // namespace cgks
