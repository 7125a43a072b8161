// cgks_api.cu -- host runtime behind the C ABI of include/cgks.h: solver
// objects (device planes, control block, tile queue), state transfer, the
// plain step loop and the batched CUDA-graph step over many grids.
#include "cgks_internal.h"
#include "../../include/cgks.h"

#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

using namespace cgks;

struct cgks_solver {
    cgks_problem prob;
    size_t device_bytes = 0;
    int nx = 0, ny = 0;
    int device = 0;
    int nsm = 1;
    cudaStream_t stream = nullptr;
    double* d_planes = nullptr;   // 3 x 12 planes: buf0, buf1, ws
    double* d_records = nullptr;  // face-row records of the stage in flight
    TileRef* d_rchunks = nullptr; // record-kernel work queue
    int nrchunks = 0;
    double* d_faces = nullptr;    // face results of the stage in flight
    TileRef* d_cchunks = nullptr; // update-kernel work queue
    int ncchunks = 0;
    double* d_stage1d = nullptr;  // 6-plane staging for dim 1
    Ctrl* d_ctrl = nullptr;
    GridDev host_desc;
    GridDev* d_desc = nullptr;
    TileRef* d_tiles = nullptr;
    int ntiles = 0;
    int shape = TILE_16x8;
};

namespace {

thread_local std::string g_last_error;
thread_local long g_last_launches = 0;

cgks_status fail(cgks_status st, const std::string& msg)
{
    g_last_error = msg;
    return st;
}

cgks_status cuda_fail(cudaError_t e, const char* where)
{
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return CGKS_E_CUDA;
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
    } while (0)

std::vector<TileRef> make_tiles(int nx, int ny, int shape, int grid)
{
    const int tw = tile_w(shape), th = tile_h(shape);
    std::vector<TileRef> t;
    for (int y0 = 0; y0 < ny; y0 += th)
        for (int x0 = 0; x0 < nx; x0 += tw) t.push_back(TileRef{grid, x0, y0, 0});
    return t;
}

cgks_status validate(const cgks_problem* p)
{
    if (!p) return fail(CGKS_E_INVAL, "problem is NULL");
    if (p->dim != 1 && p->dim != 2) return fail(CGKS_E_INVAL, "dim must be 1 or 2");
    const int ny = p->dim == 1 ? 1 : p->ny;
    if (p->nx < 1 || ny < 1) return fail(CGKS_E_INVAL, "nx and ny must be >= 1");
    const long long rows = (long long)(p->nx + 1) * (ny + 4) + (p->dim == 2 ? (long long)(ny + 1) * (p->nx + 4) : 0);
    if (4 * rows >= (1ll << 31)) return fail(CGKS_E_INVAL, "grid too large (face-row work items exceed 2^31)");
    if (!(p->x1 > p->x0) || (p->dim == 2 && !(p->y1 > p->y0))) return fail(CGKS_E_INVAL, "empty domain");
    if (!(p->gamma > 1.0) || !(p->gamma < 3.0)) return fail(CGKS_E_INVAL, "gamma out of range");
    if (!(p->cfl > 0.0)) return fail(CGKS_E_INVAL, "cfl must be > 0");
    if (!(p->eps_tau >= 0.0) || !(p->c_tau >= 0.0) || !(p->weno_eps > 0.0) || !(p->mu >= 0.0))
        return fail(CGKS_E_INVAL, "eps_tau, c_tau, mu must be >= 0 and weno_eps > 0");
    if (p->recon_vars != 0 && p->recon_vars != 1) return fail(CGKS_E_INVAL, "recon_vars must be 0 or 1");
    if (p->order != 0 && p->order != 6 && p->order != 8) return fail(CGKS_E_INVAL, "order must be 0, 6 or 8");
    const int nb = p->dim == 1 ? 2 : 4;
    for (int k = 0; k < nb; ++k) {
        if (p->bc[k] < CGKS_BC_PERIODIC || p->bc[k] > CGKS_BC_OUTFLOW) return fail(CGKS_E_INVAL, "unknown bc");
        const int n = k < 2 ? p->nx : ny;
        if (p->bc[k] == CGKS_BC_REFLECT && n < 2) return fail(CGKS_E_INVAL, "a reflecting side needs >= 2 cells");
    }
    if ((p->bc[0] == CGKS_BC_PERIODIC) != (p->bc[1] == CGKS_BC_PERIODIC))
        return fail(CGKS_E_INVAL, "periodic x needs both x sides periodic");
    if (p->dim == 2 && ((p->bc[2] == CGKS_BC_PERIODIC) != (p->bc[3] == CGKS_BC_PERIODIC)))
        return fail(CGKS_E_INVAL, "periodic y needs both y sides periodic");
    for (int k = 0; k < nb; ++k)
        if (p->bc[k] == CGKS_BC_INFLOW && (!(p->inflow[k][0] > 0.0) || !(p->inflow[k][3] > 0.0)))
            return fail(CGKS_E_INVAL, "inflow state needs rho > 0 and p > 0");
    return CGKS_OK;
}

cgks_status read_ctrl(cgks_solver* s, Ctrl* c)
{
    CK(cudaMemcpyAsync(c, s->d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return CGKS_OK;
}

int pick_shape(const cgks_problem& p)
{
    return p.dim == 1 ? TILE_64x1 : TILE_14x8;
}

}  // namespace

extern "C" {

const char* cgks_status_string(cgks_status st)
{
    switch (st) {
    case CGKS_OK: return "ok";
    case CGKS_E_INVAL: return "invalid argument";
    case CGKS_E_NOMEM: return "out of memory";
    case CGKS_E_BUDGET: return "request can never fit the memory budget";
    case CGKS_E_CUDA: return "CUDA error";
    case CGKS_E_NONPHYSICAL: return "non-physical state (rho <= 0, p <= 0 or NaN)";
    case CGKS_E_TIMEOUT: return "timeout";
    case CGKS_E_BUSY: return "busy";
    case CGKS_E_NOTFOUND: return "not found";
    }
    return "unknown status";
}

const char* cgks_last_error(void) { return g_last_error.c_str(); }

long cgks_last_launch_count(void) { return g_last_launches; }

double cgks_problem_device_bytes(const cgks_problem* prob)
{
    if (!prob || prob->nx < 1 || (prob->dim == 2 && prob->ny < 1)) return 0.0;
    const int ny = prob->dim == 1 ? 1 : prob->ny;
    const double cells = (double)prob->nx * ny;
    return 3.0 * 12.0 * cells * sizeof(double)
           + (double)(record_doubles(prob->nx, ny, prob->dim) + face_doubles(prob->nx, ny, prob->dim)) * sizeof(double)
           + 4096.0;
}

cgks_status cgks_create(const cgks_problem* prob, void* cuda_stream, cgks_solver** out)
{
    if (!out) return fail(CGKS_E_INVAL, "out is NULL");
    *out = nullptr;
    cgks_status st = validate(prob);
    if (st != CGKS_OK) return st;
    cgks_solver* s = new (std::nothrow) cgks_solver();
    if (!s) return fail(CGKS_E_NOMEM, "host allocation failed");
    s->prob = *prob;
    s->nx = prob->nx;
    s->ny = prob->dim == 1 ? 1 : prob->ny;
    s->stream = (cudaStream_t)cuda_stream;
    s->shape = pick_shape(*prob);
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, s->device);
    const size_t PL = (size_t)s->nx * s->ny;
    const size_t rec = record_doubles(s->nx, s->ny, prob->dim), fac = face_doubles(s->nx, s->ny, prob->dim);
    s->device_bytes = 3 * 12 * PL * sizeof(double) + (rec + fac) * sizeof(double);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_planes, 3 * 12 * PL * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&s->d_records, rec * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&s->d_faces, fac * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&s->d_ctrl, sizeof(Ctrl));
    if (e == cudaSuccess) e = cudaMalloc(&s->d_desc, sizeof(GridDev));
    if (e == cudaSuccess && prob->dim == 1) e = cudaMalloc(&s->d_stage1d, 6 * PL * sizeof(double));
    std::vector<TileRef> tiles = make_tiles(s->nx, s->ny, s->shape, 0);
    s->ntiles = (int)tiles.size();
    if (e == cudaSuccess) e = cudaMalloc(&s->d_tiles, tiles.size() * sizeof(TileRef));
    std::vector<TileRef> rchunks = record_chunks(s->nx, s->ny, prob->dim, prob->recon_vars, 0);
    s->nrchunks = (int)rchunks.size();
    if (e == cudaSuccess) e = cudaMalloc(&s->d_rchunks, rchunks.size() * sizeof(TileRef));
    std::vector<TileRef> cchunks = cell_chunks(s->nx, s->ny, 0);
    s->ncchunks = (int)cchunks.size();
    if (e == cudaSuccess) e = cudaMalloc(&s->d_cchunks, cchunks.size() * sizeof(TileRef));
    if (e != cudaSuccess) {
        cgks_destroy(s);
        return e == cudaErrorMemoryAllocation ? fail(CGKS_E_NOMEM, "device allocation failed")
                                              : cuda_fail(e, "cgks_create");
    }
    GridDev& G = s->host_desc;
    memset(&G, 0, sizeof(G));
    G.buf[0] = s->d_planes;
    G.buf[1] = s->d_planes + 12 * PL;
    G.ws = s->d_planes + 24 * PL;
    G.ctrl = s->d_ctrl;
    G.recx = s->d_records;
    G.recy = prob->dim == 2 ? s->d_records + (size_t)28 * (s->nx + 1) * (s->ny + 4) : nullptr;
    G.facex = s->d_faces;
    G.facey = prob->dim == 2 ? s->d_faces + (size_t)16 * (s->nx + 1) * s->ny : nullptr;
    G.nx = s->nx;
    G.ny = s->ny;
    G.dim = prob->dim;
    for (int k = 0; k < 4; ++k) G.bc[k] = (prob->dim == 1 && k >= 2) ? CGKS_BC_PERIODIC : prob->bc[k];
    G.dx = (prob->x1 - prob->x0) / prob->nx;
    G.dy = prob->dim == 1 ? 1.0 : (prob->y1 - prob->y0) / prob->ny;
    G.inv_dx = 1.0 / G.dx;
    G.inv_dy = 1.0 / G.dy;
    G.gamma = prob->gamma;
    // internal degrees of freedom of the 2D Maxwellian; a 1D problem runs as a
    // y-uniform 2D one, whose extra velocity direction plays the role of the
    // additional internal degree of freedom of the 1D model
    G.K = (4.0 - 2.0 * prob->gamma) / (prob->gamma - 1.0);
    G.cfl = prob->cfl;
    G.eps_tau = prob->eps_tau;
    G.c_tau = prob->c_tau;
    G.weno_eps = prob->weno_eps;
    G.mu = prob->mu;
    G.recon_vars = prob->recon_vars;
    G.order = prob->order == 6 ? 6 : 8;
    for (int side = 0; side < 4; ++side) {
        const double* q = prob->inflow[side];
        const double r = q[0], u = q[1], v = prob->dim == 1 ? 0.0 : q[2], p = q[3];
        G.inflow[side][0] = r;
        G.inflow[side][1] = r * u;
        G.inflow[side][2] = r * v;
        G.inflow[side][3] = p / (prob->gamma - 1.0) + 0.5 * r * (u * u + v * v);
    }
    e = cudaMemcpyAsync(s->d_desc, &G, sizeof(GridDev), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->d_tiles, tiles.data(), tiles.size() * sizeof(TileRef), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->d_rchunks, rchunks.data(), rchunks.size() * sizeof(TileRef), cudaMemcpyHostToDevice,
                            s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->d_cchunks, cchunks.data(), cchunks.size() * sizeof(TileRef), cudaMemcpyHostToDevice,
                            s->stream);
    if (e == cudaSuccess) e = launch_set_ctrl(s->d_ctrl, 0.0, 0.0, -1, 1, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        cgks_destroy(s);
        return cuda_fail(e, "cgks_create");
    }
    *out = s;
    return CGKS_OK;
}

extern "C" void cgks_forget_solver_plans(cgks_solver* s);

cgks_status cgks_set_tile_shape(cgks_solver* s, int shape)
{
    if (!s) return fail(CGKS_E_INVAL, "solver is NULL");
    if (shape < 0) shape = pick_shape(s->prob);
    if (shape >= TILE_COUNT) return fail(CGKS_E_INVAL, "unknown tile shape");
    if ((s->prob.dim == 1) != (shape == TILE_64x1)) return fail(CGKS_E_INVAL, "tile shape does not fit the dimension");
    std::vector<TileRef> tiles = make_tiles(s->nx, s->ny, shape, 0);
    TileRef* d = nullptr;
    CK(cudaMalloc(&d, tiles.size() * sizeof(TileRef)));
    cudaError_t e = cudaMemcpyAsync(d, tiles.data(), tiles.size() * sizeof(TileRef), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) { cudaFree(d); return cuda_fail(e, "cgks_set_tile_shape"); }
    cudaFree(s->d_tiles);
    s->d_tiles = d;
    s->ntiles = (int)tiles.size();
    s->shape = shape;
    return CGKS_OK;
}

cgks_status cgks_destroy(cgks_solver* s)
{
    if (!s) return fail(CGKS_E_INVAL, "solver is NULL");
    cgks_forget_solver_plans(s);
    if (s->d_planes || s->d_ctrl) cudaStreamSynchronize(s->stream);
    cudaFree(s->d_planes);
    cudaFree(s->d_records);
    cudaFree(s->d_rchunks);
    cudaFree(s->d_faces);
    cudaFree(s->d_cchunks);
    cudaFree(s->d_stage1d);
    cudaFree(s->d_ctrl);
    cudaFree(s->d_desc);
    cudaFree(s->d_tiles);
    delete s;
    return CGKS_OK;
}

static cgks_status set_state_impl(cgks_solver* s, const double* planes, int on_device, double t, long long steps)
{
    if (!s || !planes) return fail(CGKS_E_INVAL, "NULL argument");
    if (steps < 0) return fail(CGKS_E_INVAL, "steps must be >= 0");
    const size_t PL = (size_t)s->nx * s->ny;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(launch_set_ctrl(s->d_ctrl, t, 0.0, -1, 1, s->stream, steps));
    if (s->prob.dim == 1) {
        CK(cudaMemcpyAsync(s->d_stage1d, planes, 6 * PL * sizeof(double), kind, s->stream));
        CK(launch_expand1d(s->d_stage1d, s->host_desc.buf[0], s->nx, s->stream));
    } else {
        CK(cudaMemcpyAsync(s->host_desc.buf[0], planes, 12 * PL * sizeof(double), kind, s->stream));
    }
    CK(launch_cfl(s->d_desc, 0, s->host_desc, s->stream));
    if (!on_device) CK(cudaStreamSynchronize(s->stream));
    return CGKS_OK;
}

cgks_status cgks_set_state(cgks_solver* s, const double* planes, int on_device, double t)
{
    return set_state_impl(s, planes, on_device, t, 0);
}

cgks_status cgks_restore_state(cgks_solver* s, const double* planes, int on_device, double t, long steps)
{
    return set_state_impl(s, planes, on_device, t, steps);
}

cgks_status cgks_get_state(cgks_solver* s, double* planes, int on_device, double* t, long* steps)
{
    if (!s) return fail(CGKS_E_INVAL, "solver is NULL");
    Ctrl c;
    cgks_status st = read_ctrl(s, &c);
    if (st != CGKS_OK) return st;
    if (t) *t = c.t;
    if (steps) *steps = (long)c.steps;
    if (planes) {
        const size_t PL = (size_t)s->nx * s->ny;
        const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        const double* cur = s->host_desc.buf[c.par & 1];
        if (s->prob.dim == 1) {
            CK(launch_compress1d(cur, s->d_stage1d, s->nx, s->stream));
            CK(cudaMemcpyAsync(planes, s->d_stage1d, 6 * PL * sizeof(double), kind, s->stream));
        } else {
            CK(cudaMemcpyAsync(planes, cur, 12 * PL * sizeof(double), kind, s->stream));
        }
        CK(cudaStreamSynchronize(s->stream));
    }
    if (c.status & CGKS_E_NONPHYSICAL) return fail(CGKS_E_NONPHYSICAL, "non-physical state met; last valid state kept");
    return CGKS_OK;
}

static cgks_status enqueue_steps(cgks_solver* s, int nsteps, long* launches)
{
    const int nblocks = stage_blocks(s->ntiles, s->nsm);
    const int cv = s->prob.recon_vars;
    const int rblocks = record_blocks(s->nrchunks, s->nsm, cv);
    const int ublocks = update_blocks(s->ncchunks, s->nsm);
    for (int k = 0; k < nsteps; ++k) {
        CK(launch_begin_step(s->d_desc, 1, s->stream));
        for (int stage = 1; stage <= 2; ++stage) {
            CK(launch_records(stage, cv, s->d_desc, s->d_rchunks, s->nrchunks, rblocks, s->stream));
            CK(launch_stage(s->shape, stage, s->d_desc, s->d_tiles, s->ntiles, nblocks, s->stream));
            CK(launch_update(stage, s->d_desc, s->d_cchunks, s->ncchunks, ublocks, s->stream));
        }
        CK(launch_end_step(s->d_desc, 1, s->stream));
        *launches += 8;
    }
    return CGKS_OK;
}

cgks_status cgks_step(cgks_solver* s, int nsteps, double t_end, double* t_out)
{
    if (!s || nsteps < 0) return fail(CGKS_E_INVAL, "bad arguments");
    g_last_launches = 0;
    long launches = 0;
    CK(launch_set_ctrl(s->d_ctrl, 0.0, t_end > 0.0 ? t_end : 0.0, -1, 0, s->stream));
    launches += 1;
    const int chunk = t_end > 0.0 ? 32 : nsteps;
    int done_steps = 0;
    Ctrl c;
    while (done_steps < nsteps) {
        const int k = (nsteps - done_steps) < chunk ? (nsteps - done_steps) : chunk;
        cgks_status st = enqueue_steps(s, k, &launches);
        if (st != CGKS_OK) return st;
        done_steps += k;
        if (t_end > 0.0 && done_steps < nsteps) {
            st = read_ctrl(s, &c);
            if (st != CGKS_OK) return st;
            if (c.done) break;
        }
    }
    g_last_launches = launches;
    cgks_status st = read_ctrl(s, &c);
    if (st != CGKS_OK) return st;
    if (t_out) *t_out = c.t;
    if (c.status & CGKS_E_NONPHYSICAL) return fail(CGKS_E_NONPHYSICAL, "non-physical state met; last valid state kept");
    return CGKS_OK;
}

}  // extern "C"

// internal (used by the server): stop the solve after `target` steps
cgks_status cgks_set_step_target(cgks_solver* s, long long target)
{
    CK(launch_set_ctrl(s->d_ctrl, 0.0, 0.0, target, 0, s->stream));
    return CGKS_OK;
}

extern "C" {

cgks_status cgks_step_profiled(cgks_solver* s, int nsteps, double stage_ms[8])
{
    if (!s || nsteps <= 0 || !stage_ms) return fail(CGKS_E_INVAL, "bad arguments");
    g_last_launches = 0;
    CK(launch_set_ctrl(s->d_ctrl, 0.0, 0.0, -1, 0, s->stream));
    constexpr int NK = 8;
    std::vector<cudaEvent_t> ev((size_t)nsteps * (NK + 1));
    for (auto& e : ev) CK(cudaEventCreate(&e));
    const int nblocks = stage_blocks(s->ntiles, s->nsm);
    const int cv = s->prob.recon_vars;
    const int rblocks = record_blocks(s->nrchunks, s->nsm, cv);
    const int ublocks = update_blocks(s->ncchunks, s->nsm);
    for (int k = 0; k < nsteps; ++k) {
        cudaEvent_t* e = &ev[(size_t)k * (NK + 1)];
        CK(cudaEventRecord(e[0], s->stream));
        CK(launch_begin_step(s->d_desc, 1, s->stream));
        CK(cudaEventRecord(e[1], s->stream));
        for (int stage = 1; stage <= 2; ++stage) {
            cudaEvent_t* f = e + 1 + 3 * (stage - 1);
            CK(launch_records(stage, cv, s->d_desc, s->d_rchunks, s->nrchunks, rblocks, s->stream));
            CK(cudaEventRecord(f[1], s->stream));
            CK(launch_stage(s->shape, stage, s->d_desc, s->d_tiles, s->ntiles, nblocks, s->stream));
            CK(cudaEventRecord(f[2], s->stream));
            CK(launch_update(stage, s->d_desc, s->d_cchunks, s->ncchunks, ublocks, s->stream));
            CK(cudaEventRecord(f[3], s->stream));
        }
        CK(launch_end_step(s->d_desc, 1, s->stream));
        CK(cudaEventRecord(e[8], s->stream));
    }
    CK(cudaStreamSynchronize(s->stream));
    double acc[NK] = {};
    for (int k = 0; k < nsteps; ++k)
        for (int q = 0; q < NK; ++q) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, ev[(size_t)k * (NK + 1) + q], ev[(size_t)k * (NK + 1) + q + 1]));
            acc[q] += ms;
        }
    for (auto& e : ev) cudaEventDestroy(e);
    for (int q = 0; q < NK; ++q) stage_ms[q] = acc[q] / nsteps;
    g_last_launches = 1 + (long)NK * nsteps;
    Ctrl c;
    cgks_status st = read_ctrl(s, &c);
    if (st != CGKS_OK) return st;
    if (c.status & CGKS_E_NONPHYSICAL) return fail(CGKS_E_NONPHYSICAL, "non-physical state met; last valid state kept");
    return CGKS_OK;
}

// ---------------------------------------------------------------------------
// batched stepping: one persistent launch per stage over the tiles of all
// grids, captured into a CUDA graph per batch composition and replayed.  The
// tile shape of each plan is chosen by timing the candidate shapes on its first
// steps (the shape changes only the work decomposition, never the arithmetic of
// a face or a cell, so results are identical whichever shape runs).
}  // extern "C"

namespace {
std::mutex g_batch_mu;
std::map<std::vector<cgks_solver*>, cgks::BatchPlan*> g_batch_plans;
}  // namespace

namespace cgks {

void destroy_plan(BatchPlan* bp)
{
    if (!bp) return;
    for (int k = 0; k < TILE_COUNT; ++k) {
        if (bp->exec[k]) cudaGraphExecDestroy(bp->exec[k]);
        cudaFree(bp->d_tiles[k]);
    }
    for (int c = 0; c < 2; ++c) cudaFree(bp->d_rchunks[c]);
    cudaFree(bp->d_cchunks);
    cudaFree(bp->d_grids);
    delete bp;
}

static cudaError_t capture_graph(BatchPlan* bp, int shape)
{
    const int n = (int)bp->solvers.size();
    const int nblocks = stage_blocks(bp->ntiles[shape], bp->nsm);
    // first calls configure the kernels' attributes outside the capture
    cudaError_t e = launch_stage(shape, 1, bp->d_grids, bp->d_tiles[shape], 0, 1, bp->stream);
    if (e == cudaSuccess) e = launch_stage(shape, 2, bp->d_grids, bp->d_tiles[shape], 0, 1, bp->stream);
    if (e != cudaSuccess) return e;
    auto records = [&](int stage, cudaStream_t st) {
        cudaError_t r = cudaSuccess;
        for (int c = 0; c < 2 && r == cudaSuccess; ++c)
            r = launch_records(stage, c, bp->d_grids, bp->d_rchunks[c], bp->nrchunks[c],
                               record_blocks(bp->nrchunks[c], bp->nsm, c), st);
        return r;
    };
    cudaStream_t cap;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaGraph_t graph;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e1 = launch_begin_step(bp->d_grids, n, cap);
        for (int stage = 1; stage <= 2; ++stage) {
            if (e1 == cudaSuccess) e1 = records(stage, cap);
            if (e1 == cudaSuccess)
                e1 = launch_stage(shape, stage, bp->d_grids, bp->d_tiles[shape], bp->ntiles[shape], nblocks, cap);
            if (e1 == cudaSuccess)
                e1 = launch_update(stage, bp->d_grids, bp->d_cchunks, bp->ncchunks, update_blocks(bp->ncchunks, bp->nsm),
                                   cap);
        }
        if (e1 == cudaSuccess) e1 = launch_end_step(bp->d_grids, n, cap);
        e = cudaStreamEndCapture(cap, &graph);
        if (e1 != cudaSuccess) e = e1;
    }
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(&bp->exec[shape], graph, 0);
    cudaGraphDestroy(graph);
    return e;
}

cudaError_t make_plan(cgks_solver* const* solvers, int n, cudaStream_t stream, int forced_shape, BatchPlan** out)
{
    BatchPlan* bp = new BatchPlan();
    bp->solvers.assign(solvers, solvers + n);
    bp->stream = stream;
    bp->nsm = solvers[0]->nsm;
    bp->dim = solvers[0]->prob.dim;
    std::vector<GridDev> descs;
    for (int g = 0; g < n; ++g) descs.push_back(solvers[g]->host_desc);
    cudaError_t e = cudaMalloc(&bp->d_grids, descs.size() * sizeof(GridDev));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(bp->d_grids, descs.data(), descs.size() * sizeof(GridDev), cudaMemcpyHostToDevice, stream);
    long long cells = 0;
    for (int g = 0; g < n; ++g) cells += (long long)solvers[g]->nx * solvers[g]->ny;
    bp->cells = cells;
    // update-kernel queue of all grids
    {
        std::vector<TileRef> q;
        for (int g = 0; g < n; ++g) {
            std::vector<TileRef> r = cell_chunks(solvers[g]->nx, solvers[g]->ny, g);
            q.insert(q.end(), r.begin(), r.end());
        }
        bp->ncchunks = (int)q.size();
        bp->launches_per_step += 2;
        if (e == cudaSuccess) e = cudaMalloc(&bp->d_cchunks, q.size() * sizeof(TileRef));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(bp->d_cchunks, q.data(), q.size() * sizeof(TileRef), cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    }
    // record-kernel queues of the conservative and the characteristic grids
    for (int c = 0; c < 2; ++c) {
        std::vector<TileRef> q;
        for (int g = 0; g < n; ++g) {
            const cgks_problem& p = solvers[g]->prob;
            if (p.recon_vars != c) continue;
            std::vector<TileRef> r = record_chunks(solvers[g]->nx, solvers[g]->ny, p.dim, p.recon_vars, g);
            q.insert(q.end(), r.begin(), r.end());
        }
        bp->nrchunks[c] = (int)q.size();
        if (q.empty()) continue;
        bp->launches_per_step += 2;
        if (e == cudaSuccess) e = cudaMalloc(&bp->d_rchunks[c], q.size() * sizeof(TileRef));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(bp->d_rchunks[c], q.data(), q.size() * sizeof(TileRef), cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    }
    if (bp->dim == 1) { bp->candidates = {TILE_64x1}; }
    else if (forced_shape >= 0) { bp->candidates = {forced_shape}; }
    else { bp->candidates = {TILE_14x8, TILE_16x8, TILE_16x7, TILE_16x16}; }
    for (int shape : bp->candidates) {
        std::vector<TileRef> tiles;
        for (int g = 0; g < n; ++g) {
            const int tw = tile_w(shape), th = tile_h(shape);
            for (int y0 = 0; y0 < solvers[g]->ny; y0 += th)
                for (int x0 = 0; x0 < solvers[g]->nx; x0 += tw) tiles.push_back(TileRef{g, x0, y0, 0});
        }
        bp->ntiles[shape] = (int)tiles.size();
        if (e == cudaSuccess) e = cudaMalloc(&bp->d_tiles[shape], tiles.size() * sizeof(TileRef));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(bp->d_tiles[shape], tiles.data(), tiles.size() * sizeof(TileRef), cudaMemcpyHostToDevice,
                                stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e == cudaSuccess) e = capture_graph(bp, shape);
    }
    if (e != cudaSuccess) { destroy_plan(bp); return e; }
    bp->chosen = bp->candidates.size() == 1 ? bp->candidates[0] : -1;
    *out = bp;
    return cudaSuccess;
}

// run nsteps steps of the plan; while the shape is not yet chosen, each
// candidate runs timed steps and the fastest is kept
cudaError_t run_plan(BatchPlan* bp, int nsteps, long* launches)
{
    cudaError_t e = cudaSuccess;
    int k = 0;
    while (bp->chosen < 0 && k < nsteps) {
        const int shape = bp->candidates[bp->trial_idx];
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, bp->stream);
        e = cudaGraphLaunch(bp->exec[shape], bp->stream);
        cudaEventRecord(b, bp->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        if (e != cudaSuccess) return e;
        *launches += bp->launches_per_step;
        ++k;
        if (bp->trial_count[shape] > 0) bp->trial_ms[shape] += ms;   // the first run of a shape is a warm-up
        bp->trial_count[shape] += 1;
        if (bp->trial_count[shape] >= 2) {
            bp->trial_idx += 1;
            if (bp->trial_idx >= (int)bp->candidates.size()) {
                int best = bp->candidates[0];
                for (int s2 : bp->candidates)
                    if (bp->trial_ms[s2] < bp->trial_ms[best]) best = s2;
                bp->chosen = best;
            }
        }
    }
    for (; k < nsteps; ++k) {
        e = cudaGraphLaunch(bp->exec[bp->chosen], bp->stream);
        if (e != cudaSuccess) return e;
        *launches += bp->launches_per_step;
    }
    return cudaSuccess;
}

}  // namespace cgks

extern "C" {

void cgks_forget_solver_plans(cgks_solver* s)
{
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (auto it = g_batch_plans.begin(); it != g_batch_plans.end();) {
        bool has = false;
        for (cgks_solver* x : it->first) has |= (x == s);
        if (has) { cgks::destroy_plan(it->second); it = g_batch_plans.erase(it); }
        else ++it;
    }
}

cgks_status cgks_batch_step(cgks_solver* const* solvers, int n, int nsteps)
{
    if (!solvers || n <= 0 || nsteps < 0) return fail(CGKS_E_INVAL, "bad arguments");
    for (int g = 0; g < n; ++g) {
        if (!solvers[g]) return fail(CGKS_E_INVAL, "NULL solver in batch");
        if (solvers[g]->prob.dim != solvers[0]->prob.dim) return fail(CGKS_E_INVAL, "mixed dims in one batch");
    }
    std::lock_guard<std::mutex> lk(g_batch_mu);
    g_last_launches = 0;
    std::vector<cgks_solver*> key(solvers, solvers + n);
    BatchPlan* bp = nullptr;
    auto it = g_batch_plans.find(key);
    if (it != g_batch_plans.end()) bp = it->second;
    else {
        cudaError_t e = make_plan(solvers, n, solvers[0]->stream, -1, &bp);
        if (e != cudaSuccess) return cuda_fail(e, "batch plan");
        g_batch_plans[key] = bp;
    }
    long launches = 0;
    CK(launch_batch_resume(bp->d_grids, n, bp->stream));
    launches += 1;
    CK(run_plan(bp, nsteps, &launches));
    CK(cudaStreamSynchronize(bp->stream));
    g_last_launches = launches;
    return CGKS_OK;
}

int cgks_batch_tile_shape(cgks_solver* const* solvers, int n)
{
    std::lock_guard<std::mutex> lk(g_batch_mu);
    std::vector<cgks_solver*> key(solvers, solvers + n);
    auto it = g_batch_plans.find(key);
    if (it == g_batch_plans.end()) return -1;
    return it->second->chosen;
}

}  // extern "C"
