// cgks_api.cu -- host runtime behind the C ABI of include/cgks.h: solver
// objects (device planes, control block, tile queue), state transfer and the
// plain step loop (the batched step is in cgks_batch.cu, serving in
// cgks_serve.cu).
#include "cgks_internal.h"
#include "../../include/cgks.h"

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

using namespace cgks;

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

// The flux kernel's tile shape for a grid: 64x1 in 1D; in 2D 8x16 (two face segments per thread of
// the 128-thread CTA) or 14x8 (1.75), whichever needs less time over the passes of the persistent
// grid (two CTAs per SM): on 2048^2, where partial passes do not matter, a pass of 14x8 tiles takes
// 0.883 of a pass of 8x16 tiles (27.67 ms for 107.8 passes against 28.05 ms for 123.8), so 8x16
// wins on large grids and 14x8 where it needs no more passes than 8x16 (256^2: 2 passes each).
int pick_shape(const cgks_problem& p, int nsm)
{
    if (p.dim == 1) return TILE_64x1;
    const long long cap = 2LL * (nsm > 0 ? nsm : 1);
    auto passes = [&](int tx, int ty) {
        const long long tiles = (long long)((p.nx + tx - 1) / tx) * ((p.ny + ty - 1) / ty);
        return (double)((tiles + cap - 1) / cap);
    };
    return 0.883 * passes(14, 8) < passes(8, 16) ? TILE_14x8 : TILE_8x16;
}

}  // namespace

namespace cgks {

void fill_grid_desc(const cgks_problem& p, double* planes, double* records, double* faces, Ctrl* ctrl, GridDev& G)
{
    const int nx = p.nx, ny = p.dim == 1 ? 1 : p.ny;
    const size_t PL = (size_t)nx * ny;
    memset(&G, 0, sizeof(G));
    G.buf[0] = planes;
    G.buf[1] = planes + 12 * PL;
    G.ws = planes + 24 * PL;
    G.ctrl = ctrl;
    G.recx = records;
    G.recy = p.dim == 2 ? records + (size_t)28 * (nx + 1) * (ny + 4) : nullptr;
    G.facex = faces;
    G.facey = p.dim == 2 ? faces + (size_t)16 * (nx + 1) * ny : nullptr;
    G.nx = nx;
    G.ny = ny;
    G.dim = p.dim;
    for (int k = 0; k < 4; ++k) G.bc[k] = (p.dim == 1 && k >= 2) ? CGKS_BC_PERIODIC : p.bc[k];
    G.dx = (p.x1 - p.x0) / nx;
    G.dy = p.dim == 1 ? 1.0 : (p.y1 - p.y0) / ny;
    G.inv_dx = 1.0 / G.dx;
    G.inv_dy = 1.0 / G.dy;
    G.gamma = p.gamma;
    // internal degrees of freedom of the 2D Maxwellian; a 1D problem runs as a
    // y-uniform 2D one, whose extra velocity direction plays the role of the
    // additional internal degree of freedom of the 1D model
    G.K = (4.0 - 2.0 * p.gamma) / (p.gamma - 1.0);
    G.cfl = p.cfl;
    G.eps_tau = p.eps_tau;
    G.c_tau = p.c_tau;
    G.weno_eps = p.weno_eps;
    G.mu = p.mu;
    G.recon_vars = p.recon_vars;
    G.order = p.order == 6 ? 6 : 8;
    for (int side = 0; side < 4; ++side) {
        const double* q = p.inflow[side];
        const double r = q[0], u = q[1], v = p.dim == 1 ? 0.0 : q[2], pr = q[3];
        G.inflow[side][0] = r;
        G.inflow[side][1] = r * u;
        G.inflow[side][2] = r * v;
        G.inflow[side][3] = pr / (p.gamma - 1.0) + 0.5 * r * (u * u + v * v);
    }
}

size_t grid_device_bytes(const cgks_problem& p)
{
    const int ny = p.dim == 1 ? 1 : p.ny;
    return (size_t)3 * 12 * p.nx * ny * sizeof(double)
           + (record_doubles(p.nx, ny, p.dim) + face_doubles(p.nx, ny, p.dim)) * sizeof(double);
}

cgks_status validate_problem(const cgks_problem* p) { return validate(p); }

}  // namespace cgks

extern "C" {

void cgks_set_batch_error(const char* m) { g_last_error = m; }
void cgks_set_launch_count(long n) { g_last_launches = n; }

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
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, s->device);
    s->shape = pick_shape(*prob, s->nsm);
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
    fill_grid_desc(*prob, s->d_planes, s->d_records, s->d_faces, s->d_ctrl, G);
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
    if (shape < 0) shape = pick_shape(s->prob, s->nsm);
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

int cgks_tile_shape(const cgks_solver* s)
{
    return s ? s->shape : -1;
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
    cudaFree(s->d_ftiles);
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
    if (c.status & kStatusBounds) return fail(CGKS_E_CUDA, "a kernel index left its buffer (bounds-checked build)");
    if (c.status & CGKS_E_NONPHYSICAL) return fail(CGKS_E_NONPHYSICAL, "non-physical state met; last valid state kept");
    return CGKS_OK;
}

static cgks_status enqueue_steps(cgks_solver* s, int nsteps, long* launches, bool fused)
{
    const int nblocks = stage_blocks(s->ntiles, s->nsm);
    const int cv = s->prob.recon_vars;
    const int rblocks = record_blocks(s->nrchunks, s->nsm, cv);
    const int ublocks = update_blocks(s->ncchunks, s->nsm, 4);
    const int fblocks = s->nftiles < s->nsm ? s->nftiles : s->nsm;
    for (int k = 0; k < nsteps; ++k) {
        CK(launch_begin_step(s->d_desc, 1, s->stream));
        if (fused) {
            CK(launch_fused_step(s->d_desc, s->d_ftiles, s->nftiles, fblocks, s->stream));
            CK(launch_end_step(s->d_desc, 1, s->stream));
            *launches += 3;
            continue;
        }
        for (int stage = 1; stage <= 2; ++stage) {
            CK(launch_records(stage, cv, s->d_desc, s->d_rchunks, s->nrchunks, rblocks, s->stream));
            CK(launch_stage(s->shape, stage, s->d_desc, s->d_tiles, s->ntiles, nblocks, s->stream));
            CK(launch_update(stage, s->d_desc, s->d_cchunks, s->ncchunks, ublocks, s->stream, nullptr, 4));
        }
        CK(launch_end_step(s->d_desc, 1, s->stream));
        *launches += 8;
    }
    return CGKS_OK;
}

// NVTX range around a call (visible to profilers that record NVTX; no cost otherwise)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

static cgks_status step_impl(cgks_solver* s, int nsteps, double t_end, double* t_out, bool fused)
{
    if (!s || nsteps < 0) return fail(CGKS_E_INVAL, "bad arguments");
    if (fused && s->prob.dim != 2) return fail(CGKS_E_INVAL, "the fused step is 2D only");
    if (fused && !s->d_ftiles) {
        const std::vector<TileRef> tiles = make_tiles(s->nx, s->ny, TILE_16x8, 0);
        TileRef* d = nullptr;
        CK(cudaMalloc(&d, tiles.size() * sizeof(TileRef)));
        cudaError_t e = cudaMemcpyAsync(d, tiles.data(), tiles.size() * sizeof(TileRef), cudaMemcpyHostToDevice,
                                        s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) { cudaFree(d); return cuda_fail(e, "cgks_step_fused"); }
        s->d_ftiles = d;
        s->nftiles = (int)tiles.size();
    }
    NvtxRange range(fused ? "cgks_step_fused" : "cgks_step");
    g_last_launches = 0;
    long launches = 0;
    CK(launch_set_ctrl(s->d_ctrl, 0.0, t_end > 0.0 ? t_end : 0.0, -1, 0, s->stream));
    launches += 1;
    const int chunk = t_end > 0.0 ? 32 : nsteps;
    int done_steps = 0;
    Ctrl c;
    while (done_steps < nsteps) {
        const int k = (nsteps - done_steps) < chunk ? (nsteps - done_steps) : chunk;
        cgks_status st = enqueue_steps(s, k, &launches, fused);
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
    if (c.status & kStatusBounds) return fail(CGKS_E_CUDA, "a kernel index left its buffer (bounds-checked build)");
    if (c.status & CGKS_E_NONPHYSICAL) return fail(CGKS_E_NONPHYSICAL, "non-physical state met; last valid state kept");
    return CGKS_OK;
}

cgks_status cgks_step(cgks_solver* s, int nsteps, double t_end, double* t_out)
{
    return step_impl(s, nsteps, t_end, t_out, false);
}

cgks_status cgks_step_fused(cgks_solver* s, int nsteps, double t_end, double* t_out)
{
    return step_impl(s, nsteps, t_end, t_out, true);
}

}  // extern "C"

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
    const int ublocks = update_blocks(s->ncchunks, s->nsm, 4);
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
            CK(launch_update(stage, s->d_desc, s->d_cchunks, s->ncchunks, ublocks, s->stream, nullptr, 4));
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
    if (c.status & kStatusBounds) return fail(CGKS_E_CUDA, "a kernel index left its buffer (bounds-checked build)");
    if (c.status & CGKS_E_NONPHYSICAL) return fail(CGKS_E_NONPHYSICAL, "non-physical state met; last valid state kept");
    return CGKS_OK;
}

}  // extern "C"
