// cgks_noalloc.cu -- cgks_step_noalloc: the plain 2D step without any device
// allocation, for callers that cannot call cudaMalloc.
//
// Such callers exist when the library runs inside code that owns the device
// memory itself: a host application with a fixed memory pool or a custom
// allocator, or an embedding with a fixed device footprint where the allocator
// must not be re-entered.  They pass the state planes they already own;
// everything else the step needs (the second state buffer, the intermediate
// state W*, the control block, the descriptor and the tile queue) lives in
// file-scope device arrays of fixed size that every GPU loading this library
// keeps until the process exits.  The call reads the control block back and
// synchronises its stream before it returns, so it must not be called while a
// stream capture is active on that stream.
#include "cgks_internal.h"
#include "../../include/cgks.h"

#include <cuda_runtime.h>
#include <string.h>

#include <mutex>
#include <string>
#include <vector>

namespace {

constexpr size_t kMaxCells = CGKS_NOALLOC_MAX_CELLS;
constexpr int kMaxTiles = CGKS_NOALLOC_MAX_TILES;
constexpr int kMaxSide = CGKS_NOALLOC_MAX_SIDE;
// face-row records of the largest admissible grid: 2 nx ny + 5 (nx + ny) + 8
// rows is largest for nx ny = kMaxCells with one side at kMaxSide
constexpr size_t kMaxRecordRows = 2 * kMaxCells + 5 * ((size_t)kMaxSide + kMaxCells / kMaxSide) + 8;
constexpr int kMaxChunks = (int)((4 * kMaxRecordRows + 255) / 256);
// face results: 16 per face, (nx+1) ny + nx (ny+1) faces
constexpr size_t kMaxFaces = 2 * kMaxCells + (size_t)kMaxSide + kMaxCells / kMaxSide;
constexpr int kMaxCellChunks = (int)((kMaxCells + 255) / 256);

// scratch: buffer for the other state (ping-pong) and for W*, 12 planes each
static __device__ __align__(256) double g_scratch[2 * 12 * kMaxCells];
static __device__ __align__(256) cgks::Ctrl g_ctrl;
static __device__ __align__(256) cgks::GridDev g_desc;
static __device__ __align__(256) cgks::TileRef g_tiles[kMaxTiles];
static __device__ __align__(256) double g_records[28 * kMaxRecordRows];
static __device__ __align__(256) cgks::TileRef g_rchunks[kMaxChunks];
static __device__ __align__(256) double g_faces[16 * kMaxFaces];
static __device__ __align__(256) cgks::TileRef g_cchunks[kMaxCellChunks];

// device addresses of the arrays above, looked up once per device with that
// device current (host code must not use the symbols' names as addresses)
struct DeviceSymbols {
    bool ready = false;
    double* scratch = nullptr;
    cgks::Ctrl* ctrl = nullptr;
    cgks::GridDev* desc = nullptr;
    cgks::TileRef* tiles = nullptr;
    double* records = nullptr;
    cgks::TileRef* rchunks = nullptr;
    double* faces = nullptr;
    cgks::TileRef* cchunks = nullptr;
};
DeviceSymbols g_syms[cgks::kMaxDevices];
std::mutex g_mu;
thread_local std::string g_err;

cgks_status nfail(cgks_status st, const std::string& m)
{
    g_err = m;
    return st;
}

cgks_status setup_device(int dev, DeviceSymbols** out)
{
    if (dev < 0 || dev >= cgks::kMaxDevices) return nfail(CGKS_E_INVAL, "device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceSymbols& s = g_syms[dev];
    if (!s.ready) {
        cudaError_t e = cudaGetSymbolAddress((void**)&s.scratch, g_scratch);
        if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&s.ctrl, g_ctrl);
        if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&s.desc, g_desc);
        if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&s.tiles, g_tiles);
        if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&s.records, g_records);
        if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&s.rchunks, g_rchunks);
        if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&s.faces, g_faces);
        if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&s.cchunks, g_cchunks);
        if (e != cudaSuccess) return nfail(CGKS_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        s.ready = true;
    }
    *out = &s;
    return CGKS_OK;
}

// fills the descriptor, the tile queue and the record-kernel queue of this call
// (kernel arguments carry the values, so no host buffer has to outlive the call)
__global__ void noalloc_init_kernel(cgks::GridDev G, int tw, int th, int nchunks, int ncchunks)
{
    const int ntx = (G.nx + tw - 1) / tw, nty = (G.ny + th - 1) / th;
    if (blockIdx.x == 0 && threadIdx.x == 0) g_desc = G;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntx * nty; t += gridDim.x * blockDim.x)
        g_tiles[t] = cgks::TileRef{0, (t % ntx) * tw, (t / ntx) * th, 0};
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nchunks; c += gridDim.x * blockDim.x)
        g_rchunks[c] = cgks::TileRef{0, 256 * c, 0, 0};
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncchunks; c += gridDim.x * blockDim.x)
        g_cchunks[c] = cgks::TileRef{0, 256 * c, 0, 0};
}

#define NCK(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return nfail(CGKS_E_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

}  // namespace

extern "C" {

const char* cgks_noalloc_last_error(void) { return g_err.c_str(); }

cgks_status cgks_step_noalloc(const cgks_problem* prob, double* planes, int nsteps, double* t_inout,
                              void* cuda_stream)
{
    using namespace cgks;
    if (!prob || !planes || !t_inout || nsteps < 0) return nfail(CGKS_E_INVAL, "NULL argument or nsteps < 0");
    if (prob->dim != 2) return nfail(CGKS_E_INVAL, "cgks_step_noalloc takes 2D problems");
    if (prob->nx < 1 || prob->ny < 1) return nfail(CGKS_E_INVAL, "nx and ny must be >= 1");
    const size_t cells = (size_t)prob->nx * prob->ny;
    if (cells > kMaxCells) return nfail(CGKS_E_INVAL, "grid exceeds CGKS_NOALLOC_MAX_CELLS");
    if (prob->nx > kMaxSide || prob->ny > kMaxSide) return nfail(CGKS_E_INVAL, "a side exceeds CGKS_NOALLOC_MAX_SIDE");
    if (!(prob->x1 > prob->x0) || !(prob->y1 > prob->y0) || !(prob->gamma > 1.0) || !(prob->gamma < 3.0) ||
        !(prob->cfl > 0.0) || !(prob->eps_tau >= 0.0) || !(prob->c_tau >= 0.0) || !(prob->weno_eps > 0.0) || !(prob->mu >= 0.0))
        return nfail(CGKS_E_INVAL, "bad problem parameters");
    if (prob->recon_vars != 0 && prob->recon_vars != 1) return nfail(CGKS_E_INVAL, "recon_vars must be 0 or 1");
    if (prob->order != 0 && prob->order != 6 && prob->order != 8) return nfail(CGKS_E_INVAL, "order must be 0, 6 or 8");
    for (int k = 0; k < 4; ++k) {
        if (prob->bc[k] < CGKS_BC_PERIODIC || prob->bc[k] > CGKS_BC_OUTFLOW) return nfail(CGKS_E_INVAL, "unknown bc");
        const int n = k < 2 ? prob->nx : prob->ny;
        if (prob->bc[k] == CGKS_BC_REFLECT && n < 2) return nfail(CGKS_E_INVAL, "a reflecting side needs >= 2 cells");
    }
    const int shape = TILE_16x8;
    const int tw = tile_w(shape), th = tile_h(shape);
    const long long ntiles = (long long)((prob->nx + tw - 1) / tw) * ((prob->ny + th - 1) / th);
    if (ntiles > kMaxTiles) return nfail(CGKS_E_INVAL, "grid needs more tiles than CGKS_NOALLOC_MAX_TILES");

    int dev = 0, nsm = 1;
    NCK(cudaGetDevice(&dev));
    NCK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    DeviceSymbols* sym = nullptr;
    cgks_status st = setup_device(dev, &sym);
    if (st != CGKS_OK) return st;
    cudaStream_t stream = (cudaStream_t)cuda_stream;

    // descriptor: the caller's planes are state buffer 0, the scratch array
    // holds state buffer 1 and W*
    GridDev G;
    memset(&G, 0, sizeof(G));
    G.buf[0] = planes;
    G.buf[1] = sym->scratch;
    G.ws = sym->scratch + 12 * cells;
    G.ctrl = sym->ctrl;
    G.recx = sym->records;
    G.recy = sym->records + (size_t)28 * (prob->nx + 1) * (prob->ny + 4);
    G.facex = sym->faces;
    G.facey = sym->faces + (size_t)16 * (prob->nx + 1) * prob->ny;
    G.nx = prob->nx;
    G.ny = prob->ny;
    G.dim = 2;
    for (int k = 0; k < 4; ++k) G.bc[k] = prob->bc[k];
    G.dx = (prob->x1 - prob->x0) / prob->nx;
    G.dy = (prob->y1 - prob->y0) / prob->ny;
    G.inv_dx = 1.0 / G.dx;
    G.inv_dy = 1.0 / G.dy;
    G.gamma = prob->gamma;
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
        const double r = q[0], u = q[1], v = q[2], p = q[3];
        G.inflow[side][0] = r;
        G.inflow[side][1] = r * u;
        G.inflow[side][2] = r * v;
        G.inflow[side][3] = p / (prob->gamma - 1.0) + 0.5 * r * (u * u + v * v);
    }
    const int nt = (int)ntiles;
    const int cv = prob->recon_vars;
    const long long items = (long long)(cv ? 1 : 4) * record_rows(prob->nx, prob->ny, 2);
    const int nrc = (int)((items + 255) / 256);
    const int ncc = (int)((cells + 255) / 256);
    const int work = nt > nrc ? nt : nrc;
    noalloc_init_kernel<<<(work + 255) / 256, 256, 0, stream>>>(G, tw, th, nrc, ncc);
    NCK(cudaGetLastError());
    // control block starts from t, step 0, no error, state in the caller's buffer
    NCK(launch_set_ctrl(sym->ctrl, *t_inout, 0.0, -1, 1, stream));
    NCK(launch_cfl(sym->desc, 0, G, stream));
    const int nblocks = stage_blocks(nt, nsm);
    const int rblocks = record_blocks(nrc, nsm, cv);
    const int ublocks = update_blocks(ncc, nsm);
    for (int k = 0; k < nsteps; ++k) {
        NCK(launch_begin_step(sym->desc, 1, stream));
        for (int stage = 1; stage <= 2; ++stage) {
            NCK(launch_records(stage, cv, sym->desc, sym->rchunks, nrc, rblocks, stream));
            NCK(launch_stage(shape, stage, sym->desc, sym->tiles, nt, nblocks, stream));
            NCK(launch_update(stage, sym->desc, sym->cchunks, ncc, ublocks, stream));
        }
        NCK(launch_end_step(sym->desc, 1, stream));
    }
    Ctrl c;
    NCK(cudaMemcpyAsync(&c, sym->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, stream));
    NCK(cudaStreamSynchronize(stream));
    // the newest valid state is in buffer c.par; bring it to the caller's planes
    if (c.par & 1) {
        NCK(cudaMemcpyAsync(planes, sym->scratch, 12 * cells * sizeof(double), cudaMemcpyDeviceToDevice, stream));
        NCK(cudaStreamSynchronize(stream));
    }
    *t_inout = c.t;
    if (c.status & kStatusBounds)
        return nfail(CGKS_E_CUDA, "a kernel index left its buffer (bounds-checked build)");
    if (c.status & CGKS_E_NONPHYSICAL)
        return nfail(CGKS_E_NONPHYSICAL, "non-physical state met; the planes hold the last valid state");
    return CGKS_OK;
}

}  // extern "C"
