// cgks_batch.cu -- the batched engine (cgks_internal.h: BatchEngine) and the
// cgks_batch_step entry point of include/cgks.h built on it.
//
// Many grids of uneven size advance together: every kernel of a step is one
// persistent launch over a flattened work queue of all grids (tiles for the
// flux kernel, chunks of face rows for the record kernel, chunks of cells for
// the update kernel), each grid with its own dt and step control in its Ctrl.
// The step is captured once per candidate as a CUDA graph whose kernels read
// the queue lengths from device memory, so the queues can be rewritten between
// replays without a new capture.
#include "cgks_internal.h"
#include "../../include/cgks.h"

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <string.h>

#include <algorithm>
#include <list>
#include <map>
#include <mutex>
#include <string>
#include <vector>

namespace cgks {

namespace {

__global__ void snapshot_kernel(const GridDev* grids, int n, Ctrl* dst)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < n) dst[g] = *grids[g].ctrl;
}

__global__ void dummy_ctrl_kernel(Ctrl* c)
{
    memset(c, 0, sizeof(Ctrl));
    c->done = 1;
    c->steps_target = 0;
}

constexpr int kShapeCands[] = {TILE_8x16, TILE_14x8, TILE_16x8, TILE_16x16};
constexpr int kCptCands[] = {2, 4};

}  // namespace

cudaError_t BatchEngine::create(int nslots, int dim, cudaStream_t stream, int forced_shape, BatchEngine** out)
{
    *out = nullptr;
    BatchEngine* E = new BatchEngine();
    E->nslots_ = nslots;
    E->dim_ = dim;
    E->stream_ = stream;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&E->nsm_, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaMalloc(&E->d_grids_, (size_t)nslots * sizeof(GridDev));
    if (e == cudaSuccess) e = cudaMalloc(&E->d_dummy_, sizeof(Ctrl));
    if (e == cudaSuccess) e = cudaMalloc(&E->d_counts_, kQ * sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(E->d_counts_, 0, kQ * sizeof(int), stream);
    if (e == cudaSuccess) {
        dummy_ctrl_kernel<<<1, 1, 0, stream>>>(E->d_dummy_);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&E->stage_done_, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(E->stage_done_, stream);
    // candidates: shapes first (update kernel at 1 cell per thread), then cells
    // per thread with the shape the first phase picks (filled in then)
    if (dim == 1) E->cands_.push_back({TILE_64x1, 1});
    else if (forced_shape >= 0) E->cands_.push_back({forced_shape, 1});
    else for (int s : kShapeCands) E->cands_.push_back({s, 1});
    for (int c : kCptCands) E->cands_.push_back({-1, c});
    E->exec_.assign(E->cands_.size(), nullptr);
    E->trial_.assign(E->cands_.size(), -1.0);
    if (e == cudaSuccess) {
        // every slot starts empty
        std::vector<std::pair<int, GridDev>> none;
        e = E->set_members(none);
    }
    if (e != cudaSuccess) {
        delete E;
        return e;
    }
    *out = E;
    return cudaSuccess;
}

BatchEngine::~BatchEngine()
{
    if (stage_done_) cudaEventSynchronize(stage_done_);
    for (cudaGraphExec_t g : exec_)
        if (g) cudaGraphExecDestroy(g);
    for (int k = 0; k < kQ; ++k) cudaFree(d_q_[k]);
    cudaFree(d_counts_);
    cudaFree(d_dummy_);
    cudaFree(d_grids_);
    if (h_stage_) cudaFreeHost(h_stage_);
    if (stage_done_) cudaEventDestroy(stage_done_);
}

// grow queue k to hold n entries; the graphs bake the queue addresses, so a
// reallocation drops them (they are captured again before the next replay)
cudaError_t BatchEngine::ensure_capacity(int k, size_t n)
{
    if (n <= cap_[k] && d_q_[k]) return cudaSuccess;
    const size_t cap = std::max<size_t>(1024, n + n / 2);
    cudaError_t e = cudaStreamSynchronize(stream_);
    if (e != cudaSuccess) return e;
    cudaFree(d_q_[k]);
    d_q_[k] = nullptr;
    cap_[k] = 0;
    e = cudaMalloc(&d_q_[k], cap * sizeof(TileRef));
    if (e != cudaSuccess) return e;
    cap_[k] = cap;
    for (auto& g : exec_)
        if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    return cudaSuccess;
}

cudaError_t BatchEngine::set_members(const std::vector<std::pair<int, GridDev>>& members)
{
    // descriptor table: members in their slots, a done control block elsewhere
    std::vector<GridDev> table((size_t)nslots_);
    for (auto& G : table) {
        memset(&G, 0, sizeof(G));
        G.ctrl = d_dummy_;
    }
    std::vector<TileRef> q[kQ];
    cells_ = 0;
    // the tile shapes whose queues the next replays may need
    std::vector<int> shapes;
    if (chosen_ >= 0) shapes.push_back(cands_[chosen_].shape);
    else
        for (const BatchCand& c : cands_)
            if (c.shape >= 0 && std::find(shapes.begin(), shapes.end(), c.shape) == shapes.end()) shapes.push_back(c.shape);
    for (const auto& m : members) {
        const int slot = m.first;
        const GridDev& G = m.second;
        table[slot] = G;
        cells_ += (long long)G.nx * G.ny;
        for (int s : shapes) {
            const int tw = tile_w(s), th = tile_h(s);
            for (int y0 = 0; y0 < G.ny; y0 += th)
                for (int x0 = 0; x0 < G.nx; x0 += tw) q[s].push_back(TileRef{slot, x0, y0, 0});
        }
        std::vector<TileRef> r = record_chunks(G.nx, G.ny, G.dim, G.recon_vars, slot);
        q[TILE_COUNT + G.recon_vars].insert(q[TILE_COUNT + G.recon_vars].end(), r.begin(), r.end());
        std::vector<TileRef> c = cell_chunks(G.nx, G.ny, slot);
        q[TILE_COUNT + 2].insert(q[TILE_COUNT + 2].end(), c.begin(), c.end());
    }
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < kQ && e == cudaSuccess; ++k)
        if (!q[k].empty() || k >= TILE_COUNT || std::find(shapes.begin(), shapes.end(), k) != shapes.end())
            e = ensure_capacity(k, q[k].size());
    if (e != cudaSuccess) return e;
    int counts[kQ];
    size_t bytes = table.size() * sizeof(GridDev) + sizeof(counts);
    for (int k = 0; k < kQ; ++k) {
        counts[k] = (int)q[k].size();
        bytes += q[k].size() * sizeof(TileRef);
    }
    // the staging buffer is free once its previous upload has run
    e = cudaEventSynchronize(stage_done_);
    if (e != cudaSuccess) return e;
    if (bytes > stage_cap_) {
        if (h_stage_) cudaFreeHost(h_stage_);
        h_stage_ = nullptr;
        stage_cap_ = 0;
        const size_t cap = std::max<size_t>(1 << 20, bytes + bytes / 2);
        e = cudaHostAlloc(&h_stage_, cap, cudaHostAllocDefault);
        if (e != cudaSuccess) return e;
        stage_cap_ = cap;
    }
    char* p = h_stage_;
    auto put = [&](void* dst, const void* src, size_t n) {
        if (n == 0) return;
        memcpy(p, src, n);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, p, n, cudaMemcpyHostToDevice, stream_);
        p += n;
    };
    put(d_grids_, table.data(), table.size() * sizeof(GridDev));
    for (int k = 0; k < kQ; ++k)
        if (d_q_[k]) put(d_q_[k], q[k].data(), q[k].size() * sizeof(TileRef));
    put(d_counts_, counts, sizeof(counts));
    if (e == cudaSuccess) e = cudaEventRecord(stage_done_, stream_);
    // per step: begin + end, and per stage two record launches (conservative and
    // characteristic grids), flux, update
    launches_per_step_ = 2 + 2 * 4;
    return e;
}

cudaError_t BatchEngine::capture(int cand)
{
    const BatchCand c = cands_[cand];
    // the kernels' attributes are set outside the capture
    cudaError_t e = launch_stage(c.shape, 1, d_grids_, d_q_[c.shape], 0, 0, stream_);
    if (e == cudaSuccess) e = launch_stage(c.shape, 2, d_grids_, d_q_[c.shape], 0, 0, stream_);
    if (e != cudaSuccess) return e;
    cudaStream_t cap;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const int* cnt = d_counts_;
        cudaError_t e1 = launch_begin_step(d_grids_, nslots_, cap);
        for (int stage = 1; stage <= 2; ++stage) {
            for (int v = 0; v < 2 && e1 == cudaSuccess; ++v)
                e1 = launch_records(stage, v, d_grids_, d_q_[TILE_COUNT + v], (int)cap_[TILE_COUNT + v],
                                    record_blocks(1 << 30, nsm_, v), cap, cnt + TILE_COUNT + v);
            if (e1 == cudaSuccess)
                e1 = launch_stage(c.shape, stage, d_grids_, d_q_[c.shape], (int)cap_[c.shape],
                                  stage_blocks(1 << 30, nsm_), cap, cnt + c.shape);
            if (e1 == cudaSuccess)
                e1 = launch_update(stage, d_grids_, d_q_[TILE_COUNT + 2], (int)cap_[TILE_COUNT + 2],
                                   update_blocks(1 << 30, nsm_, c.cpt), cap, cnt + TILE_COUNT + 2, c.cpt);
        }
        if (e1 == cudaSuccess) e1 = launch_end_step(d_grids_, nslots_, cap);
        e = cudaStreamEndCapture(cap, &graph);
        if (e1 != cudaSuccess) e = e1;
    }
    cudaStreamDestroy(cap);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec_[cand], graph, 0);
    if (e == cudaSuccess) captures_ += 1;
    if (graph) cudaGraphDestroy(graph);
    if (e == cudaSuccess) e = cudaGraphUpload(exec_[cand], stream_);
    return e;
}

int BatchEngine::next_candidate() const
{
    if (chosen_ >= 0) return chosen_;
    // the first candidate of the current phase without enough measurements
    for (int k = 0; k < (int)cands_.size(); ++k)
        if (cands_[k].shape >= 0 && trial_[k] < 0.0) return k;
    return 0;
}

void BatchEngine::record_time(int cand, double ms_per_cell_step)
{
    if (chosen_ >= 0 || !(ms_per_cell_step > 0.0)) return;
    trial_[cand] = ms_per_cell_step;
    for (int k = 0; k < (int)cands_.size(); ++k)
        if (cands_[k].shape >= 0 && trial_[k] < 0.0) return;   // the phase is not finished
    int best = 0;
    for (int k = 0; k < (int)cands_.size(); ++k)
        if (cands_[k].shape >= 0 && trial_[k] < trial_[best]) best = k;
    if (tune_phase_ == 0) {
        // phase 2: cells per thread of the update kernel with the best shape
        tune_phase_ = 1;
        bool any = false;
        for (int k = 0; k < (int)cands_.size(); ++k)
            if (cands_[k].shape < 0) {
                cands_[k].shape = cands_[best].shape;
                any = true;
            }
        if (any) return;
    }
    chosen_ = best;
}

cudaError_t BatchEngine::replay(int cand, int nsteps, cudaEvent_t before, cudaEvent_t after, long* launches)
{
    cudaError_t e = cudaSuccess;
    if (!exec_[cand]) e = capture(cand);
    if (e == cudaSuccess && before) e = cudaEventRecord(before, stream_);
    for (int k = 0; k < nsteps && e == cudaSuccess; ++k) {
        e = cudaGraphLaunch(exec_[cand], stream_);
        if (launches) *launches += launches_per_step_;
    }
    if (e == cudaSuccess && after) e = cudaEventRecord(after, stream_);
    return e;
}

cudaError_t BatchEngine::run(int nsteps, long* launches, bool tune)
{
    cudaError_t e = cudaSuccess;
    int k = 0;
    cudaEvent_t a = nullptr, b = nullptr;
    while (tune && chosen_ < 0 && k < nsteps && e == cudaSuccess) {
        if (!a) {
            e = cudaEventCreate(&a);
            if (e == cudaSuccess) e = cudaEventCreate(&b);
            if (e != cudaSuccess) break;
        }
        // each candidate: one untimed step, then one timed step
        const int cand = next_candidate();
        e = replay(cand, 1, nullptr, nullptr, launches);
        ++k;
        if (e != cudaSuccess || k >= nsteps) break;
        e = replay(cand, 1, a, b, launches);
        ++k;
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess) record_time(cand, cells_ > 0 ? ms / (double)cells_ : 0.0);
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (e != cudaSuccess) return e;
    if (k < nsteps) e = replay(next_candidate(), nsteps - k, nullptr, nullptr, launches);
    return e;
}

cudaError_t BatchEngine::snapshot(Ctrl* dst)
{
    snapshot_kernel<<<(nslots_ + 127) / 128, 128, 0, stream_>>>(d_grids_, nslots_, dst);
    return cudaGetLastError();
}

}  // namespace cgks

// ---------------------------------------------------------------------------
// cgks_batch_step: one engine per distinct solver set, least recently used
// engines dropped beyond kMaxPlans.
using namespace cgks;

namespace {

constexpr size_t kMaxPlans = 8;

struct Plan {
    std::vector<cgks_solver*> key;
    BatchEngine* engine;
};

std::mutex g_batch_mu;
std::list<Plan> g_plans;   // most recently used first

}  // namespace

extern "C" void cgks_set_batch_error(const char* m);
extern "C" void cgks_set_launch_count(long n);

extern "C" {

void cgks_forget_solver_plans(cgks_solver* s)
{
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (auto it = g_plans.begin(); it != g_plans.end();) {
        if (std::find(it->key.begin(), it->key.end(), s) != it->key.end()) {
            delete it->engine;
            it = g_plans.erase(it);
        } else {
            ++it;
        }
    }
}

cgks_status cgks_batch_step(cgks_solver* const* solvers, int n, int nsteps)
{
    cgks_set_launch_count(0);
    if (!solvers || n <= 0 || nsteps < 0) {
        cgks_set_batch_error("bad arguments");
        return CGKS_E_INVAL;
    }
    for (int g = 0; g < n; ++g) {
        if (!solvers[g]) { cgks_set_batch_error("NULL solver in batch"); return CGKS_E_INVAL; }
        if (solvers[g]->prob.dim != solvers[0]->prob.dim) {
            cgks_set_batch_error("mixed dims in one batch");
            return CGKS_E_INVAL;
        }
    }
    std::lock_guard<std::mutex> lk(g_batch_mu);
    nvtxRangePushA("cgks_batch_step");
    struct Pop { ~Pop() { nvtxRangePop(); } } pop;
    std::vector<cgks_solver*> key(solvers, solvers + n);
    auto it = std::find_if(g_plans.begin(), g_plans.end(), [&](const Plan& p) { return p.key == key; });
    BatchEngine* E = nullptr;
    cudaError_t e = cudaSuccess;
    if (it != g_plans.end()) {
        E = it->engine;
        g_plans.splice(g_plans.begin(), g_plans, it);
    } else {
        e = BatchEngine::create(n, solvers[0]->prob.dim, solvers[0]->stream, -1, &E);
        if (e == cudaSuccess) {
            std::vector<std::pair<int, GridDev>> members;
            for (int g = 0; g < n; ++g) members.emplace_back(g, solvers[g]->host_desc);
            e = E->set_members(members);
            if (e != cudaSuccess) { delete E; E = nullptr; }
        }
        if (e != cudaSuccess) {
            cgks_set_batch_error((std::string("batch plan: ") + cudaGetErrorString(e)).c_str());
            return CGKS_E_CUDA;
        }
        g_plans.push_front(Plan{key, E});
        while (g_plans.size() > kMaxPlans) {
            delete g_plans.back().engine;
            g_plans.pop_back();
        }
    }
    long launches = 1;
    e = launch_batch_resume(E->device_table(), n, E->stream());
    if (e == cudaSuccess) e = E->run(nsteps, &launches);
    if (e == cudaSuccess) e = cudaStreamSynchronize(E->stream());
    if (e != cudaSuccess) {
        cgks_set_batch_error((std::string("batched step: ") + cudaGetErrorString(e)).c_str());
        return CGKS_E_CUDA;
    }
    cgks_set_launch_count(launches);
    return CGKS_OK;
}

int cgks_batch_tile_shape(cgks_solver* const* solvers, int n)
{
    std::lock_guard<std::mutex> lk(g_batch_mu);
    std::vector<cgks_solver*> key(solvers, solvers + n);
    for (const Plan& p : g_plans)
        if (p.key == key) return p.engine->chosen() >= 0 ? p.engine->candidate(p.engine->chosen()).shape : -1;
    return -1;
}

int cgks_batch_update_cpt(cgks_solver* const* solvers, int n)
{
    std::lock_guard<std::mutex> lk(g_batch_mu);
    std::vector<cgks_solver*> key(solvers, solvers + n);
    for (const Plan& p : g_plans)
        if (p.key == key) return p.engine->chosen() >= 0 ? p.engine->candidate(p.engine->chosen()).cpt : -1;
    return -1;
}

}  // extern "C"
