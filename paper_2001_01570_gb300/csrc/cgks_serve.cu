// cgks_serve.cu -- continuous-batching solve server behind cgks_serve_* in
// include/cgks.h.
//
// Requests (2D problems with an initial state and a step count) arrive on any
// thread.  Three threads of the server do the rest, each on its own stream:
//   scheduler   admits pending requests in arrival order into free slots while
//               their device bytes fit the HBM budget; launches rounds of
//               steps_per_round steps of the batched engine (cgks_batch.cu) over
//               the active grids (all of them, or those with the least remaining
//               work up to fill_cells cells); after each round copies all control blocks
//               to pinned host memory and, one round later, retires the grids
//               that reached their step count (or failed).  It keeps two
//               rounds in flight, so its host work overlaps the GPU's.
//   uploader    allocates an admitted request's device memory from a
//               stream-ordered pool and copies its initial state in, while
//               the rounds run; the scheduler adds the grid to the engine's
//               queues (patched in place: the captured graphs stay) at the next
//               round boundary after the copy has finished
//   downloader  copies a retired grid's state to host memory once the rounds
//               that could still touch it are done, frees its device memory and
//               completes the request
// Every grid carries its own step target and dt, so grids of any size and step
// count share a launch, and a grid's results do not depend on what it shares
// the launch with.
#include "cgks_internal.h"
#include "../../include/cgks.h"

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

using namespace cgks;

namespace {

using clock_t_ = std::chrono::steady_clock;

double now_s()
{
    return std::chrono::duration<double>(clock_t_::now().time_since_epoch()).count();
}

enum ReqState { R_PENDING, R_LOADING, R_READY, R_ACTIVE, R_RETIRING, R_DONE };

struct Request {
    long id = 0;
    cgks_problem prob;
    std::vector<double> init;      // host copy of the initial planes (until uploaded)
    int nsteps = 0;
    size_t bytes = 0;              // device bytes while admitted
    long long cells = 0;
    double t_arrival = 0, t_admit = 0, t_done = 0;
    std::vector<double> result;    // host copy of the final planes
    int status = CGKS_OK;
    bool done = false;
    ReqState state = R_PENDING;
    // device side, between admission and completion
    int slot = -1;
    char* mem = nullptr;
    GridDev desc;
    cudaEvent_t ev = nullptr;      // upload finished / last round that touches the grid
    double t_join = 0;             // when the grid's first round was launched
    long long steps_seen = 0;      // steps done at the latest snapshot read
    Ctrl final_ctrl;
    int forced_status = CGKS_OK;   // set when the scheduler stopped before the grid finished
};

// one grid's device memory: 3 x 12 state planes, face-row records, face
// results, control block, descriptor (the kernels of cgks_create's layout)
struct GridLayout {
    size_t planes, records, faces, ctrl, desc, total;
};

GridLayout grid_layout(const cgks_problem& p)
{
    GridLayout L;
    const size_t PL = (size_t)p.nx * p.ny;
    L.planes = 0;
    L.records = L.planes + 36 * PL * sizeof(double);
    L.faces = L.records + record_doubles(p.nx, p.ny, 2) * sizeof(double);
    L.ctrl = (L.faces + face_doubles(p.nx, p.ny, 2) * sizeof(double) + 255) & ~(size_t)255;
    L.desc = L.ctrl + 256;
    L.total = L.desc + ((sizeof(GridDev) + 255) & ~(size_t)255);
    return L;
}

struct InFlight {
    long round;
    int cand;
    int buf;
    long long cells;
    std::vector<long> members;       // ids of the grids this round computed (a finished request
                                     // may be freed by its caller before the round is read)
};

}  // namespace

struct cgks_server {
    cgks_serve_cfg cfg;
    int device = 0;
    cudaStream_t S = nullptr, Cu = nullptr, Cd = nullptr;
    bool own_S = false;
    cudaMemPool_t pool = nullptr;
    std::thread sched, uploader, downloader;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done, cv_up, cv_down;
    std::deque<Request*> pending, up_jobs, down_jobs;
    std::vector<Request*> ready;
    std::vector<Request*> slots;          // max_active entries, NULL = free
    std::map<long, Request*> requests;
    bool stopping = false, workers_exit = false, worker_stopped = false;
    long next_id = 1;
    size_t bytes_in_use = 0, bytes_peak = 0;
    long inflight_requests = 0;           // admitted and not yet completed
    // statistics
    long submitted = 0, completed = 0, rejected = 0, failed = 0, rounds = 0;
    double cell_updates = 0.0;
    double t_first_arrival = -1.0, t_last_done = -1.0;
    double gpu_s = 0.0, active_s = 0.0;
    std::vector<double> latencies;
    std::string worker_error;
    int worker_status = CGKS_OK;
    int tile_shape = -1, update_cpt = -1;
    long graph_captures = 0;
    double t_start = 0.0;                 // cgks_serve_start
    FILE* log = nullptr;                  // one JSON line per finished request (cfg.log_path)
};

namespace {

thread_local std::string s_err;

cgks_status sfail(cgks_status st, const std::string& m)
{
    s_err = m;
    return st;
}

// complete a request (lock held)
void finish(cgks_server* S, Request* r, int status, double t)
{
    r->status = status;
    r->done = true;
    r->state = R_DONE;
    r->t_done = t;
    if (status == CGKS_OK) {
        S->completed += 1;
        S->cell_updates += (double)r->cells * r->nsteps;
        S->latencies.push_back(r->t_done - r->t_arrival);
    } else {
        S->failed += 1;
    }
    S->t_last_done = t;
    if (S->log) {
        const double t0 = S->t_start;
        fprintf(S->log,
                "{\"id\": %ld, \"nx\": %d, \"ny\": %d, \"steps\": %d, \"cells\": %lld, \"status\": %d, "
                "\"arrival_s\": %.6f, \"admit_s\": %.6f, \"first_round_s\": %.6f, \"done_s\": %.6f, "
                "\"latency_s\": %.6f}\n",
                r->id, r->prob.nx, r->prob.ny, r->nsteps, r->cells, status, r->t_arrival - t0,
                r->t_admit > 0 ? r->t_admit - t0 : -1.0, r->t_join > 0 ? r->t_join - t0 : -1.0, t - t0,
                t - r->t_arrival);
        fflush(S->log);
    }
    S->cv_done.notify_all();
}

void upload_loop(cgks_server* S)
{
    cudaSetDevice(S->device);
    for (;;) {
        Request* r = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_up.wait(lk, [&] { return S->workers_exit || !S->up_jobs.empty(); });
            if (S->up_jobs.empty()) return;
            r = S->up_jobs.front();
            S->up_jobs.pop_front();
        }
        nvtxRangePushA("serve upload");
        const GridLayout L = grid_layout(r->prob);
        cudaError_t e = cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocFromPoolAsync((void**)&r->mem, L.total, S->pool, S->Cu);
        if (e == cudaSuccess) {
            fill_grid_desc(r->prob, (double*)(r->mem + L.planes), (double*)(r->mem + L.records),
                           (double*)(r->mem + L.faces), (Ctrl*)(r->mem + L.ctrl), r->desc);
            GridDev* d_desc = (GridDev*)(r->mem + L.desc);
            e = cudaMemcpyAsync(r->desc.buf[0], r->init.data(), 12 * (size_t)r->cells * sizeof(double),
                                cudaMemcpyHostToDevice, S->Cu);
            if (e == cudaSuccess) e = cudaMemcpyAsync(d_desc, &r->desc, sizeof(GridDev), cudaMemcpyHostToDevice, S->Cu);
            if (e == cudaSuccess) e = launch_set_ctrl(r->desc.ctrl, 0.0, 0.0, r->nsteps, 1, S->Cu);
            if (e == cudaSuccess) e = launch_cfl(d_desc, 0, r->desc, S->Cu);
            if (e == cudaSuccess) e = cudaEventRecord(r->ev, S->Cu);
            // the host copy of the initial state may go once the copy has run
            if (e == cudaSuccess) e = cudaEventSynchronize(r->ev);
        }
        nvtxRangePop();
        std::lock_guard<std::mutex> lk(S->mu);
        if (e != cudaSuccess) {
            if (r->mem) cudaFreeAsync(r->mem, S->Cu);
            r->mem = nullptr;
            if (r->ev) cudaEventDestroy(r->ev);
            r->ev = nullptr;
            S->slots[r->slot] = nullptr;
            S->bytes_in_use -= r->bytes;
            S->inflight_requests -= 1;
            finish(S, r, e == cudaErrorMemoryAllocation ? CGKS_E_NOMEM : CGKS_E_CUDA, now_s());
            S->cv_sched.notify_all();
            continue;
        }
        r->init.clear();
        r->init.shrink_to_fit();
        if (S->worker_stopped) {
            // the scheduler is gone: the downloader frees the grid and reports the failure
            r->forced_status = S->worker_status ? S->worker_status : CGKS_E_CUDA;
            memset(&r->final_ctrl, 0, sizeof(Ctrl));
            r->state = R_RETIRING;
            S->slots[r->slot] = nullptr;
            S->down_jobs.push_back(r);
            S->cv_down.notify_one();
            continue;
        }
        r->state = R_READY;
        S->ready.push_back(r);
        S->cv_sched.notify_all();
    }
}

void download_loop(cgks_server* S)
{
    cudaSetDevice(S->device);
    for (;;) {
        Request* r = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_down.wait(lk, [&] { return S->workers_exit || !S->down_jobs.empty(); });
            if (S->down_jobs.empty()) return;
            r = S->down_jobs.front();
            S->down_jobs.pop_front();
        }
        nvtxRangePushA("serve download");
        const Ctrl& c = r->final_ctrl;
        cudaError_t e = cudaStreamWaitEvent(S->Cd, r->ev, 0);
        r->result.resize((size_t)12 * r->cells);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(r->result.data(), r->desc.buf[c.par & 1], 12 * (size_t)r->cells * sizeof(double),
                                cudaMemcpyDeviceToHost, S->Cd);
        if (e == cudaSuccess) e = cudaStreamSynchronize(S->Cd);
        cudaFreeAsync(r->mem, S->Cd);
        r->mem = nullptr;
        nvtxRangePop();
        const double t = now_s();
        std::lock_guard<std::mutex> lk(S->mu);
        cudaEventDestroy(r->ev);
        r->ev = nullptr;
        S->bytes_in_use -= r->bytes;
        S->inflight_requests -= 1;
        int st = CGKS_OK;
        if (r->forced_status != CGKS_OK) st = r->forced_status;
        else if (e != cudaSuccess) st = CGKS_E_CUDA;
        else if (c.status & kStatusBounds) st = CGKS_E_CUDA;
        else if (c.status & CGKS_E_NONPHYSICAL) st = CGKS_E_NONPHYSICAL;
        else if (c.steps < r->nsteps) st = CGKS_E_CUDA;
        finish(S, r, st, t);
        S->cv_sched.notify_all();
    }
}

// scheduler thread body
// the server's streams and its stream-ordered pool (freed grids stay reserved
// for the next ones), created by the scheduler before it admits anything
cudaError_t setup_device(cgks_server* S)
{
    cudaError_t e = cudaSetDevice(S->device);
    if (e == cudaSuccess && !S->S) {
        e = cudaStreamCreateWithFlags(&S->S, cudaStreamNonBlocking);
        S->own_S = (e == cudaSuccess);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->Cu, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->Cd, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = S->device;
        e = cudaMemPoolCreate(&S->pool, &props);
        if (e == cudaSuccess) {
            unsigned long long keep = (unsigned long long)S->cfg.hbm_budget_bytes;
            e = cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    return e;
}

void sched_loop(cgks_server* S)
{
    const int nslots = S->cfg.max_active;
    BatchEngine* E = nullptr;
    Ctrl* d_snap = nullptr;
    Ctrl* h_snap = nullptr;
    cudaEvent_t ev_snap[2] = {}, ev_r0[2] = {}, ev_r1[2] = {};
    cudaError_t e = setup_device(S);
    if (e == cudaSuccess) e = BatchEngine::create(nslots, 2, S->S, S->cfg.tile_shape, &E);
    if (e == cudaSuccess) e = cudaMalloc(&d_snap, 2 * (size_t)nslots * sizeof(Ctrl));
    if (e == cudaSuccess) e = cudaHostAlloc(&h_snap, 2 * (size_t)nslots * sizeof(Ctrl), cudaHostAllocDefault);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = cudaEventCreateWithFlags(&ev_snap[b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreate(&ev_r0[b]);
        if (e == cudaSuccess) e = cudaEventCreate(&ev_r1[b]);
    }
    std::deque<InFlight> inflight;
    long round = 0;
    std::vector<std::pair<int, long>> last_run;
    double t_active0 = -1.0;   // start of the current stretch with active grids
    while (e == cudaSuccess) {
        std::vector<Request*> joined;
        int nactive = 0;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            for (Request* r : S->slots) nactive += (r && r->state == R_ACTIVE);
            const bool idle = nactive == 0 && inflight.empty() && S->ready.empty();
            if (idle && S->stopping && S->pending.empty() && S->inflight_requests == 0) break;
            // admission in arrival order: a free slot and room in the budget
            while (!S->pending.empty()) {
                Request* r = S->pending.front();
                if (S->bytes_in_use + r->bytes > (size_t)S->cfg.hbm_budget_bytes) break;
                int slot = -1;
                for (int k = 0; k < nslots && slot < 0; ++k)
                    if (!S->slots[k]) slot = k;
                if (slot < 0) break;
                S->pending.pop_front();
                S->slots[slot] = r;
                r->slot = slot;
                r->state = R_LOADING;
                r->t_admit = now_s();
                S->bytes_in_use += r->bytes;
                S->bytes_peak = std::max(S->bytes_peak, S->bytes_in_use);
                S->inflight_requests += 1;
                S->up_jobs.push_back(r);
                S->cv_up.notify_one();
            }
            joined.swap(S->ready);
            if (idle && joined.empty()) {
                // nothing to run: wait for an upload, a completion (room in the budget), a request or stop
                S->cv_sched.wait_for(lk, std::chrono::milliseconds(50));
                continue;
            }
        }
        // grids whose upload finished join at this round boundary
        for (Request* r : joined) {
            e = cudaStreamWaitEvent(S->S, r->ev, 0);
            if (e != cudaSuccess) break;
            std::lock_guard<std::mutex> lk(S->mu);
            r->state = R_ACTIVE;
        }
        if (e != cudaSuccess) break;
        // the round's grids: every active one, or (least-remaining-work order) the active grids
        // sorted by remaining cell-updates, as many as fill fill_cells; the others wait with their
        // state untouched (they are not in the descriptor table while they wait)
        std::vector<Request*> run;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (int k = 0; k < nslots; ++k) {
                Request* r = S->slots[k];
                if (r && r->state == R_ACTIVE) run.push_back(r);
            }
        }
        if (S->cfg.order == CGKS_SERVE_LEAST_WORK_FIRST && !run.empty()) {
            auto rem = [](const Request* r) { return (double)r->cells * (double)(r->nsteps - r->steps_seen); };
            std::stable_sort(run.begin(), run.end(), [&](const Request* a, const Request* b) { return rem(a) < rem(b); });
            double cells = 0.0;
            size_t n = 0;
            while (n < run.size() && (n == 0 || cells < S->cfg.fill_cells)) cells += (double)run[n++]->cells;
            run.resize(n);
            std::sort(run.begin(), run.end(), [](const Request* a, const Request* b) { return a->slot < b->slot; });
        }
        // the composition by request id (ids are never reused; a freed request's address may be)
        std::vector<std::pair<int, long>> key;
        for (Request* r : run) key.emplace_back(r->slot, r->id);
        if (key != last_run) {
            std::vector<std::pair<int, GridDev>> members;
            for (Request* r : run) members.emplace_back(r->slot, r->desc);
            e = E->set_members(members);
            if (e != cudaSuccess) break;
            last_run = key;
        }
        if (!run.empty()) {
            if (t_active0 < 0.0) t_active0 = now_s();
            {
                std::lock_guard<std::mutex> lk(S->mu);
                for (Request* r : run)
                    if (r->t_join <= 0.0) r->t_join = now_s();
            }
            const int buf = (int)(round & 1);
            const int cand = E->next_candidate();
            nvtxRangePushA("serve round");
            long launches = 0;
            e = E->replay(cand, S->cfg.steps_per_round, ev_r0[buf], ev_r1[buf], &launches);
            if (e == cudaSuccess) e = E->snapshot(d_snap + (size_t)buf * nslots);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h_snap + (size_t)buf * nslots, d_snap + (size_t)buf * nslots,
                                    (size_t)nslots * sizeof(Ctrl), cudaMemcpyDeviceToHost, S->S);
            if (e == cudaSuccess) e = cudaEventRecord(ev_snap[buf], S->S);
            nvtxRangePop();
            if (e != cudaSuccess) break;
            std::vector<long> ids;
            for (Request* r : run) ids.push_back(r->id);
            inflight.push_back(InFlight{round, cand, buf, E->member_cells(), ids});
            round += 1;
        }
        // with two rounds in flight (or nothing more to launch), retire from the older one
        if (inflight.size() >= 2 || (run.empty() && !inflight.empty())) {
            const InFlight F = inflight.front();
            inflight.pop_front();
            e = cudaEventSynchronize(ev_snap[F.buf]);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev_r0[F.buf], ev_r1[F.buf]);
            if (e != cudaSuccess) break;
            if (E->chosen() < 0 && F.cells > 0) E->record_time(F.cand, ms / ((double)F.cells * S->cfg.steps_per_round));
            const Ctrl* snap = h_snap + (size_t)F.buf * nslots;
            std::lock_guard<std::mutex> lk(S->mu);
            S->rounds += 1;
            S->gpu_s += 1e-3 * ms;
            S->graph_captures = E->captures();
            if (E->chosen() >= 0) {
                S->tile_shape = E->candidate(E->chosen()).shape;
                S->update_cpt = E->candidate(E->chosen()).cpt;
            }
            for (long id : F.members) {
                auto it = S->requests.find(id);
                if (it == S->requests.end()) continue;
                Request* r = it->second;
                if (r->state != R_ACTIVE) continue;
                const Ctrl& c = snap[r->slot];
                r->steps_seen = c.steps;
                if (!c.done) continue;
                // finished (step target reached) or failed: no later round computes it; the
                // download waits for the rounds already enqueued
                r->final_ctrl = c;
                r->state = R_RETIRING;
                e = cudaEventRecord(r->ev, S->S);
                if (e != cudaSuccess) break;
                S->slots[r->slot] = nullptr;
                S->down_jobs.push_back(r);
                S->cv_down.notify_one();
            }
            bool any_active = false;
            for (Request* r : S->slots) any_active |= (r && r->state == R_ACTIVE);
            if (!any_active && inflight.empty() && t_active0 >= 0.0) {
                S->active_s += now_s() - t_active0;
                t_active0 = -1.0;
            }
        }
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (e != cudaSuccess) {
        S->worker_error = std::string("scheduler: ") + cudaGetErrorString(e);
        S->worker_status = CGKS_E_CUDA;
    }
    S->worker_stopped = true;
    // fail what can no longer run: pending, uploaded and active requests (the
    // workers finish the uploads and downloads already handed to them)
    const double t = now_s();
    for (Request* r : S->pending) {
        if (!r->done) finish(S, r, S->worker_status ? S->worker_status : CGKS_E_CUDA, t);
    }
    S->pending.clear();
    for (Request* r : S->ready) {
        S->slots[r->slot] = nullptr;
        r->state = R_RETIRING;
        r->forced_status = S->worker_status ? S->worker_status : CGKS_E_CUDA;
        memset(&r->final_ctrl, 0, sizeof(Ctrl));
        S->down_jobs.push_back(r);
        S->cv_down.notify_one();
    }
    S->ready.clear();
    for (int k = 0; k < nslots; ++k) {
        Request* r = S->slots[k];
        if (r && (r->state == R_ACTIVE || r->state == R_READY)) {
            S->slots[k] = nullptr;
            r->state = R_RETIRING;
            r->forced_status = S->worker_status ? S->worker_status : CGKS_E_CUDA;
            memset(&r->final_ctrl, 0, sizeof(Ctrl));
            cudaEventRecord(r->ev, S->S);
            S->down_jobs.push_back(r);   // the downloader frees its memory and reports its status
            S->cv_down.notify_one();
        }
    }
    S->cv_done.notify_all();
    cudaStreamSynchronize(S->S);
    delete E;
    cudaFree(d_snap);
    if (h_snap) cudaFreeHost(h_snap);
    for (int b = 0; b < 2; ++b) {
        if (ev_snap[b]) cudaEventDestroy(ev_snap[b]);
        if (ev_r0[b]) cudaEventDestroy(ev_r0[b]);
        if (ev_r1[b]) cudaEventDestroy(ev_r1[b]);
    }
}

double percentile(std::vector<double> v, double q)
{
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (v.size() - 1);
    const size_t lo = (size_t)pos;
    const size_t hi = std::min(lo + 1, v.size() - 1);
    return v[lo] + (pos - lo) * (v[hi] - v[lo]);
}

void destroy_server(cgks_server* S)
{
    if (S->Cu) cudaStreamDestroy(S->Cu);
    if (S->Cd) cudaStreamDestroy(S->Cd);
    if (S->own_S && S->S) cudaStreamDestroy(S->S);
    if (S->pool) cudaMemPoolDestroy(S->pool);
    if (S->log) fclose(S->log);
    for (auto& kv : S->requests) delete kv.second;
    delete S;
}

}  // namespace

extern "C" {

const char* cgks_serve_last_error(void) { return s_err.c_str(); }

cgks_status cgks_serve_start(const cgks_serve_cfg* cfg, cgks_server** out)
{
    if (!cfg || !out) return sfail(CGKS_E_INVAL, "NULL argument");
    if (!(cfg->hbm_budget_bytes > 0) || cfg->max_active < 1 || cfg->steps_per_round < 1)
        return sfail(CGKS_E_INVAL, "budget, max_active and steps_per_round must be positive");
    if (cfg->tile_shape >= TILE_COUNT || cfg->tile_shape == TILE_64x1)
        return sfail(CGKS_E_INVAL, "unknown or 1D tile shape");
    if (cfg->order != CGKS_SERVE_ALL_ACTIVE && cfg->order != CGKS_SERVE_LEAST_WORK_FIRST)
        return sfail(CGKS_E_INVAL, "unknown round order");
    if (cfg->order == CGKS_SERVE_LEAST_WORK_FIRST && !(cfg->fill_cells > 0))
        return sfail(CGKS_E_INVAL, "fill_cells must be positive");
    cgks_server* S = new cgks_server();
    S->cfg = *cfg;
    S->slots.assign((size_t)cfg->max_active, nullptr);
    // the current device; the scheduler thread creates the streams and the pool
    // on it (a failure there stops the server: submissions then return its status)
    if (cudaGetDevice(&S->device) != cudaSuccess) S->device = 0;
    S->S = (cudaStream_t)cfg->cuda_stream;
    S->t_start = now_s();
    if (cfg->log_path) {
        S->log = fopen(cfg->log_path, "a");
        if (!S->log) {
            destroy_server(S);
            return sfail(CGKS_E_INVAL, std::string("cannot open the request log ") + cfg->log_path);
        }
    }
    S->cfg.log_path = nullptr;   // the caller's string is not kept
    S->uploader = std::thread(upload_loop, S);
    S->downloader = std::thread(download_loop, S);
    S->sched = std::thread(sched_loop, S);
    *out = S;
    return CGKS_OK;
}

cgks_status cgks_serve_submit(cgks_server* S, const cgks_request* req, long* req_id)
{
    if (!S || !req || !req->init_planes || !req_id) return sfail(CGKS_E_INVAL, "NULL argument");
    if (req->prob.dim != 2) return sfail(CGKS_E_INVAL, "served solves are 2D");
    if (req->nsteps < 0) return sfail(CGKS_E_INVAL, "nsteps must be >= 0");
    if (validate_problem(&req->prob) != CGKS_OK)
        return sfail(CGKS_E_INVAL, std::string("bad problem: ") + cgks_last_error());
    // the budget counts what cgks_problem_device_bytes reports (an upper bound of the allocation)
    const size_t bytes = (size_t)cgks_problem_device_bytes(&req->prob);
    std::lock_guard<std::mutex> lk(S->mu);
    if (bytes > (size_t)S->cfg.hbm_budget_bytes) {
        S->rejected += 1;
        return sfail(CGKS_E_BUDGET, "request can never fit the HBM budget");
    }
    if (S->worker_stopped)
        return sfail(S->worker_status ? (cgks_status)S->worker_status : CGKS_E_BUSY,
                     "the server's scheduler has stopped: " + S->worker_error);
    if (S->stopping) return sfail(CGKS_E_BUSY, "server is stopping");
    Request* r = new Request();
    r->id = S->next_id++;
    r->prob = req->prob;
    r->cells = (long long)req->prob.nx * req->prob.ny;
    r->init.assign(req->init_planes, req->init_planes + (size_t)12 * r->cells);
    r->nsteps = req->nsteps;
    r->bytes = bytes;
    r->t_arrival = now_s();
    if (S->t_first_arrival < 0) S->t_first_arrival = r->t_arrival;
    S->requests[r->id] = r;
    S->pending.push_back(r);
    S->submitted += 1;
    *req_id = r->id;
    S->cv_sched.notify_all();
    return CGKS_OK;
}

cgks_status cgks_serve_poll(cgks_server* S, long req_id, double* out_planes, int* done)
{
    if (!S || !done) return sfail(CGKS_E_INVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->requests.find(req_id);
    if (it == S->requests.end()) return sfail(CGKS_E_NOTFOUND, "unknown request id");
    Request* r = it->second;
    *done = r->done ? 1 : 0;
    if (!r->done) return CGKS_OK;
    cgks_status st = (cgks_status)r->status;
    if (out_planes && !r->result.empty()) std::copy(r->result.begin(), r->result.end(), out_planes);
    if (out_planes || r->result.empty()) {
        S->requests.erase(it);
        delete r;
    }
    return st;
}

cgks_status cgks_serve_wait(cgks_server* S, long req_id, double timeout_s, double* out_planes)
{
    if (!S) return sfail(CGKS_E_INVAL, "NULL server");
    {
        std::unique_lock<std::mutex> lk(S->mu);
        auto deadline = clock_t_::now() + std::chrono::duration_cast<clock_t_::duration>(
                                              std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0.0));
        for (;;) {
            auto it = S->requests.find(req_id);
            if (it == S->requests.end()) return sfail(CGKS_E_NOTFOUND, "unknown request id");
            if (it->second->done) break;
            if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
                auto jt = S->requests.find(req_id);
                if (jt == S->requests.end()) return sfail(CGKS_E_NOTFOUND, "unknown request id");
                if (!jt->second->done) return sfail(CGKS_E_TIMEOUT, "request not finished within the timeout");
            }
        }
    }
    int done = 0;
    return cgks_serve_poll(S, req_id, out_planes, &done);
}

cgks_status cgks_serve_stats(cgks_server* S, cgks_serve_stats_t* out)
{
    if (!S || !out) return sfail(CGKS_E_INVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->rejected = S->rejected;
    out->failed = S->failed;
    long active = 0;
    for (Request* r : S->slots) active += (r != nullptr);
    out->active = active;
    out->pending = (long)S->pending.size();
    out->rounds = S->rounds;
    out->cell_updates = S->cell_updates;
    out->busy_s = S->active_s;
    out->wall_s = (S->t_first_arrival >= 0 && S->t_last_done >= 0) ? S->t_last_done - S->t_first_arrival : 0.0;
    out->cell_updates_per_s = out->wall_s > 0 ? S->cell_updates / out->wall_s : 0.0;
    out->p50_s = percentile(S->latencies, 0.50);
    out->p99_s = percentile(S->latencies, 0.99);
    out->mean_s = 0.0;
    for (double l : S->latencies) out->mean_s += l;
    if (!S->latencies.empty()) out->mean_s /= S->latencies.size();
    out->hbm_in_use = (double)S->bytes_in_use;
    out->hbm_peak = (double)S->bytes_peak;
    out->tile_shape = S->tile_shape;
    out->update_cpt = S->update_cpt;
    out->gpu_s = S->gpu_s;
    out->round_overhead = S->active_s > 0 ? 1.0 - S->gpu_s / S->active_s : 0.0;
    out->graph_captures = S->graph_captures;
    return CGKS_OK;
}

cgks_status cgks_serve_stop(cgks_server* S)
{
    if (!S) return sfail(CGKS_E_INVAL, "NULL server");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
        S->cv_sched.notify_all();
    }
    if (S->sched.joinable()) S->sched.join();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->workers_exit = true;
        S->cv_up.notify_all();
        S->cv_down.notify_all();
    }
    if (S->uploader.joinable()) S->uploader.join();
    if (S->downloader.joinable()) S->downloader.join();
    cudaStreamSynchronize(S->Cu);
    cudaStreamSynchronize(S->Cd);
    const cgks_status st = (cgks_status)S->worker_status;
    if (st != CGKS_OK) s_err = S->worker_error;
    destroy_server(S);
    return st;
}

}  // extern "C"
