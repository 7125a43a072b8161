// cgks_serve.cu -- continuous-batching solve server behind cgks_serve_* in
// include/cgks.h.
//
// Requests (2D problems with an initial state and a step count) arrive on any
// thread.  One scheduler thread owns all device work:
//   admit    pending requests in arrival order while the active set is below
//            max_active and their device planes fit the HBM budget; the state
//            is uploaded and the solve joins the active set
//   run      one round = steps_per_round steps of the batched persistent
//            launch over the tiles of every active grid (a CUDA graph per
//            active-set composition); every grid carries its own step target
//            and dt, so grids of any size and step count share a launch
//   retire   grids that reached their target (or failed) are copied back to
//            host memory, their device memory is freed and their latency
//            (arrival to result) is recorded
// Requests that arrive while others run are admitted at the next round
// boundary, as slots and memory free up.
#include "cgks_internal.h"
#include "../../include/cgks.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

extern "C" void cgks_forget_solver_plans(cgks_solver* s);
cgks_status cgks_set_step_target(cgks_solver* s, long long target);

namespace {

using clock_t_ = std::chrono::steady_clock;

double now_s()
{
    return std::chrono::duration<double>(clock_t_::now().time_since_epoch()).count();
}

struct Request {
    long id = 0;
    cgks_problem prob;
    std::vector<double> init;      // host copy of the initial planes
    int nsteps = 0;
    size_t bytes = 0;              // device bytes while active
    long long cells = 0;
    double t_arrival = 0, t_admit = 0, t_done = 0;
    cgks_solver* solver = nullptr;
    std::vector<double> result;    // host copy of the final planes
    int status = CGKS_OK;
    bool done = false;
    bool taken = false;
};

}  // namespace

struct cgks_server {
    cgks_serve_cfg cfg;
    cudaStream_t stream = nullptr;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> pending;
    std::vector<Request*> active;
    std::map<long, Request*> requests;
    bool stopping = false;
    long next_id = 1;
    size_t bytes_in_use = 0, bytes_peak = 0;
    // statistics
    long submitted = 0, completed = 0, rejected = 0, failed = 0, rounds = 0;
    double cell_updates = 0.0;
    double t_first_arrival = -1.0, t_last_done = -1.0, busy_s = 0.0;
    std::vector<double> latencies;
    std::string worker_error;
    int worker_status = CGKS_OK;
    int tile_shape = -1;
};

namespace {

thread_local std::string s_err;

cgks_status sfail(cgks_status st, const std::string& m)
{
    s_err = m;
    return st;
}

size_t request_bytes(const cgks_problem& p)
{
    return (size_t)cgks_problem_device_bytes(&p);
}

// scheduler thread body
void serve_loop(cgks_server* S)
{
    cgks::BatchPlan* plan = nullptr;
    bool membership_changed = true;
    for (;;) {
        // ---- admit
        std::vector<Request*> admitted;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            while (S->pending.empty() && S->active.empty() && !S->stopping) S->cv_work.wait(lk);
            if (S->pending.empty() && S->active.empty() && S->stopping) break;
            while (!S->pending.empty() && (int)S->active.size() < S->cfg.max_active &&
                   S->bytes_in_use + S->pending.front()->bytes <= (size_t)S->cfg.hbm_budget_bytes) {
                Request* r = S->pending.front();
                S->pending.pop_front();
                S->bytes_in_use += r->bytes;
                S->bytes_peak = std::max(S->bytes_peak, S->bytes_in_use);
                admitted.push_back(r);
            }
        }
        for (Request* r : admitted) {
            cgks_status st = cgks_create(&r->prob, S->stream, &r->solver);
            if (st == CGKS_OK) st = cgks_set_state(r->solver, r->init.data(), 0, 0.0);
            if (st == CGKS_OK) st = cgks_set_step_target(r->solver, r->nsteps);
            r->t_admit = now_s();
            std::lock_guard<std::mutex> lk(S->mu);
            if (st != CGKS_OK) {
                r->status = st;
                r->done = true;
                S->failed += 1;
                S->bytes_in_use -= r->bytes;
                if (r->solver) { cgks_destroy(r->solver); r->solver = nullptr; }
                S->cv_done.notify_all();
                continue;
            }
            r->init.clear();
            r->init.shrink_to_fit();
            S->active.push_back(r);
            membership_changed = true;
        }
        std::vector<Request*> act;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            act = S->active;
        }
        if (act.empty()) continue;

        // ---- run one round of the batched launch
        const double t0 = now_s();
        if (membership_changed) {
            if (plan) cgks::destroy_plan(plan);
            plan = nullptr;
            std::vector<cgks_solver*> sol;
            for (Request* r : act) sol.push_back(r->solver);
            cudaError_t e = cgks::make_plan(sol.data(), (int)sol.size(), S->stream, S->tile_shape, &plan);
            if (e != cudaSuccess) {
                std::lock_guard<std::mutex> lk(S->mu);
                S->worker_error = std::string("batch plan: ") + cudaGetErrorString(e);
                S->worker_status = CGKS_E_CUDA;
                break;
            }
            membership_changed = false;
        }
        long launches = 0;
        cudaError_t e = cgks::run_plan(plan, S->cfg.steps_per_round, &launches);
        if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
        if (plan->chosen >= 0) S->tile_shape = plan->chosen;
        if (e != cudaSuccess) {
            std::lock_guard<std::mutex> lk(S->mu);
            S->worker_error = std::string("batched round: ") + cudaGetErrorString(e);
            S->worker_status = CGKS_E_CUDA;
            break;
        }
        // ---- retire finished grids
        std::vector<Request*> finished;
        for (Request* r : act) {
            double t = 0.0;
            long steps = 0;
            cgks_status st = cgks_get_state(r->solver, nullptr, 0, &t, &steps);
            if (st != CGKS_OK || steps >= r->nsteps) {
                r->status = st;
                r->result.resize((size_t)12 * r->cells);
                cgks_get_state(r->solver, r->result.data(), 0, nullptr, nullptr);
                finished.push_back(r);
            }
        }
        const double t1 = now_s();
        std::lock_guard<std::mutex> lk(S->mu);
        S->rounds += 1;
        S->busy_s += t1 - t0;
        for (Request* r : finished) {
            cgks_destroy(r->solver);
            r->solver = nullptr;
            r->t_done = t1;
            r->done = true;
            S->bytes_in_use -= r->bytes;
            if (r->status == CGKS_OK) {
                S->completed += 1;
                S->cell_updates += (double)r->cells * r->nsteps;
                S->latencies.push_back(r->t_done - r->t_arrival);
            } else {
                S->failed += 1;
            }
            S->t_last_done = t1;
            S->active.erase(std::find(S->active.begin(), S->active.end(), r));
            membership_changed = true;
        }
        if (!finished.empty()) S->cv_done.notify_all();
    }
    if (plan) cgks::destroy_plan(plan);
    std::lock_guard<std::mutex> lk(S->mu);
    for (Request* r : S->active) {
        if (r->solver) cgks_destroy(r->solver);
        r->solver = nullptr;
        r->done = true;
        r->status = S->worker_status ? S->worker_status : CGKS_E_CUDA;
    }
    S->active.clear();
    S->cv_done.notify_all();
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

}  // namespace

extern "C" {

const char* cgks_serve_last_error(void) { return s_err.c_str(); }

cgks_status cgks_serve_start(const cgks_serve_cfg* cfg, cgks_server** out)
{
    if (!cfg || !out) return sfail(CGKS_E_INVAL, "NULL argument");
    if (!(cfg->hbm_budget_bytes > 0) || cfg->max_active < 1 || cfg->steps_per_round < 1)
        return sfail(CGKS_E_INVAL, "budget, max_active and steps_per_round must be positive");
    cgks_server* S = new cgks_server();
    S->cfg = *cfg;
    S->stream = (cudaStream_t)cfg->cuda_stream;
    S->tile_shape = cfg->tile_shape;
    S->worker = std::thread(serve_loop, S);
    *out = S;
    return CGKS_OK;
}

cgks_status cgks_serve_submit(cgks_server* S, const cgks_request* req, long* req_id)
{
    if (!S || !req || !req->init_planes || !req_id) return sfail(CGKS_E_INVAL, "NULL argument");
    if (req->prob.dim != 2) return sfail(CGKS_E_INVAL, "served solves are 2D");
    if (req->nsteps < 0) return sfail(CGKS_E_INVAL, "nsteps must be >= 0");
    if (req->prob.nx < 1 || req->prob.ny < 1) return sfail(CGKS_E_INVAL, "bad grid");
    const size_t bytes = request_bytes(req->prob);
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stopping) return sfail(CGKS_E_BUSY, "server is stopping");
    if (bytes > (size_t)S->cfg.hbm_budget_bytes) {
        S->rejected += 1;
        return sfail(CGKS_E_BUDGET, "request can never fit the HBM budget");
    }
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
    S->cv_work.notify_one();
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
                if (!S->requests.count(req_id) || !S->requests[req_id]->done)
                    return sfail(CGKS_E_TIMEOUT, "request not finished within the timeout");
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
    out->active = (long)S->active.size();
    out->pending = (long)S->pending.size();
    out->rounds = S->rounds;
    out->cell_updates = S->cell_updates;
    out->busy_s = S->busy_s;
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
    return (cgks_status)S->worker_status;
}

cgks_status cgks_serve_stop(cgks_server* S)
{
    if (!S) return sfail(CGKS_E_INVAL, "NULL server");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
        S->cv_work.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    cgks_status st = (cgks_status)S->worker_status;
    for (auto& kv : S->requests) delete kv.second;
    for (Request* r : S->pending) (void)r;   // owned by `requests`
    delete S;
    return st;
}

}  // extern "C"
