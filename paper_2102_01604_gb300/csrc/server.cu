// server.cu -- continuous batching of fit requests (mpm_server_*).
//
// Requests (one subject each, any matrix size, contrasts and echo counts) are
// queued by mpm_server_submit.  Each mpm_server_step is one scheduling round:
//   1. admit queued requests, first come first served, while a slot is free
//      and their fit workspace fits in the free part of the caller's device
//      arena (the library allocates nothing);
//   2. advance every active request by one update on its own stream -- the
//      PCG solve of the previous update and the evaluation of the objective
//      at the new maps -- so the requests' kernels overlap on the GPU;
//   3. wait once for all slots and test convergence on the host
//      (|F_prev - F| < tol_gn |F_prev|, or gn_iters reached);
//   4. finish converged requests (uncertainty if asked, report), free their
//      workspace.
// Maps, JTV weights, gradients, Hessians and PCG state stay resident in the
// arena between rounds.  Each request runs exactly the launches of mpm_fit
// with the same schedule, so its result is the same alone and in the mix.
#include <deque>
#include <map>
#include <mutex>
#include <vector>

#include "mpm_internal.cuh"

namespace mpm {

enum ReqState { kQueued = 0, kActive = 1, kDone = 2, kFailed = 3 };

struct Request {
    int ticket;
    int state;
    mpm_problem problem;
    mpm_opts opts;
    DevProblem P;
    const void* x;
    const float *b1p, *b1m;
    float *y, *var;
    size_t ws_off, ws_bytes;
    FitWs L;
    int slot;
    int it;
    bool solve_pending, w_fresh;
    double F_prev;
    mpm_report report;
    mpm_status status;
    cudaEvent_t ready;        // inputs ready on the caller's stream
};

struct Arena {
    char* base;
    size_t bytes;
    std::map<size_t, size_t> free_;   // offset -> size, coalesced

    void init(void* b, size_t n)
    {
        base = static_cast<char*>(b);
        bytes = n;
        free_.clear();
        free_[0] = n;
    }
    bool alloc(size_t n, size_t* off)
    {
        n = (n + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n, at = it->first + n;
                free_.erase(it);
                if (rest) free_[at] = rest;
                return true;
            }
        return false;
    }
    void release(size_t off, size_t n)
    {
        n = (n + 255) & ~(size_t)255;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t largest() const
    {
        size_t m = 0;
        for (auto& f : free_) m = f.second > m ? f.second : m;
        return m;
    }
};

}  // namespace mpm

using namespace mpm;

struct mpm_server {
    std::mutex mu;
    Arena arena;
    int max_slots;
    cudaStream_t user;
    std::vector<cudaStream_t> slots;
    std::vector<int> slot_owner;       // ticket or -1
    std::deque<int> queue;
    std::map<int, Request> reqs;
    int next_ticket = 1;
    double* host_f;                    // pinned: nll, jtv per slot
    double* host_means;                // pinned: image means per slot
    unsigned* host_status;             // pinned: status word per slot
};

#define SRV_CUDA(call)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(MPM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));          \
    } while (0)

static mpm_status srv_sync(mpm_server* s)
{
    for (int k = 0; k < s->max_slots; ++k)
        if (s->slot_owner[k] >= 0) SRV_CUDA(cudaStreamSynchronize(s->slots[k]));
    return MPM_OK;
}

extern "C" {

mpm_status mpm_server_create(void* arena, size_t arena_bytes, int max_slots, void* stream,
                             mpm_server** out)
{
    if (!out) return fail(MPM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (max_slots < 1 || max_slots > MPM_MAX_BATCH)
        return fail(MPM_ERR_INVALID_ARG, "max_slots = %d outside [1, %d]", max_slots, MPM_MAX_BATCH);
    mpm_status st = check_dev(arena, "arena", false, 256);
    if (st != MPM_OK) return st;
    mpm_server* s = new mpm_server();
    s->arena.init(arena, arena_bytes);
    s->max_slots = max_slots;
    s->user = (cudaStream_t)stream;
    s->slots.resize(max_slots);
    s->slot_owner.assign(max_slots, -1);
    for (int k = 0; k < max_slots; ++k) {
        cudaError_t e = cudaStreamCreateWithFlags(&s->slots[k], cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (int j = 0; j < k; ++j) cudaStreamDestroy(s->slots[j]);
            delete s;
            return fail(MPM_ERR_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
        }
    }
    cudaError_t e = cudaHostAlloc((void**)&s->host_f, sizeof(double) * 2 * max_slots, 0);
    if (e == cudaSuccess)
        e = cudaHostAlloc((void**)&s->host_means, sizeof(double) * MPM_MAX_IMAGES * max_slots, 0);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&s->host_status, sizeof(unsigned) * max_slots, 0);
    if (e != cudaSuccess) {
        for (auto st2 : s->slots) cudaStreamDestroy(st2);
        delete s;
        return fail(MPM_ERR_CUDA, "cudaHostAlloc: %s", cudaGetErrorString(e));
    }
    *out = s;
    return MPM_OK;
}

mpm_status mpm_server_submit(mpm_server* s, const mpm_problem* problem, const mpm_opts* opts,
                             const void* x, const float* b1p, const float* b1m, float* y,
                             float* var_out, int* ticket)
{
    if (!s || !ticket) return fail(MPM_ERR_INVALID_ARG, "server and ticket must not be NULL");
    mpm_status st = check_problem(problem);
    if (st != MPM_OK) return st;
    if ((st = check_opts(opts)) != MPM_OK) return st;
    const DevProblem P = make_dev(problem);
    if (P.N == 0) return fail(MPM_ERR_INVALID_ARG, "empty volume");
    if ((st = check_dev(x, "x", false, problem->echo_dtype ? 2 : 4)) != MPM_OK) return st;
    if ((st = check_dev(b1p, "b1p", true, 4)) != MPM_OK) return st;
    if ((st = check_dev(b1m, "b1m", true, 4)) != MPM_OK) return st;
    if ((st = check_dev(y, "y_inout", false, 4)) != MPM_OK) return st;
    if ((st = check_dev(var_out, "var_out", true, 4)) != MPM_OK) return st;
    const size_t need = layout(P, MPM_CALL_FIT, nullptr).total;
    std::lock_guard<std::mutex> lk(s->mu);
    if (need > s->arena.bytes)
        return fail(MPM_ERR_WORKSPACE_TOO_SMALL, "request needs %zu bytes, the arena holds %zu",
                    need, s->arena.bytes);
    Request r;
    memset(&r, 0, sizeof r);
    r.ticket = s->next_ticket++;
    r.state = kQueued;
    r.problem = *problem;
    r.opts = *opts;
    r.P = P;
    r.x = x;
    r.b1p = b1p;
    r.b1m = b1m;
    r.y = y;
    r.var = var_out;
    r.ws_bytes = need;
    r.slot = -1;
    cudaError_t e = cudaEventCreateWithFlags(&r.ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(r.ready, s->user);
    if (e != cudaSuccess) return fail(MPM_ERR_CUDA, "event: %s", cudaGetErrorString(e));
    s->reqs[r.ticket] = r;
    s->queue.push_back(r.ticket);
    *ticket = r.ticket;
    return MPM_OK;
}

mpm_status mpm_server_step(mpm_server* s, int* n_active, int* n_queued, int* n_finished)
{
    if (!s) return fail(MPM_ERR_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    // 1. admission (first come first served)
    std::vector<int> admitted;
    while (!s->queue.empty()) {
        int k = 0;
        while (k < s->max_slots && s->slot_owner[k] >= 0) ++k;
        if (k == s->max_slots) break;
        Request& r = s->reqs[s->queue.front()];
        size_t off;
        if (!s->arena.alloc(r.ws_bytes, &off)) break;
        s->queue.pop_front();
        r.ws_off = off;
        r.L = layout(r.P, MPM_CALL_FIT, s->arena.base + off);
        r.slot = k;
        r.state = kActive;
        r.it = 0;
        r.solve_pending = false;
        s->slot_owner[k] = r.ticket;
        cudaStream_t st = s->slots[k];
        SRV_CUDA(cudaStreamWaitEvent(st, r.ready, 0));
        SRV_CUDA(cudaMemsetAsync(r.L.hdr, 0, sizeof(WsHeader), st));
        if (r.opts.init) {
            SRV_CUDA(launch_image_means(r.P, r.problem.echo_dtype, r.x, r.L.mean_parts, r.L.means, st));
            SRV_CUDA(cudaMemcpyAsync(s->host_means + (size_t)k * MPM_MAX_IMAGES, r.L.means,
                                     sizeof(double) * r.P.I, cudaMemcpyDeviceToHost, st));
        }
        admitted.push_back(r.ticket);
    }
    if (!admitted.empty()) {
        mpm_status st = srv_sync(s);
        if (st != MPM_OK) return st;
        for (int t : admitted) {
            Request& r = s->reqs[t];
            if (!r.opts.init) continue;
            float vals[4];
            initial_maps(&r.problem, s->host_means + (size_t)r.slot * MPM_MAX_IMAGES, vals);
            SRV_CUDA(launch_fill_maps(r.P, vals, r.y, s->slots[r.slot]));
        }
    }
    // 2. one update per active request, each on its own stream
    for (int k = 0; k < s->max_slots; ++k) {
        if (s->slot_owner[k] < 0) continue;
        Request& r = s->reqs[s->slot_owner[k]];
        cudaStream_t st = s->slots[k];
        const DevProblem& P = r.P;
        const FitWs& L = r.L;
        if (r.solve_pending) {
            SRV_CUDA(launch_solve(P, r.opts.cg_iters, r.opts.tol_cg, L.h, L.w, L.g, r.y, L.xbuf, r.y,
                                  nullptr, L.cg_rel + r.it - 1, L.cg_it + r.it - 1, L.solve, L.hdr,
                                  L.red, st));
            r.solve_pending = false;
        }
        r.w_fresh = (r.it % r.opts.newton_per_irls == 0);
        SRV_CUDA(launch_jtv(P, r.y, r.w_fresh ? L.w : nullptr, L.jtv + r.it, L.red, st));
        SRV_CUDA(launch_grad_hess(P, r.problem.echo_dtype, r.x, r.y, r.b1p, r.b1m, L.g, L.h,
                                  L.nll + r.it, L.red, st));
        SRV_CUDA(cudaMemcpyAsync(s->host_f + 2 * k, L.nll + r.it, sizeof(double),
                                 cudaMemcpyDeviceToHost, st));
        SRV_CUDA(cudaMemcpyAsync(s->host_f + 2 * k + 1, L.jtv + r.it, sizeof(double),
                                 cudaMemcpyDeviceToHost, st));
    }
    // 3. one wait, then the stopping test (same rule as mpm_fit)
    mpm_status st = srv_sync(s);
    if (st != MPM_OK) return st;
    std::vector<int> finishing;
    for (int k = 0; k < s->max_slots; ++k) {
        if (s->slot_owner[k] < 0) continue;
        Request& r = s->reqs[s->slot_owner[k]];
        const double F = s->host_f[2 * k] + s->host_f[2 * k + 1];
        bool stop = r.it >= r.opts.gn_iters;
        bool converged = false;
        if (!stop && r.opts.tol_gn > 0.0 && r.it > 0 &&
            std::fabs(r.F_prev - F) < r.opts.tol_gn * std::fabs(r.F_prev)) {
            stop = true;
            converged = true;
        }
        if (stop) {
            r.report.iters = r.it;
            r.status = (r.opts.tol_gn > 0.0 && !converged) ? MPM_WARN_NOT_CONVERGED : MPM_OK;
            finishing.push_back(r.ticket);
        } else {
            r.F_prev = F;
            r.solve_pending = true;
            r.it += 1;
        }
    }
    // 4. finish: uncertainty, reports, free the workspace
    if (!finishing.empty()) {
        for (int t : finishing) {
            Request& r = s->reqs[t];
            cudaStream_t stm = s->slots[r.slot];
            const int it = r.it;
            if (r.var) {
                if (!r.w_fresh)
                    SRV_CUDA(launch_jtv(r.P, r.y, r.L.w, r.L.jtv + MPM_MAX_REPORT + 1, r.L.red, stm));
                SRV_CUDA(launch_uncertainty(r.P, r.L.h, r.L.w, r.y, r.var, nullptr, nullptr,
                                            &r.L.hdr->status, stm));
            }
            SRV_CUDA(cudaMemcpyAsync(r.report.nll, r.L.nll, sizeof(double) * (it + 1), cudaMemcpyDeviceToHost, stm));
            SRV_CUDA(cudaMemcpyAsync(r.report.jtv, r.L.jtv, sizeof(double) * (it + 1), cudaMemcpyDeviceToHost, stm));
            if (it > 0) {
                SRV_CUDA(cudaMemcpyAsync(r.report.cg_rel, r.L.cg_rel, sizeof(double) * it, cudaMemcpyDeviceToHost, stm));
                SRV_CUDA(cudaMemcpyAsync(r.report.cg_done, r.L.cg_it, sizeof(int) * it, cudaMemcpyDeviceToHost, stm));
            }
            SRV_CUDA(cudaMemcpyAsync(s->host_status + r.slot, &r.L.hdr->status, sizeof(unsigned),
                                     cudaMemcpyDeviceToHost, stm));
        }
        st = srv_sync(s);
        if (st != MPM_OK) return st;
        for (int t : finishing) {
            Request& r = s->reqs[t];
            for (int i = 0; i <= r.it; ++i) r.report.F[i] = r.report.nll[i] + r.report.jtv[i];
            if (s->host_status[r.slot]) r.status = MPM_ERR_NUMERIC;
            r.state = r.status < 0 ? kFailed : kDone;
            s->slot_owner[r.slot] = -1;
            s->arena.release(r.ws_off, r.ws_bytes);
            cudaEventDestroy(r.ready);
            r.slot = -1;
        }
    }
    int active = 0;
    for (int k = 0; k < s->max_slots; ++k) active += s->slot_owner[k] >= 0;
    if (n_active) *n_active = active;
    if (n_queued) *n_queued = (int)s->queue.size();
    if (n_finished) *n_finished = (int)finishing.size();
    return MPM_OK;
}

mpm_status mpm_server_poll(mpm_server* s, int ticket, int* state, mpm_status* status,
                           mpm_report* report)
{
    if (!s || !state) return fail(MPM_ERR_INVALID_ARG, "server and state must not be NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(MPM_ERR_INVALID_ARG, "unknown ticket %d", ticket);
    const Request& r = it->second;
    *state = r.state;
    if (status) *status = r.status;
    if (report && (r.state == kDone || r.state == kFailed)) *report = r.report;
    return MPM_OK;
}

mpm_status mpm_server_destroy(mpm_server* s)
{
    if (!s) return MPM_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto st : s->slots) {
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
        }
        for (auto& kv : s->reqs)
            if (kv.second.state == kQueued || kv.second.state == kActive) cudaEventDestroy(kv.second.ready);
        cudaFreeHost(s->host_f);
        cudaFreeHost(s->host_means);
        cudaFreeHost(s->host_status);
    }
    delete s;
    return MPM_OK;
}

}  // extern "C"
