// server.cu -- continuous batching of fit requests (mpm_server_*).
//
// Requests (one subject each, any matrix size, contrasts and echo counts) are
// queued by mpm_server_submit and run asynchronously, each on its own slot
// stream, through a small state machine driven by mpm_server_step:
//   admitted  -> workspace carved from the caller's device arena; image
//                means and the constant initial maps (on the device), first
//                evaluation of the objective, its two doubles copied to
//                pinned memory;
//   evaluate  -> when that copy has landed: the stopping rule of mpm_fit
//                (|F_prev - F| < tol_gn |F_prev|, or gn_iters); if it goes
//                on, the PCG solve and update and the next evaluation are
//                enqueued at once; otherwise
//   finish    -> uncertainty (if asked) and the report copied out; when that
//                has landed the request is done and its workspace is freed.
// A step never blocks: it only queries CUDA events, so every request moves at
// its own pace and the kernels of all active requests overlap on the GPU.
// Smaller volumes run on higher-priority streams (shortest job first at the
// block scheduler), so a small request is not held behind a large one.
// Maps, JTV weights, gradient, Hessian and PCG state stay resident in the
// arena.  Each request runs exactly the launches of mpm_fit, so its result is
// the same alone and in the mix.
#include <deque>
#include <map>
#include <mutex>
#include <vector>

#include "mpm_internal.cuh"

namespace mpm {

enum ReqState { kQueued = 0, kActive = 1, kDone = 2, kFailed = 3 };
enum Phase { kEval = 1, kFinish = 2 };

struct Request {
    int ticket;
    int state;
    int phase;
    mpm_problem problem;
    mpm_opts opts;
    DevProblem P;
    const void* x;
    const float *b1p, *b1m;
    float *y, *var;
    size_t ws_off, ws_bytes;
    FitWs L;
    int slot;
    int overtaken;            // later requests admitted before this one
    cudaStream_t stream;      // the slot's stream of this request's priority
    int it;
    bool w_fresh;
    double F_prev;
    mpm_report report;
    mpm_status status;
    cudaEvent_t ready;        // inputs ready on the caller's stream
    cudaEvent_t landed;       // the slot's last enqueued host copy has completed
};

// Pinned host staging of one slot.
struct SlotHost {
    double f[2];              // nll, jtv of the latest evaluation
    unsigned status;
    mpm_report report;
};

}  // namespace mpm

using namespace mpm;

struct mpm_server {
    std::mutex mu;
    Arena arena;
    int max_slots;
    cudaStream_t user;
    int prio_hi, n_prio;               // greatest priority, number of levels
    std::vector<cudaStream_t> slots;   // [slot * n_prio + level], level 0 highest
    std::vector<int> slot_owner;       // ticket or -1
    std::deque<int> queue;
    std::map<int, Request> reqs;
    int next_ticket = 1;
    SlotHost* host;                    // pinned, one per slot
};

#define SRV_CUDA(call)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(MPM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));          \
    } while (0)

// Evaluation of the objective at the current maps (same launches as mpm_fit),
// its two doubles copied to the slot's pinned staging.
static mpm_status srv_eval(mpm_server* s, Request& r)
{
    cudaStream_t st = r.stream;
    const FitWs& L = r.L;
    r.w_fresh = (r.it % r.opts.newton_per_irls == 0);
    SRV_CUDA(launch_jtv(r.P, r.y, r.w_fresh ? L.w : nullptr, L.jtv + r.it, L.red, st));
    SRV_CUDA(launch_grad_hess(r.P, r.problem.echo_dtype, r.x, r.y, r.b1p, r.b1m, L.g, L.h,
                              L.nll + r.it, L.red, &L.hdr->status, st));
    SlotHost& h = s->host[r.slot];
    SRV_CUDA(cudaMemcpyAsync(&h.f[0], L.nll + r.it, sizeof(double), cudaMemcpyDeviceToHost, st));
    SRV_CUDA(cudaMemcpyAsync(&h.f[1], L.jtv + r.it, sizeof(double), cudaMemcpyDeviceToHost, st));
    SRV_CUDA(cudaEventRecord(r.landed, st));
    r.phase = kEval;
    return MPM_OK;
}

// Uncertainty (if asked) and the report, copied to the slot's staging.
static mpm_status srv_finish(mpm_server* s, Request& r)
{
    cudaStream_t st = r.stream;
    const FitWs& L = r.L;
    const int it = r.it;
    if (r.var) {
        if (!r.w_fresh) SRV_CUDA(launch_jtv(r.P, r.y, L.w, L.jtv + MPM_MAX_REPORT + 1, L.red, st));
        SRV_CUDA(launch_uncertainty(r.P, L.h, L.w, r.y, r.var, nullptr, nullptr, &L.hdr->status, st));
    }
    SlotHost& h = s->host[r.slot];
    SRV_CUDA(cudaMemcpyAsync(h.report.nll, L.nll, sizeof(double) * (it + 1), cudaMemcpyDeviceToHost, st));
    SRV_CUDA(cudaMemcpyAsync(h.report.jtv, L.jtv, sizeof(double) * (it + 1), cudaMemcpyDeviceToHost, st));
    if (it > 0) {
        SRV_CUDA(cudaMemcpyAsync(h.report.cg_rel, L.cg_rel, sizeof(double) * it, cudaMemcpyDeviceToHost, st));
        SRV_CUDA(cudaMemcpyAsync(h.report.cg_done, L.cg_it, sizeof(int) * it, cudaMemcpyDeviceToHost, st));
    }
    SRV_CUDA(cudaMemcpyAsync(&h.status, &L.hdr->status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    SRV_CUDA(cudaEventRecord(r.landed, st));
    r.phase = kFinish;
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
    int least = 0, greatest = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e != cudaSuccess) {
        delete s;
        return fail(MPM_ERR_CUDA, "cudaDeviceGetStreamPriorityRange: %s", cudaGetErrorString(e));
    }
    s->prio_hi = greatest;
    s->n_prio = least - greatest + 1;      // greatest is numerically the smallest
    s->slots.resize((size_t)max_slots * s->n_prio);
    s->slot_owner.assign(max_slots, -1);
    for (size_t k = 0; k < s->slots.size(); ++k) {
        e = cudaStreamCreateWithPriority(&s->slots[k], cudaStreamNonBlocking,
                                         greatest + (int)(k % s->n_prio));
        if (e != cudaSuccess) {
            for (size_t j = 0; j < k; ++j) cudaStreamDestroy(s->slots[j]);
            delete s;
            return fail(MPM_ERR_CUDA, "cudaStreamCreateWithPriority: %s", cudaGetErrorString(e));
        }
    }
    e = cudaHostAlloc((void**)&s->host, sizeof(SlotHost) * max_slots, 0);
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
    if (e != cudaSuccess) return fail(MPM_ERR_CUDA, "event: %s", cudaGetErrorString(e));
    e = cudaEventCreateWithFlags(&r.landed, cudaEventDisableTiming);
    if (e == cudaSuccess) {
        e = cudaEventRecord(r.ready, s->user);
        if (e != cudaSuccess) cudaEventDestroy(r.landed);
    }
    if (e != cudaSuccess) {
        cudaEventDestroy(r.ready);
        return fail(MPM_ERR_CUDA, "event: %s", cudaGetErrorString(e));
    }
    s->reqs[r.ticket] = r;
    s->queue.push_back(r.ticket);
    *ticket = r.ticket;
    return MPM_OK;
}

mpm_status mpm_server_step(mpm_server* s, int* n_active, int* n_queued, int* n_finished)
{
    if (!s) return fail(MPM_ERR_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    int finished = 0;
    // advance every active request whose last enqueued copy has landed
    for (int k = 0; k < s->max_slots; ++k) {
        if (s->slot_owner[k] < 0) continue;
        Request& r = s->reqs[s->slot_owner[k]];
        const cudaError_t q = cudaEventQuery(r.landed);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) return fail(MPM_ERR_CUDA, "cudaEventQuery: %s", cudaGetErrorString(q));
        SlotHost& h = s->host[k];
        if (r.phase == kEval) {
            const double F = h.f[0] + h.f[1];
            bool stop = r.it >= r.opts.gn_iters;
            bool converged = false;
            if (!stop && r.opts.tol_gn > 0.0 && r.it > 0 &&
                std::fabs(r.F_prev - F) < r.opts.tol_gn * std::fabs(r.F_prev)) {
                stop = converged = true;
            }
            mpm_status st;
            if (stop) {
                r.report.iters = r.it;
                r.status = (r.opts.tol_gn > 0.0 && !converged) ? MPM_WARN_NOT_CONVERGED : MPM_OK;
                st = srv_finish(s, r);
            } else {
                r.F_prev = F;
                const FitWs& L = r.L;
                SRV_CUDA(launch_solve(r.P, solve_opts(r.opts), L.h, L.w, L.g, r.y, nullptr,
                                      r.y, nullptr, L.cg_rel + r.it, L.cg_it + r.it, L.solve, L.hdr,
                                      L.red, r.stream));
                r.it += 1;
                st = srv_eval(s, r);
            }
            if (st != MPM_OK) return st;
        } else {                              // kFinish: the report has landed
            const int iters = r.report.iters;
            memcpy(r.report.nll, h.report.nll, sizeof(double) * (iters + 1));
            memcpy(r.report.jtv, h.report.jtv, sizeof(double) * (iters + 1));
            memcpy(r.report.cg_rel, h.report.cg_rel, sizeof(double) * iters);
            memcpy(r.report.cg_done, h.report.cg_done, sizeof(int) * iters);
            for (int i = 0; i <= iters; ++i) r.report.F[i] = r.report.nll[i] + r.report.jtv[i];
            if (h.status) r.status = MPM_ERR_NUMERIC;
            r.state = r.status < 0 ? kFailed : kDone;
            s->slot_owner[k] = -1;
            s->arena.release(r.ws_off, r.ws_bytes);
            cudaEventDestroy(r.ready);
            cudaEventDestroy(r.landed);
            r.slot = -1;
            ++finished;
        }
    }
    // admission into free slots (admit_pick) while the arena has room and the
    // GPU load allows: smallest volume first (ties by arrival); a queued request
    // overtaken by 2 x max_slots later ones is admitted before anything else,
    // so none starves.  A request's load is min(1, N / 2^21): about 2^21
    // voxels keep every kernel of a fit at a full wave, so two such fits side
    // by side only interleave their kernels; requests are admitted while the
    // active load stays <= 1.5 (one large fit and small ones beside it).
    double load = 0.0;
    for (int k = 0; k < s->max_slots; ++k)
        if (s->slot_owner[k] >= 0) load += gpu_load(s->reqs[s->slot_owner[k]].P.N);
    std::vector<Queued> view;
    while (!s->queue.empty()) {
        int k = 0;
        while (k < s->max_slots && s->slot_owner[k] >= 0) ++k;
        if (k == s->max_slots) break;
        view.clear();
        for (int t : s->queue) {
            const Request& c = s->reqs[t];
            view.push_back({c.P.N, c.ws_bytes, c.overtaken});
        }
        size_t off = 0;
        const int pi = admit_pick(view, load, s->max_slots, s->arena, &off);
        if (pi < 0) break;
        auto pick = s->queue.begin() + pi;
        load += gpu_load(s->reqs[*pick].P.N);
        Request& a = s->reqs[*pick];
        for (auto q = s->queue.begin(); q != pick; ++q) s->reqs[*q].overtaken += 1;
        s->queue.erase(pick);
        a.ws_off = off;
        a.L = layout(a.P, MPM_CALL_FIT, s->arena.base + off);
        a.slot = k;
        a.state = kActive;
        a.it = 0;
        s->slot_owner[k] = a.ticket;
        // priority level by size: volumes below 2^19 voxels highest, one level
        // lower per doubling, the rest at the lowest level
        int lv = 0;
        for (size_t n = a.P.N >> 19; n && lv < s->n_prio - 1; n >>= 1) ++lv;
        a.stream = s->slots[(size_t)k * s->n_prio + lv];
        cudaStream_t st = a.stream;
        SRV_CUDA(cudaStreamWaitEvent(st, a.ready, 0));
        SRV_CUDA(cudaMemsetAsync(a.L.hdr, 0, sizeof(WsHeader), st));
        if (a.opts.init) {
            SRV_CUDA(launch_image_means(a.P, a.problem.echo_dtype, a.x, a.L.mean_parts, a.L.means, st));
            SRV_CUDA(launch_init_maps(a.P, a.L.means, a.y, st));
        }
        mpm_status se = srv_eval(s, a);    // records `landed` and enters kEval
        if (se != MPM_OK) return se;
    }
    int active = 0;
    for (int k = 0; k < s->max_slots; ++k) active += s->slot_owner[k] >= 0;
    if (n_active) *n_active = active;
    if (n_queued) *n_queued = (int)s->queue.size();
    if (n_finished) *n_finished = finished;
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

mpm_status mpm_server_release(mpm_server* s, int ticket)
{
    if (!s) return fail(MPM_ERR_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(MPM_ERR_INVALID_ARG, "unknown ticket %d", ticket);
    // a finished request holds no slot, event or arena space any more
    if (it->second.state != kDone && it->second.state != kFailed)
        return fail(MPM_ERR_INVALID_ARG, "ticket %d is not finished", ticket);
    s->reqs.erase(it);
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
            if (kv.second.state == kQueued || kv.second.state == kActive) {
                cudaEventDestroy(kv.second.ready);
                cudaEventDestroy(kv.second.landed);
            }
        cudaFreeHost(s->host);
    }
    delete s;
    return MPM_OK;
}

}  // extern "C"
