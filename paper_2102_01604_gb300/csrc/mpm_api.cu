// mpm_api.cu -- the C ABI declared in include/mpm.h: argument checking,
// workspace layout, constant initial maps and the host loop of the fit.
#include <atomic>
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "init_maps.cuh"
#include "mpm_internal.cuh"

namespace mpm {

static std::atomic<unsigned long long> g_launches{0};

// NVTX range names of the kernel kinds (MPM_KERNEL_*): every launch is
// wrapped in a host-side range of its kind, every Newton update of a fit in
// one named after its index, so profilers can attribute and filter them
// (no cost when no tool is attached).
static const char* const kKindNames[MPM_KERNEL_KINDS] = {
    "grad_hess", "jtv", "pcg_init", "pcg_step", "pcg_final", "uncertainty", "forward", "init",
    "grad_hess_proj", "reslice", "multigrid"};

struct NvtxUpdate {
    explicit NvtxUpdate(int it)
    {
        char name[32];
        snprintf(name, sizeof name, "mpm update %d", it);
        nvtxRangePushA(name);
    }
    ~NvtxUpdate() { nvtxRangePop(); }
};

// ------------------------------------------------- diagnostic kernel timing

struct ProfRecord {
    int kind;
    cudaEvent_t a, b;
};

static std::atomic<bool> g_prof_on{false};
static thread_local bool t_capturing = false;

void LaunchScope::capturing(bool on) { t_capturing = on; }
static std::mutex g_prof_mu;
static std::vector<ProfRecord> g_prof;
static std::vector<cudaEvent_t> g_pool;

static cudaEvent_t pool_get()
{
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

LaunchScope::LaunchScope(int k, cudaStream_t s) : kind(k), st(s), rec(nullptr)
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    nvtxRangePushA(k >= 0 && k < MPM_KERNEL_KINDS ? kKindNames[k] : "mpm kernel");
    if (t_capturing || !g_prof_on.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    ProfRecord r{kind, pool_get(), pool_get()};
    if (!r.a || !r.b) return;
    cudaEventRecord(r.a, st);
    g_prof.push_back(r);
    rec = reinterpret_cast<void*>(g_prof.size());      // 1-based index of the record
}

LaunchScope::~LaunchScope()
{
    nvtxRangePop();
    if (!rec) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    const size_t i = reinterpret_cast<size_t>(rec) - 1;
    if (i < g_prof.size()) cudaEventRecord(g_prof[i].b, st);
}

int voxel_grid(long long N)
{
    const long long cap = 8LL * kNumSm;
    long long g = (N + kBlock - 1) / kBlock;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

static thread_local std::string t_err;

mpm_status fail(mpm_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return s;
}

static bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

static int n_images(const mpm_problem* p)
{
    int I = 0;
    for (int c = 0; c < p->n_contrasts; ++c) I += p->n_echoes[c];
    return I;
}

mpm_status check_problem(const mpm_problem* p)
{
    if (!p) return fail(MPM_ERR_INVALID_ARG, "problem is NULL");
    if (p->nx < 0 || p->ny < 0 || p->nz < 0)
        return fail(MPM_ERR_INVALID_ARG, "negative grid size %d x %d x %d", p->nx, p->ny, p->nz);
    const long long tiles = (long long)((p->nx + kTileX - 1) / kTileX) * ((p->ny + kTileY - 1) / kTileY);
    if (tiles > kMaxBlocks)
        return fail(MPM_ERR_INVALID_ARG, "nx * ny too large (%d x %d)", p->nx, p->ny);
    for (int d = 0; d < 3; ++d)
        if (!finite_pos(p->vx[d])) return fail(MPM_ERR_INVALID_ARG, "voxel size vx[%d] must be > 0", d);
    if (p->n_contrasts < 1 || p->n_contrasts > MPM_MAX_CONTRASTS)
        return fail(MPM_ERR_INVALID_ARG, "n_contrasts = %d outside [1, %d]", p->n_contrasts,
                    MPM_MAX_CONTRASTS);
    int I = 0, any_mt = 0;
    for (int c = 0; c < p->n_contrasts; ++c) {
        if (p->n_echoes[c] < 1) return fail(MPM_ERR_INVALID_ARG, "n_echoes[%d] < 1", c);
        I += p->n_echoes[c];
        if (I > MPM_MAX_IMAGES)
            return fail(MPM_ERR_INVALID_ARG, "more than %d images", MPM_MAX_IMAGES);
        if (!(p->alpha[c] > 0.0 && p->alpha[c] < M_PI))
            return fail(MPM_ERR_INVALID_ARG, "alpha[%d] must be in (0, pi)", c);
        if (!finite_pos(p->tr[c])) return fail(MPM_ERR_INVALID_ARG, "tr[%d] must be > 0", c);
        if (!finite_pos(p->sigma2[c])) return fail(MPM_ERR_INVALID_ARG, "sigma2[%d] must be > 0", c);
        if (p->mt[c] != 0 && p->mt[c] != 1) return fail(MPM_ERR_INVALID_ARG, "mt[%d] must be 0 or 1", c);
        any_mt |= p->mt[c];
    }
    for (int i = 0; i < I; ++i)
        if (!(std::isfinite(p->te[i]) && p->te[i] >= 0.0))
            return fail(MPM_ERR_INVALID_ARG, "te[%d] must be >= 0", i);
    const int K = any_mt ? 4 : 3;
    if (p->n_maps != K)
        return fail(MPM_ERR_INVALID_ARG, "n_maps = %d but must be %d (%s MT contrast)", p->n_maps,
                    K, any_mt ? "with an" : "without");
    for (int k = 0; k < K; ++k)
        if (!(std::isfinite(p->lambda[k]) && p->lambda[k] >= 0.0))
            return fail(MPM_ERR_INVALID_ARG, "lambda[%d] must be >= 0", k);
    if (!finite_pos(p->eps)) return fail(MPM_ERR_INVALID_ARG, "eps must be > 0");
    if (p->precond < 0 || p->precond > 2) return fail(MPM_ERR_INVALID_ARG, "precond must be 0, 1 or 2");
    if (p->echo_dtype != 0 && p->echo_dtype != 1)
        return fail(MPM_ERR_INVALID_ARG, "echo_dtype must be 0 (float32) or 1 (bfloat16)");
    return MPM_OK;
}

mpm_status check_opts(const mpm_opts* o)
{
    if (!o) return fail(MPM_ERR_INVALID_ARG, "opts is NULL");
    if (o->gn_iters < 0 || o->gn_iters > MPM_MAX_REPORT)
        return fail(MPM_ERR_INVALID_ARG, "gn_iters = %d outside [0, %d]", o->gn_iters, MPM_MAX_REPORT);
    if (o->cg_iters < 1 || o->cg_iters > 1000000)
        return fail(MPM_ERR_INVALID_ARG, "cg_iters = %d outside [1, 1e6]", o->cg_iters);
    if (o->newton_per_irls < 1) return fail(MPM_ERR_INVALID_ARG, "newton_per_irls must be >= 1");
    if (o->init != 0 && o->init != 1) return fail(MPM_ERR_INVALID_ARG, "init must be 0 or 1");
    if (o->graph < 0 || o->graph > 2) return fail(MPM_ERR_INVALID_ARG, "graph must be 0, 1 or 2");
    if (!(std::isfinite(o->tol_gn) && o->tol_gn >= 0.0) || !(std::isfinite(o->tol_cg) && o->tol_cg >= 0.0))
        return fail(MPM_ERR_INVALID_ARG, "tolerances must be finite and >= 0");
    if (o->mg_levels < 0 || o->mg_levels > 16)
        return fail(MPM_ERR_INVALID_ARG, "mg_levels = %d outside [0, 16]", o->mg_levels);
    if (o->mg_nu < 0 || o->mg_nu > 8) return fail(MPM_ERR_INVALID_ARG, "mg_nu = %d outside [0, 8]", o->mg_nu);
    if (!(std::isfinite(o->mg_omega) && o->mg_omega >= 0.0 && o->mg_omega < 2.0))
        return fail(MPM_ERR_INVALID_ARG, "mg_omega must be in [0, 2)");
    if (o->mg_coarse_sweeps < 0 || o->mg_coarse_sweeps > 1000)
        return fail(MPM_ERR_INVALID_ARG, "mg_coarse_sweeps = %d outside [0, 1000]", o->mg_coarse_sweeps);
    return MPM_OK;
}

DevProblem make_dev(const mpm_problem* p)
{
    DevProblem P;
    memset(&P, 0, sizeof P);
    P.nx = p->nx;
    P.ny = p->ny;
    P.nz = p->nz;
    P.N = (long long)p->nx * p->ny * p->nz;
    P.ihx2 = (float)(1.0 / (p->vx[0] * p->vx[0]));
    P.ihy2 = (float)(1.0 / (p->vx[1] * p->vx[1]));
    P.ihz2 = (float)(1.0 / (p->vx[2] * p->vx[2]));
    P.C = p->n_contrasts;
    P.K = p->n_maps;
    P.T = P.K * (P.K + 1) / 2;
    int i = 0;
    for (int c = 0; c < P.C; ++c) {
        P.n_echoes[c] = p->n_echoes[c];
        P.echo0[c] = i;
        P.alpha[c] = (float)p->alpha[c];
        P.tr[c] = (float)p->tr[c];
        P.isig2[c] = (float)(1.0 / p->sigma2[c]);
        P.mt[c] = p->mt[c];
        i += p->n_echoes[c];
    }
    P.I = i;
    for (int j = 0; j < i; ++j) P.te[j] = (float)p->te[j];
    for (int c = 0; c < P.C; ++c) {
        const int E = P.n_echoes[c], i0 = P.echo0[c];
        const double t0 = p->te[i0];
        const double dt = E > 1 ? (p->te[i0 + E - 1] - t0) / (E - 1) : 0.0;
        bool uni = true;
        for (int e = 0; e < E; ++e)
            if (std::fabs(p->te[i0 + e] - (t0 + e * dt)) > 1e-7 * std::fabs(p->te[i0 + E - 1]) + 1e-12)
                uni = false;
        P.te_uniform[c] = uni ? 1 : 0;
        P.dte[c] = (float)dt;
        P.same_tr[c] = (c > 0 && p->tr[c] == p->tr[c - 1]) ? 1 : 0;
    }
    P.flip_as_c0 = P.echoes_as_prev = 0u;
    for (int c = 1; c < P.C; ++c) {
        if (P.alpha[c] == P.alpha[0]) P.flip_as_c0 |= 1u << c;
        if (P.te_uniform[c] && P.te_uniform[c - 1] && P.te[P.echo0[c]] == P.te[P.echo0[c - 1]] &&
            P.dte[c] == P.dte[c - 1])
            P.echoes_as_prev |= 1u << c;
    }
    for (int k = 0; k < 4; ++k) P.lambda[k] = (float)p->lambda[k];
    P.eps2 = (float)(p->eps * p->eps);
    P.precond = p->precond;
    return P;
}

// Device (or managed) memory check: a host pointer handed to a kernel would
// fault, so it is refused here.
mpm_status check_dev(const void* ptr, const char* name, bool optional, size_t align)
{
    if (!ptr) {
        if (optional) return MPM_OK;
        return fail(MPM_ERR_INVALID_ARG, "%s is NULL", name);
    }
    if (reinterpret_cast<uintptr_t>(ptr) % align)
        return fail(MPM_ERR_INVALID_ARG, "%s is not %zu-byte aligned", name, align);
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(MPM_ERR_INVALID_ARG, "%s: not a CUDA pointer (%s)", name, cudaGetErrorString(e));
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return fail(MPM_ERR_INVALID_ARG, "%s is not device memory", name);
    return MPM_OK;
}

// ----------------------------------------------------------- workspace

static size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

constexpr int kMeanBlocksHost = 304;   // must match the launcher's cap

FitWs layout(const DevProblem& P, int call, void* base)
{
    FitWs L;
    memset(&L, 0, sizeof L);
    size_t off = 0;
    char* b = static_cast<char*>(base);
    auto take = [&](size_t bytes) -> char* {
        char* p = b ? b + off : nullptr;
        off += al(bytes);
        return p;
    };
    L.hdr = reinterpret_cast<WsHeader*>(take(kHeaderBytes));
    L.red.partials = reinterpret_cast<double*>(take(kPartialBytes));
    L.red.counter = L.hdr ? &L.hdr->counter : nullptr;
    const size_t vec = sizeof(float) * (size_t)P.K * P.N;
    if (call == MPM_CALL_FIT) {
        L.mean_parts = reinterpret_cast<double*>(take(sizeof(double) * P.I * kMeanBlocksHost));
        L.means = reinterpret_cast<double*>(take(sizeof(double) * MPM_MAX_IMAGES));
        L.nll = reinterpret_cast<double*>(take(sizeof(double) * (MPM_MAX_REPORT + 2)));
        L.jtv = reinterpret_cast<double*>(take(sizeof(double) * (MPM_MAX_REPORT + 2)));
        L.cg_rel = reinterpret_cast<double*>(take(sizeof(double) * MPM_MAX_REPORT));
        L.cg_it = reinterpret_cast<int*>(take(sizeof(int) * MPM_MAX_REPORT));
        L.w = reinterpret_cast<float*>(take(sizeof(float) * (size_t)P.N));
        L.g = reinterpret_cast<float*>(take(vec));
        L.h = reinterpret_cast<float*>(take(sizeof(float) * (size_t)P.T * P.N));
    }
    if (call == MPM_CALL_FIT || call == MPM_CALL_SOLVE) L.solve = take(solve_ws_bytes(P));
    L.total = off;
    return L;
}

mpm_status check_ws(const DevProblem& P, int call, void* ws, size_t ws_bytes, FitWs& L)
{
    const size_t need = layout(P, call, nullptr).total;
    if (ws_bytes < need)
        return fail(MPM_ERR_WORKSPACE_TOO_SMALL, "workspace of %zu bytes, %zu needed", ws_bytes, need);
    MPM_TRY(check_dev(ws, "ws", false, 256));
    L = layout(P, call, ws);
    return MPM_OK;
}

// ------------------------------------------------------ initial maps

// ------------------------------------------------------------------ fits

// One subject's fit: arguments checked, workspace carved.
struct FitJob {
    const mpm_problem* problem;
    mpm_opts opts;
    DevProblem P;
    const void* x;
    const float *b1p, *b1m;
    float *y, *var;
    void* ws;
    size_t ws_bytes;
    FitWs L;
    bool empty;
    bool proj;        // spatial projection (mpm_fit_proj): pj holds it
    ProjJob pj;
};

// The likelihood pieces of update `it`: the fused voxel pass, or its
// projected form (per-contrast passes on the acquisition grids and the push).
static cudaError_t launch_lik(const FitJob& j, int it, cudaStream_t st)
{
    const FitWs& L = j.L;
    if (j.proj) return launch_grad_hess_proj(j.P, j.pj, j.y, L.g, L.h, L.nll + it, L.red, st);
    return launch_grad_hess(j.P, j.problem->echo_dtype, j.x, j.y, j.b1p, j.b1m, L.g, L.h,
                            L.nll + it, L.red, &L.hdr->status, st);
}

static mpm_status fit_prepare(const mpm_problem* problem, const mpm_opts* opts, const void* x,
                              const float* b1p, const float* b1m, float* y, float* var_out,
                              void* ws, size_t ws_bytes, FitJob& job)
{
    MPM_TRY(check_problem(problem));
    MPM_TRY(check_opts(opts));
    job.problem = problem;
    job.opts = *opts;
    job.P = make_dev(problem);
    job.x = x;
    job.b1p = b1p;
    job.b1m = b1m;
    job.y = y;
    job.var = var_out;
    job.ws = ws;
    job.ws_bytes = ws_bytes;
    job.empty = job.P.N == 0;
    job.proj = false;
    if (job.empty) return MPM_OK;
    MPM_TRY(check_dev(x, "x", false, problem->echo_dtype ? 2 : 4));
    MPM_TRY(check_dev(b1p, "b1p", true, 4));
    MPM_TRY(check_dev(b1m, "b1m", true, 4));
    MPM_TRY(check_dev(y, "y_inout", false, 4));
    MPM_TRY(check_dev(var_out, "var_out", true, 4));
    MPM_TRY(check_ws(job.P, MPM_CALL_FIT, ws, ws_bytes, job.L));
    return MPM_OK;
}

// The updates of a fit whose schedule needs no host decision (tol_gn = 0):
// every launch of every update, the final evaluation and the uncertainty.
// Enqueued on `st`; nothing here synchronises, so it can be captured.
static cudaError_t fit_enqueue_updates(const FitJob& j, cudaStream_t st, int* iters_out)
{
    const DevProblem& P = j.P;
    const FitWs& L = j.L;
    const int npi = j.opts.newton_per_irls;
    bool w_fresh = false;
    cudaError_t e = cudaSuccess;
    int it = 0;
    for (;; ++it) {
        NvtxUpdate range(it);
        w_fresh = (it % npi == 0);
        if ((e = launch_jtv(P, j.y, w_fresh ? L.w : nullptr, L.jtv + it, L.red, st))) return e;
        if ((e = launch_lik(j, it, st))) return e;
        if (it >= j.opts.gn_iters) break;
        if ((e = launch_solve(P, solve_opts(j.opts), L.h, L.w, L.g, j.y, nullptr, j.y,
                              nullptr, L.cg_rel + it, L.cg_it + it, L.solve, L.hdr, L.red, st)))
            return e;
    }
    if (j.var) {
        if (!w_fresh && (e = launch_jtv(P, j.y, L.w, L.jtv + MPM_MAX_REPORT + 1, L.red, st))) return e;
        if ((e = launch_uncertainty(P, L.h, L.w, j.y, j.var, nullptr, nullptr, &L.hdr->status, st)))
            return e;
    }
    *iters_out = it;
    return e;
}

// Same with the host-side stopping test on the objective (tol_gn > 0).
static mpm_status fit_run_adaptive(const FitJob& j, cudaStream_t st, int* iters_out, bool* converged)
{
    const DevProblem& P = j.P;
    const FitWs& L = j.L;
    const int npi = j.opts.newton_per_irls;
    bool w_fresh = false;
    double F_prev = 0.0;
    int it = 0;
    *converged = false;
    for (;; ++it) {
        NvtxUpdate range(it);
        w_fresh = (it % npi == 0);
        MPM_CUDA(launch_jtv(P, j.y, w_fresh ? L.w : nullptr, L.jtv + it, L.red, st));
        MPM_CUDA(launch_lik(j, it, st));
        if (it >= j.opts.gn_iters) break;
        double v[2];
        MPM_CUDA(cudaMemcpyAsync(&v[0], L.nll + it, sizeof(double), cudaMemcpyDeviceToHost, st));
        MPM_CUDA(cudaMemcpyAsync(&v[1], L.jtv + it, sizeof(double), cudaMemcpyDeviceToHost, st));
        MPM_CUDA(cudaStreamSynchronize(st));
        const double F = v[0] + v[1];
        if (it > 0 && std::fabs(F_prev - F) < j.opts.tol_gn * std::fabs(F_prev)) {
            *converged = true;
            break;
        }
        F_prev = F;
        MPM_CUDA(launch_solve(P, solve_opts(j.opts), L.h, L.w, L.g, j.y, nullptr, j.y,
                              nullptr, L.cg_rel + it, L.cg_it + it, L.solve, L.hdr, L.red, st));
    }
    if (j.var) {
        if (!w_fresh) MPM_CUDA(launch_jtv(P, j.y, L.w, L.jtv + MPM_MAX_REPORT + 1, L.red, st));
        MPM_CUDA(launch_uncertainty(P, L.h, L.w, j.y, j.var, nullptr, nullptr, &L.hdr->status, st));
    }
    *iters_out = it;
    return MPM_OK;
}

// ------------------------------------------------------- graph capture

// Private streams used to capture graphs (created once, never destroyed).
static std::mutex g_stream_mu;
static std::vector<cudaStream_t> g_streams;

static cudaError_t private_streams(int n, std::vector<cudaStream_t>& out)
{
    std::lock_guard<std::mutex> lk(g_stream_mu);
    while ((int)g_streams.size() < n) {
        cudaStream_t s;
        cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
        g_streams.push_back(s);
    }
    out.assign(g_streams.begin(), g_streams.begin() + n);
    return cudaSuccess;
}

// Instantiated graphs keyed by everything the captured launches depend on.
struct GraphEntry {
    std::string key;
    cudaGraphExec_t exec;
    std::vector<int> iters;
    unsigned long long kernels;   // kernel launches captured (counted again on every replay)
};
static std::mutex g_graph_mu;
static std::vector<GraphEntry> g_graphs;      // most recent last
constexpr size_t kGraphCacheSize = 8;

static std::string graph_key(const FitJob* jobs, int n)
{
    int dev = -1;
    cudaGetDevice(&dev);
    std::string k(reinterpret_cast<const char*>(&dev), sizeof dev);
    for (int i = 0; i < n; ++i) {
        const FitJob& j = jobs[i];
        // The kernels' view of the problem (make_dev zero-fills it before
        // setting its fields, so entries past n_contrasts or the image count
        // do not split the cache as the caller's struct could), the echo
        // type, the schedule field by field (mpm_opts has tail padding), and
        // every pointer the launches use.
        k.append(reinterpret_cast<const char*>(&j.P), sizeof(DevProblem));
        const long long sched[9] = {j.problem->echo_dtype, j.opts.gn_iters, j.opts.cg_iters,
                                    j.opts.newton_per_irls, j.opts.init, j.opts.graph,
                                    j.opts.mg_levels, j.opts.mg_nu, j.opts.mg_coarse_sweeps};
        const double tols[3] = {j.opts.tol_gn, j.opts.tol_cg, j.opts.mg_omega};
        k.append(reinterpret_cast<const char*>(sched), sizeof sched);
        k.append(reinterpret_cast<const char*>(tols), sizeof tols);
        const void* ptrs[7] = {j.x, j.b1p, j.b1m, j.y, j.var, j.ws, (const void*)j.ws_bytes};
        k.append(reinterpret_cast<const char*>(ptrs), sizeof ptrs);
        k.push_back(j.proj ? 1 : 0);
        if (j.proj) proj_key(j.pj, k);
    }
    return k;
}

// Capture `nlanes` chains of launches as parallel branches of one graph:
// enqueue(l, stream) puts lane l's launches on its stream.
template <class Enqueue>
static mpm_status capture_lanes(size_t nlanes, Enqueue enqueue, GraphEntry& out)
{
    MPM_CUDA(prime_tma_kernels());
    std::vector<cudaStream_t> ss;
    MPM_CUDA(private_streams((int)nlanes + 1, ss));
    cudaStream_t root = ss[0];
    cudaGraph_t graph = nullptr;
    std::vector<cudaEvent_t> evs;
    cudaEvent_t fork;
    MPM_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    evs.push_back(fork);
    LaunchScope::capturing(true);
    const unsigned long long before = g_launches.load();
    cudaError_t e = cudaStreamBeginCapture(root, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaEventRecord(fork, root);
    for (size_t l = 0; l < nlanes && e == cudaSuccess; ++l) {
        cudaStream_t b = ss[1 + l];
        e = cudaStreamWaitEvent(b, fork, 0);
        if (e == cudaSuccess) e = enqueue(l, b);
        cudaEvent_t join;
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
        if (e == cudaSuccess) {
            evs.push_back(join);
            e = cudaEventRecord(join, b);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(root, join, 0);
        }
    }
    cudaError_t e2 = cudaStreamEndCapture(root, &graph);
    LaunchScope::capturing(false);
    // launches made while capturing are not executed: count them at each replay
    out.kernels = g_launches.load() - before;
    g_launches.fetch_sub(out.kernels);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&out.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(MPM_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
    }
    return MPM_OK;
}

// Capture the updates of every job as parallel branches of one graph.
static mpm_status capture_updates(FitJob* jobs, int n, GraphEntry& out)
{
    // Lanes of the graph, each a chain of subjects on one stream, all lanes
    // side by side (lane_plan).  Subjects that fill the GPU on their own run
    // in one lane: side by side, two such fits only interleave their one-wave
    // kernels.
    std::vector<long long> voxels(n);
    std::vector<char> empty(n);
    for (int i = 0; i < n; ++i) {
        voxels[i] = jobs[i].P.N;
        empty[i] = jobs[i].empty ? 1 : 0;
    }
    const std::vector<std::vector<int>> lanes = lane_plan(voxels, empty);
    out.iters.assign(n, 0);
    return capture_lanes(
        lanes.size(),
        [&](size_t l, cudaStream_t b) {
            cudaError_t e = cudaSuccess;
            for (size_t k = 0; k < lanes[l].size() && e == cudaSuccess; ++k)
                e = fit_enqueue_updates(jobs[lanes[l][k]], b, &out.iters[lanes[l][k]]);
            return e;
        },
        out);
}

// ------------------------------------------- phase-batched graph (graph = 2)

// One subject of a phase-batched fit: its grids and the TMA maps of its solve.
struct PhasedSubject {
    FitJob* j;
    StencilGrid sg;          // 32 x 8 stencil grid of the JTV kernel
    StencilGrid ig;          // and of the PCG start
    SolveBufs B;
    StepMaps maps;
    int nchunk;              // z ranges of its share of the iteration's wave
    unsigned step_blocks;    // that share
    unsigned vox_blocks;     // grid of the per-voxel kernels
};

// Batch classes: subjects that share every template parameter of the kernels
// (map count, Hessian loading, echo storage, tile shape of the iteration).
static long long phased_class(const FitJob& j, int tile)
{
    return ((j.P.K * 10LL + j.P.precond) * 10 + j.problem->echo_dtype) * 10 + tile;
}

// Every launch of the fits of one group (at most kBatchMax subjects of one
// class), each phase of each update as one launch for the whole group.  Enqueued on `st`; nothing
// here synchronises, so it can be captured.
static cudaError_t enqueue_phased(std::vector<PhasedSubject>& subj, int tile, cudaStream_t st,
                                  std::vector<int>& iters, const std::vector<int>& index)
{
    const int n = (int)subj.size();
    const FitJob& j0 = *subj[0].j;
    const mpm_opts& o = j0.opts;          // one schedule for the whole batch
    const int K = j0.P.K, pre = j0.P.precond, dtype = j0.problem->echo_dtype;
    const int npi = o.newton_per_irls;
    const double tol2 = o.tol_cg > 0.0 ? o.tol_cg * o.tol_cg : 0.0;
    std::vector<JtvArgs> ja(n);
    std::vector<GradArgs> ga(n);
    std::vector<InitArgs> ia(n);
    std::vector<StepArgs> sa(n);
    std::vector<FinalArgs> fa(n);
    std::vector<UncArgs> ua;
    std::vector<unsigned> bst(n), bini(n), bvox(n), bstep(n);
    for (int s = 0; s < n; ++s) {
        const StencilGrid& g = subj[s].sg;
        bst[s] = g.grid.x * g.grid.y * g.grid.z;
        const StencilGrid& gi = subj[s].ig;
        bini[s] = gi.grid.x * gi.grid.y * gi.grid.z;
        bvox[s] = subj[s].vox_blocks;
        bstep[s] = subj[s].step_blocks;
    }
    auto jtv = [&](bool fresh, int slot) {
        for (int s = 0; s < n; ++s) {
            const FitJob& j = *subj[s].j;
            const StencilGrid& g = subj[s].sg;
            ja[s] = JtvArgs{j.P, g.zc, g.grid.x, g.grid.y, g.grid.z, j.y, fresh ? j.L.w : nullptr,
                            j.L.jtv + slot, j.L.red};
        }
        return launch_jtv_batch(K, ja.data(), bst.data(), n, st);
    };
    cudaError_t e = cudaSuccess;
    bool w_fresh = false;
    int it = 0;
    for (;; ++it) {
        NvtxUpdate range(it);
        w_fresh = (it % npi == 0);
        if ((e = jtv(w_fresh, it))) return e;
        for (int s = 0; s < n; ++s) {
            const FitJob& j = *subj[s].j;
            ga[s] = GradArgs{j.P, j.x, j.y, j.b1p, j.b1m, j.L.g, j.L.h, j.L.nll + it, j.L.red,
                             &j.L.hdr->status};
        }
        if ((e = launch_grad_hess_batch(K, pre, dtype, ga.data(), bvox.data(), n, st))) return e;
        if (it >= o.gn_iters) break;
        for (int s = 0; s < n; ++s) {
            const FitJob& j = *subj[s].j;
            const StencilGrid& g = subj[s].ig;
            ia[s] = InitArgs{j.P, g.zc, g.grid.x, g.grid.y, g.grid.z, j.L.h, j.L.w, j.L.g, j.y,
                             subj[s].B.z[0], tol2, j.L.hdr, nullptr, j.L.red};
        }
        if ((e = launch_pcg_init_batch(K, ia.data(), bini.data(), n, st))) return e;
        for (int c = 0; c < o.cg_iters; ++c) {
            const int rr = (tol2 > 0.0 || c == o.cg_iters - 1) ? 1 : 0;
            for (int s = 0; s < n; ++s) {
                const FitJob& j = *subj[s].j;
                sa[s] = step_args(j.P, subj[s].maps, subj[s].nchunk, c, rr, j.L.hdr, nullptr, j.L.red);
            }
            if ((e = launch_step_batch(K, tile, step_mode(c), sa.data(), bstep.data(), n, st))) return e;
        }
        for (int s = 0; s < n; ++s) {
            const FitJob& j = *subj[s].j;
            fa[s] = FinalArgs{j.P.N, subj[s].B, nullptr, j.y, j.L.hdr, j.L.cg_rel + it, j.L.cg_it + it};
        }
        if ((e = launch_pcg_final_batch(K, fa.data(), bvox.data(), n, st))) return e;
    }
    // the posterior variance of the subjects that ask for it
    std::vector<JtvArgs> jv;
    std::vector<unsigned> bjv, buv;
    ua.clear();
    for (int s = 0; s < n; ++s) {
        const FitJob& j = *subj[s].j;
        if (!j.var) continue;
        const StencilGrid& g = subj[s].sg;
        jv.push_back(JtvArgs{j.P, g.zc, g.grid.x, g.grid.y, g.grid.z, j.y, j.L.w,
                             j.L.jtv + MPM_MAX_REPORT + 1, j.L.red});
        bjv.push_back(bst[s]);
        ua.push_back(UncArgs{j.P, j.L.h, j.L.w, j.y, j.var, nullptr, nullptr, &j.L.hdr->status});
        buv.push_back(bvox[s]);
    }
    if (!ua.empty()) {
        const int m = (int)ua.size();
        if (!w_fresh && (e = launch_jtv_batch(K, jv.data(), bjv.data(), m, st))) return e;
        if ((e = launch_uncertainty_batch(K, ua.data(), buv.data(), m, st))) return e;
    }
    for (int s = 0; s < n; ++s) iters[index[s]] = it;
    return e;
}

// The groups of a phase-batched graph: each batch class split into groups of
// at most kBatchMax subjects that share the GPU's wave of the iteration kernel
// (share_wave: the shares that let the launch end soonest).  A subject takes its solo fit's tile shape;
// one that cannot take part (projection, multigrid, a volume or buffer the
// TMA-staged iteration cannot take) is marked in `rest` and runs in a lane of
// its own kind (capture_updates' lanes) beside the groups.
static void plan_phased(FitJob* jobs, int n, std::vector<std::vector<PhasedSubject>>& groups,
                        std::vector<int>& tiles, std::vector<std::vector<int>>& index,
                        std::vector<char>& rest)
{
    std::map<long long, std::vector<PhasedSubject>> classes;
    std::map<long long, int> class_tile;
    rest.assign(n, 0);
    for (int i = 0; i < n; ++i) {
        FitJob& j = jobs[i];
        if (j.empty) continue;
        rest[i] = 1;
        if (j.proj || j.opts.mg_levels > 0) continue;
        const int tile = tma_tile_choice(j.P);
        PhasedSubject ps;
        ps.j = &j;
        ps.B = solve_bufs(j.P, j.L.solve);
        if (!make_step_maps(j.P, j.L.h, j.L.w, ps.B, tile, &ps.maps)) continue;

        rest[i] = 0;
        const long long key = phased_class(j, tile);
        classes[key].push_back(ps);
        class_tile[key] = tile;
    }
    for (auto& kv : classes) {
        std::vector<PhasedSubject>& members = kv.second;
        const int tile = class_tile[kv.first];
        for (size_t g0 = 0; g0 < members.size(); g0 += kBatchMax) {
            const size_t g1 = std::min(members.size(), g0 + (size_t)kBatchMax);
            std::vector<PhasedSubject> grp(members.begin() + g0, members.begin() + g1);
            std::vector<int> idx;
            // the stencil kernels' blocks shared in proportion to the voxels
            long long vox = 0;
            for (const PhasedSubject& ps : grp) vox += ps.j->P.N;
            for (PhasedSubject& ps : grp) {
                const double share = (double)ps.j->P.N / (double)vox;
                ps.sg = stencil_grid(ps.j->P, kTileX, kTileY, 2, share);
                ps.ig = stencil_grid(ps.j->P, kTileX, kTileY, kInitWaves, share);
                const long long cap = std::max(1LL, std::llround(share * voxel_grid(1LL << 40)));
                ps.vox_blocks = (unsigned)std::min<long long>(voxel_grid(ps.j->P.N), cap);
            }
            std::vector<long long> t, blocks;
            std::vector<int> nz, chunks;
            for (const PhasedSubject& ps : grp) {
                t.push_back(tma_tiles_of(ps.j->P, tile));
                nz.push_back(ps.j->P.nz);
            }
            share_wave(t, nz, tma_wave_blocks(grp[0].j->P, tile), blocks, chunks);
            for (size_t k = 0; k < grp.size(); ++k) {
                grp[k].nchunk = chunks[k];
                grp[k].step_blocks = (unsigned)blocks[k];
                idx.push_back((int)(grp[k].j - jobs));
            }
            groups.push_back(grp);
            tiles.push_back(tile);
            index.push_back(idx);
        }
    }
}

// Capture the updates of every job phase by phase: one launch per phase of
// every update for each group of plan_phased, the groups in lanes, and beside
// them the lanes of the subjects that cannot be batched.
static mpm_status capture_phased(FitJob* jobs, int n, GraphEntry& out)
{
    std::vector<std::vector<PhasedSubject>> groups;
    std::vector<int> tiles;
    std::vector<std::vector<int>> index;
    std::vector<char> rest;
    plan_phased(jobs, n, groups, tiles, index, rest);
    if (groups.empty()) return capture_updates(jobs, n, out);
    std::vector<long long> voxels(n);
    std::vector<char> skip(n);
    for (int i = 0; i < n; ++i) {
        voxels[i] = jobs[i].P.N;
        skip[i] = rest[i] ? 0 : 1;
    }
    const std::vector<std::vector<int>> lanes = lane_plan(voxels, skip);
    out.iters.assign(n, 0);
    // The groups are placed in lanes by the same rule as single subjects
    // (lane_plan on their voxel totals): groups that fill the GPU run one
    // after another, each of their launches sized for the whole GPU; smaller
    // groups run side by side.
    std::vector<long long> gvox(groups.size(), 0);
    for (size_t g = 0; g < groups.size(); ++g)
        for (const PhasedSubject& ps : groups[g]) gvox[g] += ps.j->P.N;
    const std::vector<std::vector<int>> glanes = lane_plan(gvox, std::vector<char>(groups.size(), 0));
    return capture_lanes(
        glanes.size() + lanes.size(),
        [&](size_t l, cudaStream_t b) {
            cudaError_t e = cudaSuccess;
            if (l < glanes.size()) {
                for (size_t k = 0; k < glanes[l].size() && e == cudaSuccess; ++k) {
                    const int g = glanes[l][k];
                    e = enqueue_phased(groups[g], tiles[g], b, out.iters, index[g]);
                }
                return e;
            }
            const std::vector<int>& lane = lanes[l - glanes.size()];
            for (size_t k = 0; k < lane.size() && e == cudaSuccess; ++k)
                e = fit_enqueue_updates(jobs[lane[k]], b, &out.iters[lane[k]]);
            return e;
        },
        out);
}

// Initial maps (image means and the constant maps, on the device), then the
// updates -- as one graph launch when the schedule is fixed and opts.graph is
// set, else as direct launches -- then one read-back of every report.
static mpm_status fit_run(FitJob* jobs, int n, mpm_report* reports, cudaStream_t st)
{
    for (int i = 0; i < n; ++i)
        if (reports) memset(&reports[i], 0, sizeof(mpm_report));
    // clear status words and counters; image means and, from them, the
    // constant starting maps, all on the device (no host round trip)
    for (int i = 0; i < n; ++i) {
        FitJob& j = jobs[i];
        if (j.empty) continue;
        MPM_CUDA(cudaMemsetAsync(j.L.hdr, 0, sizeof(WsHeader), st));
        if (j.opts.init) {
            if (j.proj)
                MPM_CUDA(proj_image_means(j.P, j.pj, j.L.mean_parts, j.L.means, st));
            else
                MPM_CUDA(launch_image_means(j.P, j.problem->echo_dtype, j.x, j.L.mean_parts, j.L.means, st));
            MPM_CUDA(launch_init_maps(j.P, j.L.means, j.y, st));
        }
    }

    std::vector<int> iters(n, 0);
    std::vector<char> converged(n, 0);
    const bool fixed = jobs[0].opts.tol_gn == 0.0;
    if (fixed && jobs[0].opts.graph) {
        const std::string key = graph_key(jobs, n);
        cudaGraphExec_t exec = nullptr;
        unsigned long long kernels = 0;
        {
            std::lock_guard<std::mutex> lk(g_graph_mu);
            for (size_t g = 0; g < g_graphs.size(); ++g)
                if (g_graphs[g].key == key) {
                    GraphEntry hit = g_graphs[g];
                    g_graphs.erase(g_graphs.begin() + g);
                    g_graphs.push_back(hit);
                    exec = hit.exec;
                    iters = hit.iters;
                    kernels = hit.kernels;
                    break;
                }
        }
        if (!exec) {
            GraphEntry ge;
            ge.key = key;
            if (jobs[0].opts.graph == 2)
                MPM_TRY(capture_phased(jobs, n, ge));
            else
                MPM_TRY(capture_updates(jobs, n, ge));
            exec = ge.exec;
            iters = ge.iters;
            kernels = ge.kernels;
            std::lock_guard<std::mutex> lk(g_graph_mu);
            g_graphs.push_back(ge);
            if (g_graphs.size() > kGraphCacheSize) {
                cudaGraphExecDestroy(g_graphs.front().exec);
                g_graphs.erase(g_graphs.begin());
            }
        }
        MPM_CUDA(cudaGraphLaunch(exec, st));
        g_launches.fetch_add(kernels);
    } else if (fixed) {
        for (int i = 0; i < n; ++i)
            if (!jobs[i].empty) MPM_CUDA(fit_enqueue_updates(jobs[i], st, &iters[i]));
    } else {
        for (int i = 0; i < n; ++i) {
            if (jobs[i].empty) continue;
            bool c = false;
            MPM_TRY(fit_run_adaptive(jobs[i], st, &iters[i], &c));
            converged[i] = c;
        }
    }

    // read back every report with one synchronisation
    struct Back {
        double nll[MPM_MAX_REPORT + 1], jtv[MPM_MAX_REPORT + 1], cgr[MPM_MAX_REPORT];
        int cgi[MPM_MAX_REPORT];
        unsigned status;
    };
    std::vector<Back> back(n);
    for (int i = 0; i < n; ++i) {
        const FitJob& j = jobs[i];
        if (j.empty) continue;
        const int it = iters[i];
        MPM_CUDA(cudaMemcpyAsync(back[i].nll, j.L.nll, sizeof(double) * (it + 1), cudaMemcpyDeviceToHost, st));
        MPM_CUDA(cudaMemcpyAsync(back[i].jtv, j.L.jtv, sizeof(double) * (it + 1), cudaMemcpyDeviceToHost, st));
        if (it > 0) {
            MPM_CUDA(cudaMemcpyAsync(back[i].cgr, j.L.cg_rel, sizeof(double) * it, cudaMemcpyDeviceToHost, st));
            MPM_CUDA(cudaMemcpyAsync(back[i].cgi, j.L.cg_it, sizeof(int) * it, cudaMemcpyDeviceToHost, st));
        }
        MPM_CUDA(cudaMemcpyAsync(&back[i].status, &j.L.hdr->status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    }
    MPM_CUDA(cudaStreamSynchronize(st));
    mpm_status result = MPM_OK;
    for (int i = 0; i < n; ++i) {
        const FitJob& j = jobs[i];
        if (j.empty) continue;
        const int it = iters[i];
        if (reports) {
            mpm_report& r = reports[i];
            r.iters = it;
            for (int k = 0; k <= it; ++k) {
                r.nll[k] = back[i].nll[k];
                r.jtv[k] = back[i].jtv[k];
                r.F[k] = back[i].nll[k] + back[i].jtv[k];
            }
            for (int k = 0; k < it; ++k) {
                r.cg_rel[k] = back[i].cgr[k];
                r.cg_done[k] = back[i].cgi[k];
            }
        }
        const unsigned status = back[i].status;
        if (status && result >= 0)
            result = fail(MPM_ERR_NUMERIC, "%sdevice status 0x%x (%s%s%s)",
                          n > 1 ? "a subject reported " : "", status,
                          status & kStatusNotPD ? "non positive definite block " : "",
                          status & kStatusNaN ? "NaN in a reduction " : "",
                          status & kStatusTimeout ? "copy wait timed out" : "");
        if (j.opts.tol_gn > 0.0 && !converged[i] && result == MPM_OK) result = MPM_WARN_NOT_CONVERGED;
    }
    return result;
}

}  // namespace mpm

using namespace mpm;

// ================================================================= C ABI

extern "C" {

const char* mpm_status_string(mpm_status s)
{
    switch (s) {
    case MPM_OK: return "ok";
    case MPM_WARN_NOT_CONVERGED: return "not converged within gn_iters";
    case MPM_ERR_INVALID_ARG: return "invalid argument";
    case MPM_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
    case MPM_ERR_CUDA: return "CUDA error";
    case MPM_ERR_NUMERIC: return "numeric failure (non positive definite block or NaN)";
    case MPM_ERR_TIMEOUT: return "timeout";
    default: return "unknown status";
    }
}

const char* mpm_last_error(void) { return t_err.c_str(); }

unsigned long long mpm_kernel_launches(void) { return g_launches.load(); }

mpm_status mpm_test_copy_timeout(int withhold, double wait_us)
{
    if (!(wait_us >= 0.0) || !std::isfinite(wait_us))
        return fail(MPM_ERR_INVALID_ARG, "wait_us must be finite and >= 0");
    long long cycles = 0;
    if (wait_us > 0.0) {
        int dev = 0, khz = 0;
        MPM_CUDA(cudaGetDevice(&dev));
        MPM_CUDA(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
        cycles = (long long)(wait_us * 1e-3 * (double)khz);
        if (cycles < 1) cycles = 1;
    }
    set_copy_test(withhold, cycles);
    return MPM_OK;
}

mpm_status mpm_profile_enable(int on)
{
    g_prof_on.store(on != 0);
    return MPM_OK;
}

mpm_status mpm_profile_read(double* ms, unsigned long long* launches, int n)
{
    if (n < 0) return fail(MPM_ERR_INVALID_ARG, "n < 0");
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (int k = 0; k < n; ++k) {
        if (ms) ms[k] = 0.0;
        if (launches) launches[k] = 0;
    }
    mpm_status st = MPM_OK;
    for (const ProfRecord& r : g_prof) {
        float t = 0.0f;
        if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) {
            cudaGetLastError();
            st = fail(MPM_ERR_CUDA, "event timing failed");
        } else if (r.kind < n) {
            if (ms) ms[r.kind] += t;
            if (launches) launches[r.kind] += 1;
        }
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_prof.clear();
    return st;
}

mpm_status mpm_workspace_size(const mpm_problem* problem, const mpm_opts* opts, int call,
                              size_t* bytes)
{
    MPM_TRY(check_problem(problem));
    if (!bytes) return fail(MPM_ERR_INVALID_ARG, "bytes is NULL");
    if (call < MPM_CALL_FIT || call > MPM_CALL_JTV) return fail(MPM_ERR_INVALID_ARG, "unknown call %d", call);
    if ((call == MPM_CALL_FIT || call == MPM_CALL_SOLVE)) MPM_TRY(check_opts(opts));
    *bytes = layout(make_dev(problem), call, nullptr).total;
    return MPM_OK;
}

mpm_status mpm_forward(const mpm_problem* problem, const float* y, const float* b1p,
                       const float* b1m, float* s, void* stream)
{
    MPM_TRY(check_problem(problem));
    const DevProblem P = make_dev(problem);
    if (P.N == 0) return MPM_OK;
    MPM_TRY(check_dev(y, "y", false, 4));
    MPM_TRY(check_dev(b1p, "b1p", true, 4));
    MPM_TRY(check_dev(b1m, "b1m", true, 4));
    MPM_TRY(check_dev(s, "s", false, 4));
    MPM_CUDA(launch_forward(P, y, b1p, b1m, s, (cudaStream_t)stream));
    return MPM_OK;
}

mpm_status mpm_grad_hess(const mpm_problem* problem, const void* x, const float* y,
                         const float* b1p, const float* b1m, float* g, float* h, double* nll,
                         void* ws, size_t ws_bytes, void* stream)
{
    MPM_TRY(check_problem(problem));
    const DevProblem P = make_dev(problem);
    cudaStream_t st = (cudaStream_t)stream;
    MPM_TRY(check_dev(nll, "nll", false, 8));
    if (P.N == 0) {
        MPM_CUDA(cudaMemsetAsync(nll, 0, sizeof(double), st));
        return MPM_OK;
    }
    MPM_TRY(check_dev(x, "x", false, problem->echo_dtype ? 2 : 4));
    MPM_TRY(check_dev(y, "y", false, 4));
    MPM_TRY(check_dev(b1p, "b1p", true, 4));
    MPM_TRY(check_dev(b1m, "b1m", true, 4));
    MPM_TRY(check_dev(g, "g", false, 4));
    MPM_TRY(check_dev(h, "h", false, 4));
    FitWs L;
    MPM_TRY(check_ws(P, MPM_CALL_GRAD_HESS, ws, ws_bytes, L));
    MPM_CUDA(cudaMemsetAsync(L.hdr, 0, sizeof(WsHeader), st));
    MPM_CUDA(launch_grad_hess(P, problem->echo_dtype, x, y, b1p, b1m, g, h, nll, L.red,
                              &L.hdr->status, st));
    return MPM_OK;
}

mpm_status mpm_jtv_weights(const mpm_problem* problem, const float* y, float* w, double* jtv,
                           void* ws, size_t ws_bytes, void* stream)
{
    MPM_TRY(check_problem(problem));
    const DevProblem P = make_dev(problem);
    cudaStream_t st = (cudaStream_t)stream;
    MPM_TRY(check_dev(jtv, "jtv", false, 8));
    if (P.N == 0) {
        MPM_CUDA(cudaMemsetAsync(jtv, 0, sizeof(double), st));
        return MPM_OK;
    }
    MPM_TRY(check_dev(y, "y", false, 4));
    MPM_TRY(check_dev(w, "w", true, 4));
    FitWs L;
    MPM_TRY(check_ws(P, MPM_CALL_JTV, ws, ws_bytes, L));
    MPM_CUDA(cudaMemsetAsync(L.hdr, 0, sizeof(WsHeader), st));
    MPM_CUDA(launch_jtv(P, y, w, jtv, L.red, st));
    return MPM_OK;
}

mpm_status mpm_solve(const mpm_problem* problem, const mpm_opts* opts, const float* h,
                     const float* w, const float* g, const float* y, float* delta, double* resid,
                     void* ws, size_t ws_bytes, void* stream)
{
    MPM_TRY(check_problem(problem));
    MPM_TRY(check_opts(opts));
    const DevProblem P = make_dev(problem);
    cudaStream_t st = (cudaStream_t)stream;
    if (P.N == 0) {
        if (resid) {
            MPM_TRY(check_dev(resid, "resid", false, 8));
            MPM_CUDA(cudaMemsetAsync(resid, 0, sizeof(double), st));
        }
        return MPM_OK;
    }
    MPM_TRY(check_dev(h, "h", false, 4));
    MPM_TRY(check_dev(w, "w", false, 4));
    MPM_TRY(check_dev(g, "g", false, 4));
    MPM_TRY(check_dev(y, "y", false, 4));
    MPM_TRY(check_dev(delta, "delta", false, 4));
    MPM_TRY(check_dev(resid, "resid", true, 8));
    FitWs L;
    MPM_TRY(check_ws(P, MPM_CALL_SOLVE, ws, ws_bytes, L));
    MPM_CUDA(cudaMemsetAsync(L.hdr, 0, sizeof(WsHeader), st));
    MPM_CUDA(launch_solve(P, solve_opts(*opts), h, w, g, y, delta, nullptr, resid,
                          nullptr, nullptr, L.solve, L.hdr, L.red, st));
    return MPM_OK;
}

mpm_status mpm_uncertainty(const mpm_problem* problem, const float* h, const float* w,
                           const float* y, float* var, float* logdet, float* moments,
                           void* stream)
{
    MPM_TRY(check_problem(problem));
    const DevProblem P = make_dev(problem);
    if (P.N == 0) return MPM_OK;
    MPM_TRY(check_dev(h, "h", false, 4));
    MPM_TRY(check_dev(w, "w", false, 4));
    MPM_TRY(check_dev(var, "var", false, 4));
    MPM_TRY(check_dev(logdet, "logdet", true, 4));
    MPM_TRY(check_dev(moments, "moments", true, 4));
    MPM_TRY(check_dev(y, "y", moments == nullptr, 4));
    // The status word of the uncertainty pass is not reported through a
    // workspace (the call takes none): a non positive definite block yields
    // non-finite variances instead.
    MPM_CUDA(launch_uncertainty(P, h, w, y, var, logdet, moments, nullptr, (cudaStream_t)stream));
    return MPM_OK;
}

mpm_status mpm_autotune(const mpm_problem* problem, const mpm_opts* opts, void* ws,
                        size_t ws_bytes, void* stream, int* tile, float* ms)
{
    MPM_TRY(check_problem(problem));
    MPM_TRY(check_opts(opts));
    const DevProblem P = make_dev(problem);
    const int want = tile ? *tile : -1;
    if (want >= MPM_TILE_SHAPES) return fail(MPM_ERR_INVALID_ARG, "tile %d out of range", want);
    if (tile) *tile = -1;
    if (P.N == 0) return MPM_OK;
    float t_ms[MPM_TILE_SHAPES];
    int best = -1;
    if (want >= 0) {
        // pin the requested shape without timing
        for (int i = 0; i < MPM_TILE_SHAPES; ++i) t_ms[i] = -1.0f;
        tma_tile_set(P, want);
        best = want;
    } else {
        FitWs L;
        MPM_TRY(check_ws(P, MPM_CALL_SOLVE, ws, ws_bytes, L));
        MPM_CUDA(tma_autotune(P, L.solve, L.hdr, L.red, (cudaStream_t)stream, &best, t_ms));
    }
    if (tile) *tile = best;
    if (ms)
        for (int i = 0; i < MPM_TILE_SHAPES; ++i) ms[i] = i < tma_tile_count() ? t_ms[i] : -1.0f;
    return MPM_OK;
}

mpm_status mpm_workspace_status(const void* ws, size_t ws_bytes, void* stream)
{
    if (ws_bytes < sizeof(WsHeader)) return fail(MPM_ERR_WORKSPACE_TOO_SMALL, "workspace too small");
    MPM_TRY(check_dev(ws, "ws", false, 256));
    cudaStream_t st = (cudaStream_t)stream;
    unsigned status = 0;
    MPM_CUDA(cudaMemcpyAsync(&status, ws, sizeof status, cudaMemcpyDeviceToHost, st));
    MPM_CUDA(cudaStreamSynchronize(st));
    if (status) return fail(MPM_ERR_NUMERIC, "device status 0x%x (%s%s%s)", status,
                            status & kStatusNotPD ? "non positive definite block " : "",
                            status & kStatusNaN ? "NaN in a reduction " : "",
                            status & kStatusTimeout ? "copy wait timed out" : "");
    return MPM_OK;
}

mpm_status mpm_fit(const mpm_problem* problem, const mpm_opts* opts, const void* x,
                   const float* b1p, const float* b1m, float* y, float* var_out, void* ws,
                   size_t ws_bytes, mpm_report* report, void* stream)
{
    FitJob job;
    MPM_TRY(fit_prepare(problem, opts, x, b1p, b1m, y, var_out, ws, ws_bytes, job));
    return fit_run(&job, 1, report, (cudaStream_t)stream);
}

mpm_status mpm_fit_proj(const mpm_problem* problem, const mpm_projection* proj,
                        const mpm_opts* opts, const void* const* x, const float* const* b1p,
                        const float* const* b1m, float* y, float* var_out, void* ws,
                        size_t ws_bytes, mpm_report* report, void* stream)
{
    FitJob job;
    MPM_TRY(check_problem(problem));
    MPM_TRY(check_opts(opts));
    job.problem = problem;
    job.opts = *opts;
    job.P = make_dev(problem);
    job.x = nullptr;
    job.b1p = job.b1m = nullptr;
    job.y = y;
    job.var = var_out;
    job.ws = ws;
    job.ws_bytes = ws_bytes;
    job.empty = job.P.N == 0;
    job.proj = true;
    memset(&job.pj, 0, sizeof job.pj);
    if (job.empty) {
        if (report) memset(report, 0, sizeof *report);
        return MPM_OK;
    }
    MPM_TRY(check_dev(y, "y_inout", false, 4));
    MPM_TRY(check_dev(var_out, "var_out", true, 4));
    mpm_status s = proj_prepare(problem, proj, x, b1p, b1m, ws, ws_bytes, job.pj, job.L);
    if (s == MPM_OK) s = fit_run(&job, 1, report, (cudaStream_t)stream);
    proj_release(job.pj);
    return s;
}

mpm_status mpm_fit_batch(int n, const mpm_problem* const* problems, const mpm_opts* opts,
                         const void* const* x, const float* const* b1p, const float* const* b1m,
                         float* const* y, float* const* var_out, void* const* ws,
                         const size_t* ws_bytes, mpm_report* reports, void* stream)
{
    if (n < 0 || n > MPM_MAX_BATCH) return fail(MPM_ERR_INVALID_ARG, "batch size %d outside [0, %d]", n, MPM_MAX_BATCH);
    if (n == 0) return MPM_OK;
    if (!problems || !x || !y || !ws || !ws_bytes)
        return fail(MPM_ERR_INVALID_ARG, "problems, x, y, ws and ws_bytes must not be NULL");
    std::vector<FitJob> jobs(n);
    for (int i = 0; i < n; ++i) {
        mpm_status s = fit_prepare(problems[i], opts, x[i], b1p ? b1p[i] : nullptr,
                                   b1m ? b1m[i] : nullptr, y[i], var_out ? var_out[i] : nullptr,
                                   ws[i], ws_bytes[i], jobs[i]);
        if (s != MPM_OK) return fail(s, "subject %d: %s", i, t_err.c_str());
    }
    return fit_run(jobs.data(), n, reports, (cudaStream_t)stream);
}

}  // extern "C"
