// mpm_internal.cuh -- host side of the sm_103a MPM library shared by its
// translation units: launch helpers, kernel launchers, the workspace layout,
// argument checks and status macros (device_common.cuh holds what the kernels
// share).  Internal: not part of the C ABI (include/mpm.h).
#pragma once

#include <string>

#include "device_common.cuh"
#include "host_logic.h"
#include "pcg_step.cuh"
#include "batch.cuh"

namespace mpm {

// ------------------------------------------------------- launch helpers

struct StencilGrid {
    dim3 grid, block;
    int zc;           // z planes per block (TMA iteration: number of z ranges)
};

// Blocks of a z-marching stencil kernel: about `waves` waves of 8 resident
// blocks per SM over tile columns cut into z ranges; a volume that shares a
// launch with others takes `share` of those blocks.
StencilGrid stencil_grid(const DevProblem& P, int tile_x, int tile_y, int waves = 2,
                         double share = 1.0);
constexpr int kInitWaves = 4;   // the PCG start's (shorter z ranges measured faster)
int voxel_grid(long long N);

// Every kernel launch goes through a LaunchScope: it counts the launch and,
// when diagnostic timing is on (mpm_profile_enable), brackets it with CUDA
// events on its stream, accumulated per kernel kind (MPM_KERNEL_*).
struct LaunchScope {
    LaunchScope(int kind, cudaStream_t st);
    ~LaunchScope();
    static void capturing(bool on);   // no timing events while this thread captures a graph
    int kind;
    cudaStream_t st;
    void* rec;
};

// ------------------------------------------------------- kernel launchers
// (defined in voxel_kernels.cu and stencil_kernels.cu; return cudaError_t of
// the launch)

cudaError_t launch_forward(const DevProblem& P, const float* y, const float* b1p,
                           const float* b1m, float* s, cudaStream_t st);
// The voxel pass; `status` receives kStatusTimeout if a staged copy never
// lands (voxel_tma.cu).
cudaError_t launch_grad_hess(const DevProblem& P, int echo_dtype, const void* x,
                             const float* y, const float* b1p, const float* b1m, float* g,
                             float* h, double* nll, Reduce red, unsigned* status, cudaStream_t st);
bool grad_hess_tma_ok(const DevProblem& P, const void* x, const float* y, const float* b1p,
                      const float* b1m, const float* g, const float* h);
// The staged pass over several subjects (one wave shared by their chunks);
// false, with nothing launched, when some subject cannot take it.
bool launch_grad_hess_tma_batch(int K, int precond, int echo_dtype, const GradArgs* a, int n,
                                cudaStream_t st, cudaError_t* err);
cudaError_t launch_grad_hess_tma(const DevProblem& P, int echo_dtype, const void* x, const float* y,
                                 const float* b1p, const float* b1m, float* g, float* h, double* nll,
                                 Reduce red, unsigned* status, cudaStream_t st);
cudaError_t launch_uncertainty(const DevProblem& P, const float* h, const float* w,
                               const float* y, float* var, float* logdet, float* moments,
                               unsigned* status, cudaStream_t st);
cudaError_t launch_image_means(const DevProblem& P, int echo_dtype, const void* x,
                               double* partials, double* means, cudaStream_t st);
// The constant starting maps from the image means in device memory
// (init_maps.cuh), written to y.
cudaError_t launch_init_maps(const DevProblem& P, const double* means, float* y, cudaStream_t st);

cudaError_t launch_jtv(const DevProblem& P, const float* y, float* w, double* jtv,
                       Reduce red, cudaStream_t st);
// Schedule of one solve (from mpm_opts; the multigrid fields resolved to
// their defaults).
struct SolveOpts {
    int cg_iters;
    double tol_cg;
    int mg_levels;          // 0: block-Jacobi PCG (Eq. 42); > 0: multigrid-preconditioned CG
    int mg_nu;
    float mg_omega;
    int mg_coarse_sweeps;
};
SolveOpts solve_opts(const mpm_opts& o);
cudaError_t launch_solve(const DevProblem& P, const SolveOpts& so, const float* h,
                         const float* w, const float* g, const float* y, float* delta,
                         float* y_update, double* resid, double* report_rel,
                         int* report_it, void* solve_ws, WsHeader* hdr, Reduce red,
                         cudaStream_t st);
size_t solve_ws_bytes(const DevProblem& P);   // enough for either solver
size_t mg_ws_bytes(const DevProblem& P);      // multigrid.cu
cudaError_t launch_solve_mg(const DevProblem& P, const SolveOpts& o, const float* h, const float* w,
                            const float* g, const float* y, float* delta, float* y_update,
                            double* resid, double* report_rel, int* report_it, void* solve_ws,
                            WsHeader* hdr, Reduce red, cudaStream_t st);

// TMA-staged PCG iteration (stencil_tma.cu).  make_step_maps returns false
// when the volume or the pointers do not meet the copy engine's alignment
// rules; the plain kernel is used then.
struct StepMaps {
    CUtensorMap z[2], v[2], p[3];   // halo boxes of the solve's vectors
    CUtensorMap p2[3], x;           // tile boxes (x fold)
    CUtensorMap w, h;
    SolveBufs B;
    int tile;          // index of the tile shape the maps were encoded for
};
int tma_tile_count();
bool make_step_maps(const DevProblem& P, const float* h, const float* w, const SolveBufs& B,
                    int tile, StepMaps* out);
StencilGrid tma_grid(const DevProblem& P, int tile);
cudaError_t prime_tma_kernels();   // shared-memory opt-ins, done before any graph capture
cudaError_t prime_voxel_kernels(); // those of the staged voxel pass (voxel_tma.cu)
int tma_tile_choice(const DevProblem& P);   // tile shape for this volume (tuned or default)
void tma_tile_set(const DevProblem& P, int tile);
// Times every applicable tile shape of the TMA iteration on this volume
// (operands taken from the solve workspace, zeroed), records the fastest for
// later solves and returns it (-1 when TMA does not apply); ms[i] receives
// the mean time of shape i (or -1).  Synchronises the stream.
cudaError_t tma_autotune(const DevProblem& P, void* solve_ws, WsHeader* hdr, Reduce red,
                         cudaStream_t st, int* best, float* ms);
// Iteration j (mode kMode*) of a solve; want_rr also reduces the |r|^2 sums.
cudaError_t launch_step_tma(const DevProblem& P, const StencilGrid& g, const StepMaps& m, int j,
                            int mode, int want_rr, WsHeader* hdr, double* resid, Reduce red,
                            cudaStream_t st);
// Launches serving several subjects (batch.cuh): blocks[s] hardware blocks
// for subject s, n <= kBatchMax.
SolveBufs solve_bufs(const DevProblem& P, void* solve_ws);
cudaError_t launch_jtv_batch(int K, const JtvArgs* a, const unsigned* blocks, int n, cudaStream_t st);
cudaError_t launch_grad_hess_batch(int K, int precond, int echo_dtype, const GradArgs* a,
                                   const unsigned* blocks, int n, cudaStream_t st);
cudaError_t launch_pcg_init_batch(int K, const InitArgs* a, const unsigned* blocks, int n,
                                  cudaStream_t st);
StepArgs step_args(const DevProblem& P, const StepMaps& m, int nchunk, int j, int want_rr,
                   WsHeader* hdr, double* resid, Reduce red);
cudaError_t launch_step_batch(int K, int tile, int mode, const StepArgs* a, const unsigned* blocks,
                              int n, cudaStream_t st);
cudaError_t launch_pcg_final_batch(int K, const FinalArgs* a, const unsigned* blocks, int n,
                                   cudaStream_t st);
cudaError_t launch_uncertainty_batch(int K, const UncArgs* a, const unsigned* blocks, int n,
                                     cudaStream_t st);
int step_mode(int j);                               // kMode* of PCG iteration j
int tma_tiles_of(const DevProblem& P, int tile);    // tiles of the (x, y) plane
int tma_wave_blocks(const DevProblem& P, int tile); // resident blocks of the TMA iteration, whole GPU

// Test hook: with withhold set, the TMA iteration's producer issues no copies;
// every bounded wait gives up after wait_cycles clock cycles (<= 0: default).
void set_copy_test(int withhold, long long wait_cycles);
int copy_withhold();
long long copy_wait_cycles();

// ------------------------------------------- host helpers of the entry points
// (mpm_api.cu)

constexpr size_t kHeaderBytes = 4096;                              // WsHeader, padded
constexpr size_t kPartialBytes = sizeof(double) * 8 * kMaxBlocks;  // reduction partials (8 sums)

// Carving of a fit / solve workspace (mpm_api.cu).
struct FitWs {
    WsHeader* hdr;
    Reduce red;
    double* mean_parts;
    double* means;
    double* nll;       // [MPM_MAX_REPORT + 2]
    double* jtv;       // [MPM_MAX_REPORT + 2]
    double* cg_rel;    // [MPM_MAX_REPORT]
    int* cg_it;        // [MPM_MAX_REPORT]
    float* w;
    float* g;
    float* h;
    void* solve;
    size_t total;
};

FitWs layout(const DevProblem& P, int call, void* base);   // base NULL: sizes only

// Spatial projection (projection.cu): per-contrast inputs on the acquisition
// grids, and the opaque projection and workspace of one projected fit.
struct ProjIn {
    int echo_dtype;
    const void* x[MPM_MAX_CONTRASTS];
    const float* b1p[MPM_MAX_CONTRASTS];
    const float* b1m[MPM_MAX_CONTRASTS];
};
struct ProjJob {
    void* Q;          // DevProj
    void* W;          // ProjWs
    ProjIn in;
};
cudaError_t launch_grad_hess_proj(const DevProblem& P, const ProjJob& pj, const float* y, float* g,
                                  float* h, double* nll, Reduce red, cudaStream_t st);
mpm_status proj_prepare(const mpm_problem* problem, const mpm_projection* proj, const void* const* x,
                        const float* const* b1p, const float* const* b1m, void* ws, size_t ws_bytes,
                        ProjJob& pj, FitWs& L);
void proj_release(ProjJob& pj);
size_t proj_key_bytes();
void proj_key(const ProjJob& pj, std::string& k);
cudaError_t proj_image_means(const DevProblem& P, const ProjJob& pj, double* parts, double* means,
                             cudaStream_t st);
mpm_status check_ws(const DevProblem& P, int call, void* ws, size_t ws_bytes, FitWs& L);

mpm_status fail(mpm_status s, const char* fmt, ...);

// Return the status of a failing call (with the CUDA error text).
#define MPM_CUDA(call)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(MPM_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),   \
                        __FILE__, __LINE__);                                             \
    } while (0)

#define MPM_TRY(expr)                     \
    do {                                  \
        mpm_status s_ = (expr);           \
        if (s_ != MPM_OK) return s_;      \
    } while (0)

mpm_status check_problem(const mpm_problem* p);
mpm_status check_opts(const mpm_opts* o);
mpm_status check_dev(const void* ptr, const char* name, bool optional, size_t align);
DevProblem make_dev(const mpm_problem* p);

}  // namespace mpm
