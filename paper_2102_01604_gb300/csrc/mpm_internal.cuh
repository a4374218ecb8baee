// mpm_internal.cuh -- device-side problem descriptor, workspace layout and
// shared device helpers of the sm_103a MPM library.  Internal: not part of the
// C ABI (include/mpm.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>

#include "../../include/mpm.h"

namespace mpm {

constexpr int kBlock = 256;            // threads per block of every kernel
constexpr int kTileX = 32;             // stencil tile: 32 x 8 (x, y), marched along z
constexpr int kTileY = 8;
constexpr int kMaxBlocks = 32768;      // bound on the blocks of a reducing launch
constexpr int kNumSm = 152;

// Problem as the kernels see it: passed by value as a kernel parameter.
struct DevProblem {
    int nx, ny, nz;
    long long N;
    float ihx2, ihy2, ihz2;             // 1 / voxel size^2 per axis
    int C, K, T, I;
    int n_echoes[MPM_MAX_CONTRASTS];
    int echo0[MPM_MAX_CONTRASTS];       // index of the first image of contrast c
    float alpha[MPM_MAX_CONTRASTS];
    float tr[MPM_MAX_CONTRASTS];
    float isig2[MPM_MAX_CONTRASTS];     // 1 / sigma^2
    int mt[MPM_MAX_CONTRASTS];
    float te[MPM_MAX_IMAGES];
    float dte[MPM_MAX_CONTRASTS];       // echo spacing when the echoes are equally spaced
    int te_uniform[MPM_MAX_CONTRASTS];  // 1: te = te0 + e * dte for every echo of c
    int same_tr[MPM_MAX_CONTRASTS];     // 1: tr[c] == tr[c - 1]
    float lambda[4];
    float eps2;
    int precond;
};

// Packed upper-triangle position of (a, b), a <= b, for K maps.
__host__ __device__ constexpr int tri(int K, int a, int b)
{
    return a * K - a * (a - 1) / 2 + (b - a);
}

// Status bits recorded on the device.
enum : unsigned { kStatusNotPD = 1u, kStatusNaN = 2u, kStatusTimeout = 4u };

// Device scalars of one PCG solve (lives in the workspace).
struct SolveScalars {
    double rz;        // r . z of the current residual
    double rr0;       // |r_0|^2
    double rr;        // |r_k|^2 of the current residual
    double alpha;     // step of the latest completed matvec
    double beta;      // coefficient of the next direction update
    double tol2;      // (tol_cg)^2, 0 = off
    int it;           // PCG iterations completed
    int xcount;       // iterations already folded into x
    int done;         // 1 = no further iterations
    int pad;
};

// Reduction scratch: per-block partials and an arrival counter.  The counter
// is zero between launches (the last block resets it).
struct Reduce {
    double* partials;        // [kMaxBlocks * 2]
    unsigned int* counter;
};

// Workspace header, first bytes of every workspace.
struct WsHeader {
    unsigned int status;     // kStatus* bits
    unsigned int counter;    // reduction arrival counter
    SolveScalars sc;
};

// ------------------------------------------------------------------ helpers

// Compensated float32 accumulator for the float64-class sums (CG inner
// products, residual norms, likelihood and JTV energy).  GB300 issues float64
// arithmetic at a small fraction of its float32 rate, so each thread keeps its
// running sum as an unevaluated pair hi + lo updated by Knuth's two-sum (an
// error-free transformation: hi + lo is the exact sum of the added float32
// values up to the rounding of lo); warps combine pairs the same way, and only
// per-warp and per-block partials are converted to float64 and reduced in a
// fixed order.
struct Acc {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float x)
    {
        const float s = __fadd_rn(hi, x);
        const float bp = __fsub_rn(s, hi);
        const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
        hi = s;
        lo = __fadd_rn(lo, e);
    }
    __device__ __forceinline__ void add(const Acc& o)
    {
        add(o.hi);
        lo = __fadd_rn(lo, o.lo);
    }
};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Sum of v over the block, valid in thread 0.  Fixed order (deterministic).
__device__ __forceinline__ double block_sum(double v, double* sh /* one per warp */)
{
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nw = (blockDim.x * blockDim.y + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if ((tid & 31) == 0) sh[tid >> 5] = v;
    __syncthreads();
    v = 0.0;
    if (tid < 32) {
        v = tid < nw ? sh[tid] : 0.0;
        v = warp_sum(v);
    }
    return v;
}

// Warp-level combination of compensated pairs (lane 0 holds the result),
// then float64 for the few per-warp values.
__device__ __forceinline__ double warp_acc(Acc a)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Acc b;
        b.hi = __shfl_down_sync(0xffffffffu, a.hi, o);
        b.lo = __shfl_down_sync(0xffffffffu, a.lo, o);
        a.add(b);
    }
    return (double)a.hi + (double)a.lo;
}

__device__ __forceinline__ double block_acc(Acc a, double* sh /* one per warp */)
{
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nw = (blockDim.x * blockDim.y + 31) >> 5;
    const double w = warp_acc(a);
    __syncthreads();
    if ((tid & 31) == 0) sh[tid >> 5] = w;
    __syncthreads();
    double v = 0.0;
    if (tid < 32) {
        v = tid < nw ? sh[tid] : 0.0;
        v = warp_sum(v);
    }
    return v;
}

// Last-block-done reduction of NV values per block.  Every thread calls it
// with its own compensated partials; returns true in exactly one block (the
// last to arrive), where out[j] (valid in thread 0) holds the grid-wide sums
// in a fixed summation order.  The counter is reset for the next launch.
template <int NV>
__device__ __forceinline__ bool grid_reduce(const Acc (&v)[NV], Reduce red, double (&out)[NV])
{
    __shared__ double sh[32];          // one slot per warp of the block (up to 1024 threads)
    __shared__ bool am_last;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nthreads = blockDim.x * blockDim.y;
    const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const unsigned nblocks = gridDim.x * gridDim.y * gridDim.z;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        double s = block_acc(v[j], sh);
        if (tid == 0) red.partials[(size_t)j * kMaxBlocks + bid] = s;
    }
    if (tid == 0) {
        __threadfence();
        unsigned prev = atomicAdd(red.counter, 1u);
        am_last = (prev == nblocks - 1);
    }
    __syncthreads();
    if (!am_last) return false;
    __threadfence();
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        double s = 0.0;
        for (unsigned b = tid; b < nblocks; b += nthreads)
            s += __ldcg(&red.partials[(size_t)j * kMaxBlocks + b]);
        out[j] = block_sum(s, sh);
    }
    if (tid == 0) *red.counter = 0u;
    return true;
}

template <typename T>
__device__ __forceinline__ float load_echo(const T* p, long long i);

template <>
__device__ __forceinline__ float load_echo<float>(const float* p, long long i)
{
    return __ldg(p + i);
}

template <>
__device__ __forceinline__ float load_echo<__nv_bfloat16>(const __nv_bfloat16* p, long long i)
{
    return __bfloat162float(p[i]);
}

// ------------------------------------------------------- launch helpers

struct StencilGrid {
    dim3 grid, block;
    int zc;           // z planes per block (TMA matvec: number of z ranges)
};

StencilGrid stencil_grid(const DevProblem& P, int tile_x, int tile_y);
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
cudaError_t launch_grad_hess(const DevProblem& P, int echo_dtype, const void* x,
                             const float* y, const float* b1p, const float* b1m, float* g,
                             float* h, double* nll, Reduce red, cudaStream_t st);
cudaError_t launch_uncertainty(const DevProblem& P, const float* h, const float* w,
                               const float* y, float* var, float* logdet, float* moments,
                               unsigned* status, cudaStream_t st);
cudaError_t launch_image_means(const DevProblem& P, int echo_dtype, const void* x,
                               double* partials, double* means, cudaStream_t st);
cudaError_t launch_fill_maps(const DevProblem& P, const float* values, float* y,
                             cudaStream_t st);

cudaError_t launch_jtv(const DevProblem& P, const float* y, float* w, double* jtv,
                       Reduce red, cudaStream_t st);
cudaError_t launch_solve(const DevProblem& P, int cg_iters, double tol_cg, const float* h,
                         const float* w, const float* g, const float* y, float* delta,
                         float* y_update, double* resid, double* report_rel,
                         int* report_it, void* solve_ws, WsHeader* hdr, Reduce red,
                         cudaStream_t st);
size_t solve_ws_bytes(const DevProblem& P);

// TMA-staged stencil matvec (stencil_tma.cu).  make_tma_maps returns false
// when the volume or the pointers do not meet the copy engine's alignment
// rules; the shared-memory kernel is used then.
struct TmaMaps {
    CUtensorMap p[2], w, h;
    int tile;          // index of the tile shape the maps were encoded for
};
int tma_tile_count();
bool make_tma_maps(const DevProblem& P, const float* h, const float* w, const float* p0,
                   const float* p1, int tile, TmaMaps* out);
StencilGrid tma_grid(const DevProblem& P, int tile);
cudaError_t prime_tma_kernels();   // shared-memory opt-ins, done before any graph capture
int tma_tile_choice(const DevProblem& P);   // tile shape for this volume (tuned or default)
void tma_tile_set(const DevProblem& P, int tile);
// Times every applicable tile shape of the TMA matvec on this volume (operands
// taken from the solve workspace, zeroed), records the fastest for later
// solves and returns it (-1 when TMA does not apply); ms[i] receives the mean
// time of shape i (or -1).  Synchronises the stream.
cudaError_t tma_autotune(const DevProblem& P, void* solve_ws, WsHeader* hdr, Reduce red,
                         cudaStream_t st, int* best, float* ms);
cudaError_t launch_matvec_tma(const DevProblem& P, const StencilGrid& g, const TmaMaps& m,
                              int k_it, float* q, WsHeader* hdr, Reduce red, cudaStream_t st);

// ------------------------------------------- host helpers of the entry points
// (mpm_api.cu)

constexpr size_t kHeaderBytes = 4096;                              // WsHeader, padded
constexpr size_t kPartialBytes = sizeof(double) * 2 * kMaxBlocks;  // reduction partials

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
    float* xbuf;
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
void initial_maps(const mpm_problem* p, const double* mean, float out[4]);

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
