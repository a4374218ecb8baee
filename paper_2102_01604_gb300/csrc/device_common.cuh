// device_common.cuh -- what every kernel of the sm_103a MPM library shares:
// launch constants, the problem descriptor passed to kernels, the device
// scalars and reduction scratch in the workspace, the compensated float32
// accumulators and the deterministic grid reduction.  Internal.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

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
    unsigned flip_as_c0;                // bit c (c > 0): alpha[c] == alpha[0]
    unsigned echoes_as_prev;            // bit c (c > 0): c and c - 1 both have equally spaced
                                        // echoes with the same first time and spacing
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
    double rz;        // r . z of the next residual (expanded, pcg_step.cuh)
    double rr0;       // |r_0|^2
    double rr;        // |r_k|^2 of the current residual
    double alpha;     // step of the latest completed iteration
    double alpha_prev;  // step of the iteration before it
    double beta;      // coefficient of the next direction update
    double tol2;      // (tol_cg)^2, 0 = off
    int it;           // PCG iterations completed
    int xcount;       // iterations already folded into x (x is updated every other iteration)
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

// A block's place in its launch: the hardware grid for a launch of one
// subject, or the subject's share of a launch that serves several subjects
// (blocks [start, start + count) of it belong to one subject and see a grid
// of `count` blocks, shaped gx x gy x gz).
struct VGrid {
    unsigned bx, by, bz;     // block index
    unsigned gx, gy, gz;     // grid dimensions
    __device__ unsigned id() const { return bx + gx * (by + gy * bz); }
    __device__ unsigned count() const { return gx * gy * gz; }
};

__device__ __forceinline__ VGrid hw_grid()
{
    return VGrid{blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x, gridDim.y, gridDim.z};
}

// The subject of this block in a launch of several (start[s] is the first
// hardware block of subject s, start[n] the total), and its virtual grid of
// shape gx x gy x gz (gx gy gz = start[s + 1] - start[s]).
__device__ __forceinline__ int batch_subject(const unsigned* start, int n)
{
    int s = 0;
    while (s + 1 < n && blockIdx.x >= start[s + 1]) ++s;
    return s;
}

__device__ __forceinline__ VGrid batch_grid(unsigned first, unsigned gx, unsigned gy, unsigned gz)
{
    const unsigned v = blockIdx.x - first;
    return VGrid{v % gx, (v / gx) % gy, v / (gx * gy), gx, gy, gz};
}

// Last-block-done reduction of NV values per block.  Every thread calls it
// with its own compensated partials; returns true in exactly one block (the
// last to arrive), where out[j] (valid in thread 0) holds the grid-wide sums
// in a fixed summation order.  The counter is reset for the next launch.
// The grid is the block's launch, or its subject's share of a launch (vg).
template <int NV>
__device__ __forceinline__ bool grid_reduce(const Acc (&v)[NV], Reduce red, double (&out)[NV],
                                            const VGrid& vg)
{
    __shared__ double sh[32];          // one slot per warp of the block (up to 1024 threads)
    __shared__ bool am_last;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nthreads = blockDim.x * blockDim.y;
    const unsigned bid = vg.id();
    const unsigned nblocks = vg.count();
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

template <int NV>
__device__ __forceinline__ bool grid_reduce(const Acc (&v)[NV], Reduce red, double (&out)[NV])
{
    return grid_reduce<NV>(v, red, out, hw_grid());
}

// Hint the line holding p into L2 (kernels fetch the operands of a later
// voxel or plane this way while they compute the current one).
__device__ __forceinline__ void prefetch_l2(const void* p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
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

}  // namespace mpm
