// projection.cu -- spatial projection (Sec. 2.4) on sm_103a.
//
// Contrast c was acquired on its own grid of M_c voxels; the 3 x 4 affine A_c
// maps its voxel coordinates (i, j, k, 1) to reconstruction voxel
// coordinates.  The reslicing Psi_c interpolates the K maps trilinearly at
// A_c m; acquisition voxels whose point falls outside the reconstruction grid
// carry no data term.  The likelihood becomes l(y) = sum_c l_c(Psi_c y), with
// gradient sum_c Psi_c' g_c and, for the Hessian, the block-diagonal
// majoriser sum_c Psi_c' H_c (the interpolation weights of an inside voxel are
// non-negative and sum to one).
//
//   k_grad_hess_proj  per acquisition voxel of one contrast: interpolate the
//                     maps (8 corners), then the same per-contrast voxel model
//                     as k_grad_hess (voxel_model.cuh); writes g_c and H_c
//                     (interleaved per acquisition voxel) and the contrast's NLL
//   k_push_all        per reconstruction voxel: gathers, over every contrast,
//                     the acquisition voxels whose interpolation stencil holds
//                     it (a box around A_c^-1 n) with the pull's own weights,
//                     so the push is the exact adjoint of the pull and its sum
//                     order is fixed (no atomics); writes g and H once
//   k_pull / k_push   Psi_c u and Psi_c' u for any number of channels
//
// Coordinates are float32; pull and push evaluate them with the same
// instructions, so both see identical weights.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "mpm_internal.cuh"
#include "voxel_model.cuh"

namespace mpm {

struct ProjC {
    int mx, my, mz;
    long long M;
    float A[12];      // acquisition voxel (i, j, k, 1) -> reconstruction coordinates
    float Ai[12];     // the inverse map
    float ext[3];     // half-extent of A^-1 applied to the cube (-1, 1)^3
};

struct DevProj {
    int C;
    ProjC c[MPM_MAX_CONTRASTS];
};

// g_c and H_c of one acquisition voxel are stored together, K + T floats
// padded to a multiple of 4 (16 for K = 4, 12 for K = 3), so the push reads
// them as whole 16-byte vectors from one line.
template <int K>
struct GhStride {
    static constexpr int T = K * (K + 1) / 2;
    static constexpr int S = (K + T + 3) / 4 * 4;     // floats per voxel
    static constexpr int V = S / 4;                    // float4 per voxel
};

__host__ __device__ constexpr int gh_floats(int K) { return (K + K * (K + 1) / 2 + 3) / 4 * 4; }

// Per-contrast g_c / H_c buffers of the projected voxel pass.
struct ProjBufs {
    const float4* gh[MPM_MAX_CONTRASTS];
};

// Reconstruction coordinate of acquisition voxel (i, j, k); true when it lies
// in [0, n_d - 1] on every axis.
__device__ __forceinline__ bool reslice(const ProjC& q, int i, int j, int k, int nx, int ny,
                                        int nz, float r[3])
{
#pragma unroll
    for (int d = 0; d < 3; ++d)
        r[d] = fmaf(q.A[4 * d], (float)i, fmaf(q.A[4 * d + 1], (float)j, fmaf(q.A[4 * d + 2], (float)k, q.A[4 * d + 3])));
    return r[0] >= 0.0f && r[0] <= (float)(nx - 1) && r[1] >= 0.0f && r[1] <= (float)(ny - 1) &&
           r[2] >= 0.0f && r[2] <= (float)(nz - 1);
}

// Cell corner and fractional offsets of an inside point.
struct Cell {
    int b[3];
    float f[3];
};

__device__ __forceinline__ Cell cell_of(const float r[3])
{
    Cell c;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float fl = floorf(r[d]);
        c.b[d] = (int)fl;
        c.f[d] = r[d] - fl;
    }
    return c;
}

// Weight of corner (cx, cy, cz) of the cell: the same product, in the same
// order, in every kernel.
__device__ __forceinline__ float corner_weight(const Cell& c, int cx, int cy, int cz)
{
    const float wx = cx ? c.f[0] : 1.0f - c.f[0];
    const float wy = cy ? c.f[1] : 1.0f - c.f[1];
    const float wz = cz ? c.f[2] : 1.0f - c.f[2];
    return wx * wy * wz;
}

// Interpolate `channels` planar reconstruction images u[ch * N + n] at the
// cell; corners past the last voxel (weight 0) are skipped.
template <int CH>
__device__ __forceinline__ void interpolate(const Cell& c, const float* __restrict__ u, long long N,
                                            int nx, int ny, int nz, float (&out)[CH])
{
#pragma unroll
    for (int ch = 0; ch < CH; ++ch) out[ch] = 0.0f;
    for (int cz = 0; cz < 2; ++cz) {
        const int z = c.b[2] + cz;
        if (z > nz - 1) continue;
        for (int cy = 0; cy < 2; ++cy) {
            const int y = c.b[1] + cy;
            if (y > ny - 1) continue;
            for (int cx = 0; cx < 2; ++cx) {
                const int x = c.b[0] + cx;
                if (x > nx - 1) continue;
                const float w = corner_weight(c, cx, cy, cz);
                const long long n = (long long)x + (long long)nx * (y + (long long)ny * z);
#pragma unroll
                for (int ch = 0; ch < CH; ++ch) out[ch] = fmaf(w, __ldg(u + ch * N + n), out[ch]);
            }
        }
    }
}

// Box of acquisition voxels that can pull reconstruction voxel (x, y, z).
__device__ __forceinline__ void candidate_box(const ProjC& q, int x, int y, int z, int lo[3],
                                              int hi[3])
{
    const int md[3] = {q.mx, q.my, q.mz};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float a = fmaf(q.Ai[4 * d], (float)x, fmaf(q.Ai[4 * d + 1], (float)y, fmaf(q.Ai[4 * d + 2], (float)z, q.Ai[4 * d + 3])));
        const float e = q.ext[d] + 1e-3f;
        lo[d] = max(0, (int)ceilf(a - e));
        hi[d] = min(md[d] - 1, (int)floorf(a + e));
    }
}

// Calls f(w, m) for every acquisition voxel m of contrast q that pulls
// reconstruction voxel (x, y, z), with the weight the pull uses, in a fixed
// order (f is taken by value and returned).  Each coordinate is built with
// the same fused multiply-adds as reslice(), so every weight is bit-identical
// to the pull's; axes are tested one at a time and most candidates are
// rejected on the first.
template <typename F>
__device__ __forceinline__ F gather_pullers(const ProjC& q, int x, int y, int z, int nx, int ny,
                                            int nz, F f)
{
    int lo[3], hi[3];
    candidate_box(q, x, y, z, lo, hi);
    for (int k = lo[2]; k <= hi[2]; ++k)
        for (int j = lo[1]; j <= hi[1]; ++j)
            for (int i = lo[0]; i <= hi[0]; ++i) {
                const float r0 = fmaf(q.A[0], (float)i, fmaf(q.A[1], (float)j, fmaf(q.A[2], (float)k, q.A[3])));
                if (!(r0 >= 0.0f && r0 <= (float)(nx - 1))) continue;
                const float b0 = floorf(r0);
                const int dx = x - (int)b0;
                if ((unsigned)dx > 1u) continue;
                const float r1 = fmaf(q.A[4], (float)i, fmaf(q.A[5], (float)j, fmaf(q.A[6], (float)k, q.A[7])));
                if (!(r1 >= 0.0f && r1 <= (float)(ny - 1))) continue;
                const float b1 = floorf(r1);
                const int dy = y - (int)b1;
                if ((unsigned)dy > 1u) continue;
                const float r2 = fmaf(q.A[8], (float)i, fmaf(q.A[9], (float)j, fmaf(q.A[10], (float)k, q.A[11])));
                if (!(r2 >= 0.0f && r2 <= (float)(nz - 1))) continue;
                const float b2 = floorf(r2);
                const int dz = z - (int)b2;
                if ((unsigned)dz > 1u) continue;
                Cell c;
                c.f[0] = r0 - b0;
                c.f[1] = r1 - b1;
                c.f[2] = r2 - b2;
                const float w = corner_weight(c, dx, dy, dz);
                if (w == 0.0f) continue;
                f(w, (long long)i + (long long)q.mx * (j + (long long)q.my * k));
            }
    return f;
}

// ------------------------------------------------- projected voxel pass

template <int K, int PRE, typename XT>
__global__ void __launch_bounds__(kBlock) k_grad_hess_proj(DevProblem P, ProjC q, int c,
                                                           const float* __restrict__ y,
                                                           const XT* __restrict__ x,
                                                           const float* __restrict__ b1p,
                                                           const float* __restrict__ b1m,
                                                           float4* __restrict__ gh, double* nll,
                                                           Reduce red)
{
    constexpr int T = K * (K + 1) / 2;
    using GS = GhStride<K>;
    // each warp's 32 voxels are staged here and written as one contiguous run
    __shared__ float4 stage[kBlock / 32][32 * GS::V];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const long long M = q.M;
    const long long sxy = (long long)q.mx * q.my;
    Acc nll_acc;
    // the loop runs whole warps (all lanes the same number of times)
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long trips = (M + stride - 1) / stride;
    for (long long it = 0; it < trips; ++it) {
        const long long m0 = it * stride + blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31);
        const long long m = m0 + lane;
        const bool live = m < M;
        if (m + stride < M) {   // the next trip's echoes and B1 values into L2
            for (int e = 0; e < P.n_echoes[c]; ++e) prefetch_l2(x + e * M + m + stride);
            if (b1p) prefetch_l2(b1p + m + stride);
            if (b1m) prefetch_l2(b1m + m + stride);
        }
        const int i = (int)(m % q.mx), j = (int)((m / q.mx) % q.my), k = (int)(m / sxy);
        float G[K], H[T];
#pragma unroll
        for (int t = 0; t < K; ++t) G[t] = 0.0f;
#pragma unroll
        for (int t = 0; t < T; ++t) H[t] = 0.0f;
        float nll_v = 0.0f;
        float r[3];
        if (live && reslice(q, i, j, k, P.nx, P.ny, P.nz, r)) {
            float yv[K];
            interpolate<K>(cell_of(r), y, P.N, P.nx, P.ny, P.nz, yv);
            float yk[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int t = 0; t < K; ++t) yk[t] = yv[t];
            float a, r1, r2, dl, mm;
            map_params_v(yk, K, a, r1, r2, dl, mm);
            const float bp = b1p ? __ldg(b1p + m) : 1.0f;
            const float bm = b1m ? __ldg(b1m + m) : 1.0f;
            const ContrastTerms ct = contrast_terms(P, c, a, relax(P.tr[c], r1), dl, mm, bp, bm);
            accumulate_contrast<K, PRE, XT>(P, c, ct, r2, x + m, M, G, H, nll_v);
        }
        float o[GS::S];
#pragma unroll
        for (int t = 0; t < K; ++t) o[t] = G[t];
#pragma unroll
        for (int t = 0; t < T; ++t) o[K + t] = H[t];
#pragma unroll
        for (int t = K + T; t < GS::S; ++t) o[t] = 0.0f;
#pragma unroll
        for (int v = 0; v < GS::V; ++v)
            stage[wp][lane * GS::V + v] = make_float4(o[4 * v], o[4 * v + 1], o[4 * v + 2], o[4 * v + 3]);
        __syncwarp();
        const long long end = M * GS::V;                 // float4 entries of the buffer
#pragma unroll
        for (int v = 0; v < GS::V; ++v) {
            const long long e = m0 * GS::V + v * 32 + lane;
            if (e < end) gh[e] = stage[wp][v * 32 + lane];
        }
        __syncwarp();
        nll_acc.add(nll_v);
    }
    Acc v[1] = {nll_acc};
    double out[1];
    if (grid_reduce<1>(v, red, out) && threadIdx.x == 0) *nll = out[0];
}

__device__ __forceinline__ float lane4(const float4& e, int u)
{
    return u == 0 ? e.x : u == 1 ? e.y : u == 2 ? e.z : e.w;
}

// g = sum_c Psi_c' g_c, h = sum_c Psi_c' H_c; nll = sum_c nll_c (fixed order).
template <int K>
__global__ void __launch_bounds__(kBlock, 4) k_push_all(DevProblem P, DevProj Q, ProjBufs B,
                                                     float* __restrict__ g, float* __restrict__ h,
                                                     const double* nll_parts, double* nll)
{
    using GS = GhStride<K>;
    constexpr int T = K * (K + 1) / 2;
    constexpr int CH = K + T;                     // channels: g, then the packed H
    const long long N = P.N;
    const long long sxy = (long long)P.nx * P.ny;
    if (blockIdx.x == 0 && threadIdx.x == 0 && nll) {
        double s = 0.0;
        for (int c = 0; c < Q.C; ++c) s += nll_parts[c];
        *nll = s;
    }
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % P.nx), y = (int)((n / P.nx) % P.ny), z = (int)(n / sxy);
        float A[CH];
#pragma unroll
        for (int t = 0; t < CH; ++t) A[t] = 0.0f;
        // unrolled, so each contrast's affine is read as constant operands
#pragma unroll
        for (int c = 0; c < MPM_MAX_CONTRASTS; ++c) {
            if (c >= Q.C) break;
            const ProjC& q = Q.c[c];
            const float4* __restrict__ src = B.gh[c];
            auto add = [&](float w, long long m) {
#pragma unroll
                for (int v = 0; v < GS::V; ++v) {
                    const float4 e = __ldg(src + m * GS::V + v);
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (4 * v + u < CH) A[4 * v + u] = fmaf(w, lane4(e, u), A[4 * v + u]);
                }
            };
            gather_pullers(q, x, y, z, P.nx, P.ny, P.nz, add);
        }
#pragma unroll
        for (int t = 0; t < K; ++t) g[t * N + n] = A[t];
#pragma unroll
        for (int t = 0; t < T; ++t) h[t * N + n] = A[K + t];
    }
}

// ---------------------------------------------- Psi and Psi' on their own

__global__ void __launch_bounds__(kBlock) k_pull(DevProblem P, ProjC q, int channels,
                                                 const float* __restrict__ u,
                                                 float* __restrict__ out)
{
    const long long M = q.M;
    const long long sxy = (long long)q.mx * q.my;
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < M;
         m += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(m % q.mx), j = (int)((m / q.mx) % q.my), k = (int)(m / sxy);
        float r[3];
        const bool in = reslice(q, i, j, k, P.nx, P.ny, P.nz, r);
        const Cell cl = cell_of(r);
        for (int ch = 0; ch < channels; ++ch) {
            float v[1] = {0.0f};
            if (in) interpolate<1>(cl, u + ch * P.N, P.N, P.nx, P.ny, P.nz, v);
            out[ch * M + m] = v[0];
        }
    }
}

// Running sum of w * u[m] for one channel.
struct SumInto {
    float s;
    const float* __restrict__ u;
    __device__ __forceinline__ void operator()(float w, long long m) { s = fmaf(w, __ldg(u + m), s); }
};

__global__ void __launch_bounds__(kBlock) k_push(DevProblem P, ProjC q, int channels,
                                                 const float* __restrict__ u,
                                                 float* __restrict__ out, int accumulate)
{
    const long long N = P.N, M = q.M;
    const long long sxy = (long long)P.nx * P.ny;
    const long long total = N * channels;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
         id += (long long)gridDim.x * blockDim.x) {
        const long long ch = id / N, n = id - ch * N;
        const int x = (int)(n % P.nx), y = (int)((n / P.nx) % P.ny), z = (int)(n / sxy);
        SumInto acc{accumulate ? out[id] : 0.0f, u + ch * M};
        acc = gather_pullers(q, x, y, z, P.nx, P.ny, P.nz, acc);
        out[id] = acc.s;
    }
}

// ------------------------------------------------------------------ host

static mpm_status make_proj(const mpm_problem* p, const mpm_projection* proj, DevProj& Q)
{
    if (!proj) return fail(MPM_ERR_INVALID_ARG, "projection is NULL");
    memset(&Q, 0, sizeof Q);
    Q.C = p->n_contrasts;
    for (int c = 0; c < Q.C; ++c) {
        ProjC& q = Q.c[c];
        q.mx = proj->dims[c][0];
        q.my = proj->dims[c][1];
        q.mz = proj->dims[c][2];
        if (q.mx < 1 || q.my < 1 || q.mz < 1)
            return fail(MPM_ERR_INVALID_ARG, "contrast %d: acquisition grid %d x %d x %d", c, q.mx,
                        q.my, q.mz);
        q.M = (long long)q.mx * q.my * q.mz;
        const double* A = proj->affine[c];
        for (int t = 0; t < 12; ++t)
            if (!std::isfinite(A[t]) || std::fabs(A[t]) > 1e7)
                return fail(MPM_ERR_INVALID_ARG, "contrast %d: affine entry %d is not finite", c, t);
        // inverse of the linear part by the adjugate, in double
        const double a = A[0], b = A[1], cc = A[2], d = A[4], e = A[5], f = A[6], g = A[8],
                     h = A[9], i = A[10];
        const double det = a * (e * i - f * h) - b * (d * i - f * g) + cc * (d * h - e * g);
        const double scale = std::fabs(a) + std::fabs(b) + std::fabs(cc) + std::fabs(d) +
                             std::fabs(e) + std::fabs(f) + std::fabs(g) + std::fabs(h) + std::fabs(i);
        if (!(std::fabs(det) > 1e-9 * scale * scale * scale))
            return fail(MPM_ERR_INVALID_ARG, "contrast %d: affine is singular", c);
        double L[9] = {(e * i - f * h) / det,  (cc * h - b * i) / det, (b * f - cc * e) / det,
                       (f * g - d * i) / det,  (a * i - cc * g) / det, (cc * d - a * f) / det,
                       (d * h - e * g) / det,  (b * g - a * h) / det,  (a * e - b * d) / det};
        for (int r = 0; r < 3; ++r) {
            double t = 0.0, ex = 0.0;
            for (int s = 0; s < 3; ++s) {
                t -= L[3 * r + s] * A[4 * s + 3];
                ex += std::fabs(L[3 * r + s]);
            }
            // a reconstruction voxel gathers from a box of 2 ext + 1 acquisition
            // voxels per axis: acquisition voxels at least a quarter of the
            // reconstruction voxel size keep it at 9 or fewer
            if (ex > 4.0)
                return fail(MPM_ERR_INVALID_ARG,
                            "contrast %d: acquisition voxels more than 4x smaller than the "
                            "reconstruction voxels along axis %d (inverse affine row sum %.3g)",
                            c, r, ex);
            for (int s = 0; s < 3; ++s) q.Ai[4 * r + s] = (float)L[3 * r + s];
            q.Ai[4 * r + 3] = (float)t;
            q.ext[r] = (float)ex;
            for (int s = 0; s < 4; ++s) q.A[4 * r + s] = (float)A[4 * r + s];
        }
    }
    return MPM_OK;
}

// Workspace of the projected calls: the plain layout of `call` for the
// reconstruction grid, then the contrasts' NLL parts and g_c / H_c buffers.
struct ProjWs {
    FitWs L;
    double* nll_parts;
    float4* gh[MPM_MAX_CONTRASTS];
    size_t total;
};

static ProjWs proj_layout(const DevProblem& P, const DevProj& Q, int call, void* base)
{
    ProjWs W;
    memset(&W, 0, sizeof W);
    W.L = layout(P, call, base);
    size_t off = W.L.total;
    char* b = static_cast<char*>(base);
    auto take = [&](size_t bytes) -> char* {
        char* p = b ? b + off : nullptr;
        off += (bytes + 255) & ~(size_t)255;
        return p;
    };
    W.nll_parts = reinterpret_cast<double*>(take(sizeof(double) * MPM_MAX_CONTRASTS));
    for (int c = 0; c < Q.C; ++c) {
        W.gh[c] = reinterpret_cast<float4*>(take(sizeof(float) * (size_t)gh_floats(P.K) * Q.c[c].M));
    }
    W.total = off;
    return W;
}

template <int K, int PRE>
static cudaError_t grad_hess_proj_k(const DevProblem& P, const DevProj& Q, const ProjIn& in,
                                    const float* y, const ProjWs& W, float* g, float* h,
                                    double* nll, Reduce red, cudaStream_t st)
{
    for (int c = 0; c < Q.C; ++c) {
        const int grid = voxel_grid(Q.c[c].M);
        LaunchScope ls(MPM_KERNEL_GRAD_HESS_PROJ, st);
        if (in.echo_dtype == 1)
            k_grad_hess_proj<K, PRE, __nv_bfloat16><<<grid, kBlock, 0, st>>>(
                P, Q.c[c], c, y, static_cast<const __nv_bfloat16*>(in.x[c]), in.b1p[c], in.b1m[c],
                W.gh[c], W.nll_parts + c, red);
        else
            k_grad_hess_proj<K, PRE, float><<<grid, kBlock, 0, st>>>(
                P, Q.c[c], c, y, static_cast<const float*>(in.x[c]), in.b1p[c], in.b1m[c],
                W.gh[c], W.nll_parts + c, red);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    ProjBufs B;
    memset(&B, 0, sizeof B);
    for (int c = 0; c < Q.C; ++c) {
        B.gh[c] = W.gh[c];
    }
    LaunchScope ls(MPM_KERNEL_RESLICE, st);
    k_push_all<K><<<voxel_grid(P.N), kBlock, 0, st>>>(P, Q, B, g, h, W.nll_parts, nll);
    return cudaGetLastError();
}

template <int K>
static cudaError_t grad_hess_proj_pre(const DevProblem& P, const DevProj& Q, const ProjIn& in,
                                      const float* y, const ProjWs& W, float* g, float* h,
                                      double* nll, Reduce red, cudaStream_t st)
{
    if (P.precond == 1) return grad_hess_proj_k<K, 1>(P, Q, in, y, W, g, h, nll, red, st);
    if (P.precond == 2) return grad_hess_proj_k<K, 2>(P, Q, in, y, W, g, h, nll, red, st);
    return grad_hess_proj_k<K, 0>(P, Q, in, y, W, g, h, nll, red, st);
}

cudaError_t launch_grad_hess_proj(const DevProblem& P, const ProjJob& pj, const float* y, float* g,
                                  float* h, double* nll, Reduce red, cudaStream_t st)
{
    const DevProj& Q = *static_cast<const DevProj*>(pj.Q);
    const ProjWs& W = *static_cast<const ProjWs*>(pj.W);
    if (P.K == 4) return grad_hess_proj_pre<4>(P, Q, pj.in, y, W, g, h, nll, red, st);
    return grad_hess_proj_pre<3>(P, Q, pj.in, y, W, g, h, nll, red, st);
}

}  // namespace mpm

using namespace mpm;

namespace {

mpm_status check_proj_inputs(const mpm_problem* problem, const DevProj& Q, const void* const* x,
                             const float* const* b1p, const float* const* b1m, ProjIn& in)
{
    if (!x) return fail(MPM_ERR_INVALID_ARG, "x (array of per-contrast pointers) is NULL");
    memset(&in, 0, sizeof in);
    in.echo_dtype = problem->echo_dtype;
    const size_t ealign = problem->echo_dtype ? 2 : 4;
    for (int c = 0; c < Q.C; ++c) {
        char name[32];
        snprintf(name, sizeof name, "x[%d]", c);
        MPM_TRY(check_dev(x[c], name, false, ealign));
        in.x[c] = x[c];
        in.b1p[c] = b1p ? b1p[c] : nullptr;
        in.b1m[c] = b1m ? b1m[c] : nullptr;
        snprintf(name, sizeof name, "b1p[%d]", c);
        MPM_TRY(check_dev(in.b1p[c], name, true, 4));
        snprintf(name, sizeof name, "b1m[%d]", c);
        MPM_TRY(check_dev(in.b1m[c], name, true, 4));
    }
    return MPM_OK;
}

}  // namespace

extern "C" {

mpm_status mpm_workspace_size_proj(const mpm_problem* problem, const mpm_projection* proj,
                                   const mpm_opts* opts, int call, size_t* bytes)
{
    if (!bytes) return fail(MPM_ERR_INVALID_ARG, "bytes is NULL");
    MPM_TRY(check_problem(problem));
    if (call != MPM_CALL_FIT && call != MPM_CALL_GRAD_HESS)
        return fail(MPM_ERR_INVALID_ARG, "call must be MPM_CALL_FIT or MPM_CALL_GRAD_HESS");
    if (call == MPM_CALL_FIT) MPM_TRY(check_opts(opts));
    DevProj Q;
    MPM_TRY(make_proj(problem, proj, Q));
    *bytes = proj_layout(make_dev(problem), Q, call, nullptr).total;
    return MPM_OK;
}

mpm_status mpm_pull(const mpm_problem* problem, const mpm_projection* proj, int contrast,
                    int channels, const float* u, float* out, void* stream)
{
    MPM_TRY(check_problem(problem));
    DevProj Q;
    MPM_TRY(make_proj(problem, proj, Q));
    if (contrast < 0 || contrast >= Q.C)
        return fail(MPM_ERR_INVALID_ARG, "contrast %d outside [0, %d)", contrast, Q.C);
    if (channels < 1) return fail(MPM_ERR_INVALID_ARG, "channels must be >= 1");
    MPM_TRY(check_dev(u, "u", false, 4));
    MPM_TRY(check_dev(out, "out", false, 4));
    const DevProblem P = make_dev(problem);
    if (P.N == 0) return MPM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    LaunchScope ls(MPM_KERNEL_RESLICE, st);
    k_pull<<<voxel_grid(Q.c[contrast].M), kBlock, 0, st>>>(P, Q.c[contrast], channels, u, out);
    MPM_CUDA(cudaGetLastError());
    return MPM_OK;
}

mpm_status mpm_push(const mpm_problem* problem, const mpm_projection* proj, int contrast,
                    int channels, const float* u, float* out, int accumulate, void* stream)
{
    MPM_TRY(check_problem(problem));
    DevProj Q;
    MPM_TRY(make_proj(problem, proj, Q));
    if (contrast < 0 || contrast >= Q.C)
        return fail(MPM_ERR_INVALID_ARG, "contrast %d outside [0, %d)", contrast, Q.C);
    if (channels < 1) return fail(MPM_ERR_INVALID_ARG, "channels must be >= 1");
    MPM_TRY(check_dev(u, "u", false, 4));
    MPM_TRY(check_dev(out, "out", false, 4));
    const DevProblem P = make_dev(problem);
    if (P.N == 0) return MPM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    LaunchScope ls(MPM_KERNEL_RESLICE, st);
    k_push<<<voxel_grid(P.N), kBlock, 0, st>>>(P, Q.c[contrast], channels, u, out, accumulate);
    MPM_CUDA(cudaGetLastError());
    return MPM_OK;
}

mpm_status mpm_grad_hess_proj(const mpm_problem* problem, const mpm_projection* proj,
                              const void* const* x, const float* const* b1p,
                              const float* const* b1m, const float* y, float* g, float* h,
                              double* nll, void* ws, size_t ws_bytes, void* stream)
{
    MPM_TRY(check_problem(problem));
    DevProj Q;
    MPM_TRY(make_proj(problem, proj, Q));
    ProjIn in;
    MPM_TRY(check_proj_inputs(problem, Q, x, b1p, b1m, in));
    MPM_TRY(check_dev(y, "y", false, 4));
    MPM_TRY(check_dev(g, "g", false, 4));
    MPM_TRY(check_dev(h, "h", false, 4));
    MPM_TRY(check_dev(nll, "nll", false, 8));
    const DevProblem P = make_dev(problem);
    if (P.N == 0) return MPM_OK;
    const ProjWs need = proj_layout(P, Q, MPM_CALL_GRAD_HESS, nullptr);
    if (ws_bytes < need.total)
        return fail(MPM_ERR_WORKSPACE_TOO_SMALL, "workspace of %zu bytes, %zu needed", ws_bytes,
                    need.total);
    MPM_TRY(check_dev(ws, "ws", false, 256));
    const ProjWs W = proj_layout(P, Q, MPM_CALL_GRAD_HESS, ws);
    DevProj Qm = Q;
    cudaStream_t st = (cudaStream_t)stream;
    MPM_CUDA(cudaMemsetAsync(W.L.hdr, 0, sizeof(WsHeader), st));
    ProjWs Wm = W;
    ProjJob pj;
    pj.Q = &Qm;
    pj.W = &Wm;
    pj.in = in;
    MPM_CUDA(launch_grad_hess_proj(P, pj, y, g, h, nll, W.L.red, st));
    return MPM_OK;
}

}  // extern "C"

namespace mpm {

// Pieces of mpm_fit_proj that live with the projection: validation, the
// workspace layout and the image means over the acquisition grids.
mpm_status proj_prepare(const mpm_problem* problem, const mpm_projection* proj, const void* const* x,
                        const float* const* b1p, const float* const* b1m, void* ws, size_t ws_bytes,
                        ProjJob& pj, FitWs& L)
{
    DevProj* Q = new DevProj;
    ProjWs* W = new ProjWs;
    pj.Q = Q;
    pj.W = W;
    MPM_TRY(make_proj(problem, proj, *Q));
    MPM_TRY(check_proj_inputs(problem, *Q, x, b1p, b1m, pj.in));
    const DevProblem P = make_dev(problem);
    const ProjWs need = proj_layout(P, *Q, MPM_CALL_FIT, nullptr);
    if (ws_bytes < need.total)
        return fail(MPM_ERR_WORKSPACE_TOO_SMALL, "workspace of %zu bytes, %zu needed", ws_bytes,
                    need.total);
    MPM_TRY(check_dev(ws, "ws", false, 256));
    *W = proj_layout(P, *Q, MPM_CALL_FIT, ws);
    L = W->L;
    return MPM_OK;
}

void proj_release(ProjJob& pj)
{
    delete static_cast<DevProj*>(pj.Q);
    delete static_cast<ProjWs*>(pj.W);
    pj.Q = pj.W = nullptr;
}

size_t proj_key_bytes() { return sizeof(DevProj); }

// Bytes that identify a projected fit in the graph cache.
void proj_key(const ProjJob& pj, std::string& k)
{
    k.append(static_cast<const char*>(pj.Q), sizeof(DevProj));
    k.append(reinterpret_cast<const char*>(&pj.in), sizeof(ProjIn));
}

// Image means of every contrast over its own acquisition grid, written to
// means[echo0[c] + e].
cudaError_t proj_image_means(const DevProblem& P, const ProjJob& pj, double* parts, double* means,
                             cudaStream_t st)
{
    const DevProj& Q = *static_cast<const DevProj*>(pj.Q);
    for (int c = 0; c < Q.C; ++c) {
        DevProblem Pc = P;
        Pc.nx = Q.c[c].mx;
        Pc.ny = Q.c[c].my;
        Pc.nz = Q.c[c].mz;
        Pc.N = Q.c[c].M;
        Pc.I = P.n_echoes[c];
        cudaError_t e = launch_image_means(Pc, pj.in.echo_dtype, pj.in.x[c], parts, means + P.echo0[c], st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace mpm
