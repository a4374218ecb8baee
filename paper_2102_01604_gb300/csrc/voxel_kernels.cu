// voxel_kernels.cu -- per-voxel kernels of the MPM library (sm_103a):
//   k_forward       noise-free images (Eq. 26 with the B1 footnote)
//   k_grad_hess     the fused voxel pass: signal, residual, gradient and the
//                   approximate Hessian of Eq. 24, NLL reduced in float64
//   k_uncertainty   diagonal of the inverse preconditioner blocks (Eq. 43),
//                   log-determinant, log-normal moments (Eqs. 44-47); float32
//                   on equilibrated blocks, float64 for ill-conditioned ones
//   k_image_means / k_means_final / k_init_maps   constant initial maps
//
// One thread per voxel (grid-stride), or two neighbouring voxels per thread in
// the voxel pass; images are read as planes [I][N], so each warp loads 128
// (256) contiguous bytes per echo.
#include "init_maps.cuh"
#include "mpm_internal.cuh"
#include "voxel_model.cuh"

namespace mpm {

// ------------------------------------------------------------ forward model

__global__ void __launch_bounds__(kBlock) k_forward(DevProblem P, const float* __restrict__ y,
                                                    const float* __restrict__ b1p,
                                                    const float* __restrict__ b1m,
                                                    float* __restrict__ s)
{
    const long long N = P.N;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        float a, r1, r2, dl, m;
        map_params(y, N, n, P.K, a, r1, r2, dl, m);
        const float bp = b1p ? __ldg(b1p + n) : 1.0f;
        for (int c = 0; c < P.C; ++c) {
            const float bm = b1m ? __ldg(b1m + c * N + n) : 1.0f;
            const ContrastTerms t = contrast_terms(P, c, a, relax(P.tr[c], r1), dl, m, bp, bm);
            const int i0 = P.echo0[c];
            for (int e = 0; e < P.n_echoes[c]; ++e)
                s[(i0 + e) * N + n] = t.s0 * expf(-P.te[i0 + e] * r2);
        }
    }
}

// ------------------------------------------------------ fused voxel pass

// Hint voxel n (the next one of this thread's grid-stride loop, n < N) into
// L2: its echoes, maps and B1 values, so that their DRAM latency overlaps the
// arithmetic of the current voxel.
template <typename XT>
__device__ __forceinline__ void prefetch_voxel(const DevProblem& P, const XT* x, const float* y,
                                               const float* b1p, const float* b1m, long long n)
{
    const long long N = P.N;
    for (int i = 0; i < P.I; ++i) prefetch_l2(x + i * N + n);
    for (int k = 0; k < P.K; ++k) prefetch_l2(y + k * N + n);
    if (b1p) prefetch_l2(b1p + n);
    if (b1m)
        for (int c = 0; c < P.C; ++c) prefetch_l2(b1m + c * N + n);
}

// The fused voxel pass: per voxel, accumulate_contrast for every contrast.
// Each thread takes V neighbouring voxels per grid-stride step (V divides N,
// every array aligned to V elements), reading each plane with one V-wide load;
// every voxel's arithmetic is the same for V = 1 and V = 2.
template <int K, int PRE, typename XT, int V>
__device__ __forceinline__ void grad_hess_body(const DevProblem& P, const XT* __restrict__ x,
                                               const float* __restrict__ y,
                                               const float* __restrict__ b1p,
                                               const float* __restrict__ b1m, float* __restrict__ g,
                                               float* __restrict__ h, double* nll, Reduce red,
                                               const VGrid& vg)
{
    constexpr int T = K * (K + 1) / 2;
    const long long N = P.N;
    const long long NV = N / V;
    const long long step = (long long)vg.gx * blockDim.x;
    Acc nll_acc;
    for (long long u = vg.bx * (long long)blockDim.x + threadIdx.x; u < NV; u += step) {
        const long long n = u * V;
        if (u + step < NV) prefetch_voxel<XT>(P, x, y, b1p, b1m, (u + step) * V);
        float a[V], r1[V], r2[V], dl[V], m[V], bp[V];
        {
            float yv[K][V];
#pragma unroll
            for (int k = 0; k < K; ++k) load_vec<V, float>(y + k * N + n, yv[k]);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                float yk[4];
#pragma unroll
                for (int k = 0; k < K; ++k) yk[k] = yv[k][v];
                map_params_v(yk, K, a[v], r1[v], r2[v], dl[v], m[v]);
            }
        }
        if (b1p) {
            load_vec<V, float>(b1p + n, bp);
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) bp[v] = 1.0f;
        }
        float G[V][K], H[V][T], nll_v[V];
        Relax R[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
#pragma unroll
            for (int k = 0; k < K; ++k) G[v][k] = 0.0f;
#pragma unroll
            for (int k = 0; k < T; ++k) H[v][k] = 0.0f;
            nll_v[v] = 0.0f;
            R[v] = Relax{0.f, 0.f, 0.f};
        }
        for (int c = 0; c < P.C; ++c) {
            float bm[V];
            if (b1m) {
                load_vec<V, float>(b1m + c * N + n, bm);
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) bm[v] = 1.0f;
            }
            ContrastTerms t[V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                if (!P.same_tr[c]) R[v] = relax(P.tr[c], r1[v]);
                t[v] = contrast_terms(P, c, a[v], R[v], dl[v], m[v], bp[v], bm[v]);
            }
            accumulate_contrast_v<K, PRE, XT, V>(P, c, t, r2, x + (long long)P.echo0[c] * N + n, N,
                                                 G, H, nll_v);
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            float o[V];
#pragma unroll
            for (int v = 0; v < V; ++v) o[v] = G[v][k];
            store_vec<V>(g + k * N + n, o);
        }
#pragma unroll
        for (int k = 0; k < T; ++k) {
            float o[V];
#pragma unroll
            for (int v = 0; v < V; ++v) o[v] = H[v][k];
            store_vec<V>(h + k * N + n, o);
        }
#pragma unroll
        for (int v = 0; v < V; ++v) nll_acc.add(nll_v[v]);
    }
    Acc v[1] = {nll_acc};
    double out[1];
    if (grid_reduce<1>(v, red, out, vg) && threadIdx.x == 0) *nll = out[0];
}

// Two voxels per thread hold twice the state: half the resident blocks.
template <int V>
struct GradOcc {
    static constexpr int kMinBlocks = V == 1 ? 4 : 2;
};

template <int K, int PRE, typename XT, int V>
__global__ void __launch_bounds__(kBlock, GradOcc<V>::kMinBlocks)
    k_grad_hess(DevProblem P, const XT* __restrict__ x, const float* __restrict__ y,
                const float* __restrict__ b1p, const float* __restrict__ b1m, float* __restrict__ g,
                float* __restrict__ h, double* nll, Reduce red)
{
    grad_hess_body<K, PRE, XT, V>(P, x, y, b1p, b1m, g, h, nll, red, hw_grid());
}

template <int K, int PRE, typename XT, int V>
__global__ void __launch_bounds__(kBlock, GradOcc<V>::kMinBlocks)
    k_grad_hess_batch(const __grid_constant__ Batch<GradArgs> b)
{
    const int s = batch_subject(b.start, b.n);
    const GradArgs& a = b.a[s];
    grad_hess_body<K, PRE, XT, V>(a.P, static_cast<const XT*>(a.x), a.y, a.b1p, a.b1m, a.g, a.h,
                                  a.nll, a.red,
                                  batch_grid(b.start[s], b.start[s + 1] - b.start[s], 1, 1));
}

// Whether the voxel pass may take two voxels per thread: N even and every
// array aligned to two elements (each plane then starts aligned too).
static bool pairs_ok(long long N, int echo_dtype, const void* x, const float* y, const float* b1p,
                     const float* b1m, const float* g, const float* h)
{
    auto al = [](const void* p, uintptr_t a) { return reinterpret_cast<uintptr_t>(p) % a == 0; };
    return N % 2 == 0 && al(x, echo_dtype == 1 ? 4 : 8) && al(y, 8) && al(b1p, 8) && al(b1m, 8) &&
           al(g, 8) && al(h, 8);
}

// --------------------------------------------------------- uncertainty

// 1 / sqrt(s) in float64 without a float64 square root or division: the
// float32 estimate refined by one Newton-Raphson step on f(r) = r^-2 - s,
// r <- r (3 - s r^2) / 2, which doubles its correct bits (about 22 -> 44, far
// beyond the float32 variances it feeds).  Outside the float32 range it falls
// back to 1 / sqrt(s).
__device__ __forceinline__ double rsqrt_newton(double s)
{
    if (!(s > 1e-30 && s < 1e30)) return 1.0 / sqrt(s);
    const double r = (double)rsqrtf((float)s);
    return r * (1.5 - 0.5 * s * r * r);
}

constexpr float kPivotMin = 1e-2f;   // smallest equilibrated pivot of the float32 path

// The diagonal of M^-1 and log det M of one block M (K x K, symmetric, float32
// entries) in float32, through the Cholesky factor L of the equilibrated block
// A = S M S, S = diag(s_k), s_k ~ M_kk^-1/2 (so A has a unit diagonal up to
// rounding): (M^-1)_kk = s_k^2 sum_j (L^-1)_jk^2 and log det M = sum_j log
// L_jj^2 - 2 sum_k log s_k.  M comes from float32 H and w, so its variances
// already carry a relative uncertainty of about kappa(M) 2^-24; the float32
// factorization adds about K kappa(A) 2^-24, and kappa(A) is of the order of
// 1 / (smallest pivot L_jj^2).  False, with nothing written, when a pivot is
// below kPivotMin (or M_kk is not positive): such blocks take block_var_f64.
template <int K>
__device__ __forceinline__ bool block_var_f32(const float (&M)[K][K], bool want_ld, float (&var)[K],
                                              float& ld)
{
    float sc[K];
#pragma unroll
    for (int a = 0; a < K; ++a) {
        if (!(M[a][a] > 0.0f)) return false;
        sc[a] = rsqrtf(M[a][a]);
    }
    float A[K][K];
#pragma unroll
    for (int a = 0; a < K; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) A[a][b] = M[a][b] * sc[a] * sc[b];
    float L[K][K], inv[K];
    float lsum = 0.0f;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        float p = A[j][j];
#pragma unroll
        for (int k = 0; k < j; ++k) p -= L[j][k] * L[j][k];
        if (!(p >= kPivotMin)) return false;
        inv[j] = rsqrtf(p);
        L[j][j] = p * inv[j];
        if (want_ld) lsum += logf(p) - 2.0f * logf(sc[j]);
#pragma unroll
        for (int i = j + 1; i < K; ++i) {
            float v = A[i][j];
#pragma unroll
            for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
            L[i][j] = v * inv[j];
        }
    }
    float Li[K][K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
#pragma unroll
        for (int i = 0; i < K; ++i) Li[i][j] = 0.0f;
        Li[j][j] = inv[j];
#pragma unroll
        for (int i = j + 1; i < K; ++i) {
            float v = 0.0f;
#pragma unroll
            for (int k = j; k < i; ++k) v -= L[i][k] * Li[k][j];
            Li[i][j] = v * inv[i];
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float v = 0.0f;
#pragma unroll
        for (int j = k; j < K; ++j) v += Li[j][k] * Li[j][k];
        var[k] = v * sc[k] * sc[k];
    }
    ld = lsum;
    return true;
}

// What block_var_f64 returns (by value, so that the float32 path keeps its
// values in registers).
struct BlockVar {
    float var[4];
    float ld;
    bool ok;          // false: a pivot was not positive
};

// The same in float64 (H_kk + lambda_k d in float64; dl_k = lambda_k d), for
// the blocks the float32 path declines.
template <int K>
__device__ __noinline__ BlockVar block_var_f64(const float* __restrict__ h, long long n, long long N,
                                               double dl0, double dl1, double dl2, double dl3, bool want_ld)
{
    BlockVar out;
    double M[K][K], L[K][K];
#pragma unroll
    for (int a = 0; a < K; ++a)
#pragma unroll
        for (int b = a; b < K; ++b) M[a][b] = M[b][a] = __ldg(h + tri(K, a, b) * N + n);
    const double dl[4] = {dl0, dl1, dl2, dl3};
#pragma unroll
    for (int a = 0; a < K; ++a) M[a][a] += dl[a];
    bool ok = true;
    double lsum = 0.0;              // log det M, only when asked (log in float64 is costly)
    double inv[K];                  // 1 / L_jj
#pragma unroll
    for (int j = 0; j < K; ++j) {
        double s = M[j][j];
#pragma unroll
        for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
        if (!(s > 0.0)) { ok = false; s = 1e-300; }
        inv[j] = rsqrt_newton(s);
        L[j][j] = s * inv[j];
        if (want_ld) lsum += log(s);
#pragma unroll
        for (int i = j + 1; i < K; ++i) {
            double v = M[i][j];
#pragma unroll
            for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
            L[i][j] = v * inv[j];
        }
    }
    double Li[K][K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
#pragma unroll
        for (int i = 0; i < K; ++i) Li[i][j] = 0.0;
        Li[j][j] = inv[j];
#pragma unroll
        for (int i = j + 1; i < K; ++i) {
            double v = 0.0;
#pragma unroll
            for (int k = j; k < i; ++k) v -= L[i][k] * Li[k][j];
            Li[i][j] = v * inv[i];
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double v = 0.0;
#pragma unroll
        for (int j = k; j < K; ++j) v += Li[j][k] * Li[j][k];
        out.var[k] = (float)v;
    }
    out.ld = (float)lsum;
    out.ok = ok;
    return out;
}

// (x, y, z) of voxel n.
__device__ __forceinline__ void voxel_coords(const DevProblem& P, long long n, int& x, int& yy, int& z)
{
    if (P.N <= 0xffffffffLL) {          // 32-bit division where the index fits
        const unsigned u = (unsigned)n, r = u / (unsigned)P.nx;
        x = (int)(u - r * (unsigned)P.nx);
        yy = (int)(r % (unsigned)P.ny);
        z = (int)(r / (unsigned)P.ny);
    } else {
        x = (int)(n % P.nx);
        yy = (int)((n / P.nx) % P.ny);
        z = (int)(n / ((long long)P.nx * P.ny));
    }
}

// Block n of the preconditioner, M = H_n + diag(lambda_k d_n) with
// d_n = sum_{m in N(n)} (w_n + w_m) / h^2: the diagonal of M^-1 (the
// posterior variances, Eq. 43), -log det M, and the log-normal moments of
// r1 = exp(y_R1) and t1 = 1 / r1 from the log-R1 variance (Eqs. 44-47).
// Each thread takes V neighbouring voxels (V = 2: N even, arrays 8-byte
// aligned), loading their H entries and weights as pairs before it inverts
// the blocks one by one, so that twice the bytes are in flight per thread.
template <int K, int V>
__device__ __forceinline__ void uncertainty_body(const DevProblem& P, const float* __restrict__ h,
                                                 const float* __restrict__ w, const float* __restrict__ y,
                                                 float* __restrict__ var, float* __restrict__ logdet,
                                                 float* __restrict__ moments, unsigned* status,
                                                 const VGrid& vg)
{
    constexpr int T = K * (K + 1) / 2;
    const long long N = P.N;
    const long long sxy = (long long)P.nx * P.ny;
    const long long units = N / V;
    for (long long u = vg.bx * (long long)blockDim.x + threadIdx.x; u < units;
         u += (long long)vg.gx * blockDim.x) {
        const long long n0 = u * V;
        float hv[T][V], wc[V];
#pragma unroll
        for (int t = 0; t < T; ++t) load_vec<V, float>(h + t * N + n0, hv[t]);
        load_vec<V, float>(w + n0, wc);
        float vv[V][K], ld[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const long long n = n0 + v;
            int x, yy, z;
            voxel_coords(P, n, x, yy, z);
            // d_n in float32 (six terms, relative error about 4e-7, far
            // inside the variance's tolerance); the pair's own weights serve
            // as each other's x neighbours
            const float wn = wc[v];
            float d32 = 0.0f;
            if (x > 0) d32 += (wn + (v > 0 ? wc[v - 1] : __ldg(w + n - 1))) * P.ihx2;
            if (x < P.nx - 1) d32 += (wn + (v + 1 < V ? wc[v + 1] : __ldg(w + n + 1))) * P.ihx2;
            if (yy > 0) d32 += (wn + __ldg(w + n - P.nx)) * P.ihy2;
            if (yy < P.ny - 1) d32 += (wn + __ldg(w + n + P.nx)) * P.ihy2;
            if (z > 0) d32 += (wn + __ldg(w + n - sxy)) * P.ihz2;
            if (z < P.nz - 1) d32 += (wn + __ldg(w + n + sxy)) * P.ihz2;
            float M[K][K];
#pragma unroll
            for (int a2 = 0; a2 < K; ++a2)
#pragma unroll
                for (int b2 = a2; b2 < K; ++b2) M[a2][b2] = M[b2][a2] = hv[tri(K, a2, b2)][v];
#pragma unroll
            for (int a2 = 0; a2 < K; ++a2) M[a2][a2] += P.lambda[a2] * d32;
            ld[v] = 0.0f;
            if (!block_var_f32<K>(M, logdet != nullptr, vv[v], ld[v])) {
                const double d = d32;
                const BlockVar b = block_var_f64<K>(h, n, N, P.lambda[0] * d, P.lambda[1] * d,
                                                    P.lambda[2] * d, K == 4 ? P.lambda[3] * d : 0.0,
                                                    logdet != nullptr);
#pragma unroll
                for (int k = 0; k < K; ++k) vv[v][k] = b.var[k];
                ld[v] = b.ld;
                if (!b.ok && status) atomicOr(status, kStatusNotPD);
            }
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            float o[V];
#pragma unroll
            for (int v = 0; v < V; ++v) o[v] = vv[v][k];
            store_vec<V>(var + k * N + n0, o);
        }
        if (logdet) {
            float o[V];
#pragma unroll
            for (int v = 0; v < V; ++v) o[v] = -ld[v];
            store_vec<V>(logdet + n0, o);
        }
        if (moments && y) {
            // E r1 = exp(y + s2 / 2), Var r1 = (exp(s2) - 1) exp(2 y + s2); t1 with -y
            float lr1[V], m[4][V];
            load_vec<V, float>(y + N + n0, lr1);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const float s2 = vv[v][1], em1 = expm1f(s2);
                m[0][v] = expf(fmaf(0.5f, s2, lr1[v]));
                m[1][v] = em1 * expf(fmaf(2.0f, lr1[v], s2));
                m[2][v] = expf(fmaf(0.5f, s2, -lr1[v]));
                m[3][v] = em1 * expf(fmaf(-2.0f, lr1[v], s2));
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) store_vec<V>(moments + j * N + n0, m[j]);
        }
    }
}

template <int K, int V>
__global__ void __launch_bounds__(kBlock) k_uncertainty(DevProblem P, const float* __restrict__ h,
                                                        const float* __restrict__ w,
                                                        const float* __restrict__ y,
                                                        float* __restrict__ var,
                                                        float* __restrict__ logdet,
                                                        float* __restrict__ moments,
                                                        unsigned* status)
{
    uncertainty_body<K, V>(P, h, w, y, var, logdet, moments, status, hw_grid());
}

template <int K, int V>
__global__ void __launch_bounds__(kBlock) k_uncertainty_batch(const __grid_constant__ Batch<UncArgs> b)
{
    const int s = batch_subject(b.start, b.n);
    const UncArgs& a = b.a[s];
    uncertainty_body<K, V>(a.P, a.h, a.w, a.y, a.var, a.logdet, a.moments, a.status,
                        batch_grid(b.start[s], b.start[s + 1] - b.start[s], 1, 1));
}

// -------------------------------------------------- constant initial maps

constexpr int kMeanBlocks = 304;

template <typename XT>
__global__ void __launch_bounds__(kBlock) k_image_means(DevProblem P, const XT* __restrict__ x,
                                                        double* partials)
{
    __shared__ double sh[kBlock / 32];
    const long long N = P.N;
    const int i = blockIdx.y;
    Acc acc;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x)
        acc.add(load_echo<XT>(x, i * N + n));
    const double tot = block_acc(acc, sh);
    if (threadIdx.x == 0) partials[i * gridDim.x + blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kBlock) k_means_final(DevProblem P, const double* partials,
                                                        int nparts, double* means)
{
    __shared__ double sh[kBlock / 32];
    const int i = blockIdx.x;
    double acc = 0.0;
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) acc += partials[i * nparts + b];
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) means[i] = acc / (double)P.N;
}

// The starting maps from the image means: each block's first thread derives
// the K values (a few hundred float64 operations) and the block fills its
// share of the maps.
__global__ void __launch_bounds__(kBlock) k_init_maps(DevProblem P, const double* __restrict__ means,
                                                      float* __restrict__ y)
{
    __shared__ float v[4];
    if (threadIdx.x == 0) initial_map_values(P, means, v);
    __syncthreads();
    const long long total = P.N * P.K;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x)
        y[i] = v[i / P.N];
}

// ------------------------------------------------------------- launchers

cudaError_t launch_forward(const DevProblem& P, const float* y, const float* b1p,
                           const float* b1m, float* s, cudaStream_t st)
{
    LaunchScope ls(MPM_KERNEL_FORWARD, st);
    k_forward<<<voxel_grid(P.N), kBlock, 0, st>>>(P, y, b1p, b1m, s);
    return cudaGetLastError();
}

template <int K, int PRE, int V>
static void grad_hess_v(const DevProblem& P, int echo_dtype, const void* x, const float* y,
                        const float* b1p, const float* b1m, float* g, float* h, double* nll,
                        Reduce red, cudaStream_t st)
{
    const int grid = voxel_grid(P.N / V);
    if (echo_dtype == 1)
        k_grad_hess<K, PRE, __nv_bfloat16, V><<<grid, kBlock, 0, st>>>(
            P, static_cast<const __nv_bfloat16*>(x), y, b1p, b1m, g, h, nll, red);
    else
        k_grad_hess<K, PRE, float, V><<<grid, kBlock, 0, st>>>(
            P, static_cast<const float*>(x), y, b1p, b1m, g, h, nll, red);
}

template <int K, int PRE>
static void grad_hess_dtype(const DevProblem& P, int echo_dtype, const void* x,
                            const float* y, const float* b1p, const float* b1m, float* g,
                            float* h, double* nll, Reduce red, cudaStream_t st)
{
    if (pairs_ok(P.N, echo_dtype, x, y, b1p, b1m, g, h))
        grad_hess_v<K, PRE, 2>(P, echo_dtype, x, y, b1p, b1m, g, h, nll, red, st);
    else
        grad_hess_v<K, PRE, 1>(P, echo_dtype, x, y, b1p, b1m, g, h, nll, red, st);
}

template <int K>
static void grad_hess_pre(const DevProblem& P, int echo_dtype, const void* x, const float* y,
                          const float* b1p, const float* b1m, float* g, float* h,
                          double* nll, Reduce red, cudaStream_t st)
{
    switch (P.precond) {
    case 0: grad_hess_dtype<K, 0>(P, echo_dtype, x, y, b1p, b1m, g, h, nll, red, st); break;
    case 1: grad_hess_dtype<K, 1>(P, echo_dtype, x, y, b1p, b1m, g, h, nll, red, st); break;
    default: grad_hess_dtype<K, 2>(P, echo_dtype, x, y, b1p, b1m, g, h, nll, red, st); break;
    }
}

cudaError_t launch_grad_hess(const DevProblem& P, int echo_dtype, const void* x,
                             const float* y, const float* b1p, const float* b1m, float* g,
                             float* h, double* nll, Reduce red, unsigned* status, cudaStream_t st)
{
    LaunchScope ls(MPM_KERNEL_GRAD_HESS, st);
    if (grad_hess_tma_ok(P, x, y, b1p, b1m, g, h))
        return launch_grad_hess_tma(P, echo_dtype, x, y, b1p, b1m, g, h, nll, red, status, st);
    if (P.K == 4)
        grad_hess_pre<4>(P, echo_dtype, x, y, b1p, b1m, g, h, nll, red, st);
    else
        grad_hess_pre<3>(P, echo_dtype, x, y, b1p, b1m, g, h, nll, red, st);
    return cudaGetLastError();
}

// Whether the uncertainty pass may take two voxels per thread: N even and
// every array it reads or writes 8-byte aligned.
static bool unc_pairs_ok(const DevProblem& P, const float* h, const float* w, const float* y,
                         const float* var, const float* logdet, const float* moments)
{
    auto al = [](const void* p) { return reinterpret_cast<uintptr_t>(p) % 8 == 0; };
    return P.N % 2 == 0 && al(h) && al(w) && al(y) && al(var) && al(logdet) && al(moments);
}

cudaError_t launch_uncertainty(const DevProblem& P, const float* h, const float* w,
                               const float* y, float* var, float* logdet, float* moments,
                               unsigned* status, cudaStream_t st)
{
    LaunchScope ls(MPM_KERNEL_UNCERTAINTY, st);
    const bool pairs = unc_pairs_ok(P, h, w, y, var, logdet, moments);
    const int grid = voxel_grid(pairs ? P.N / 2 : P.N);
#define MPM_UNC(KK, VV) k_uncertainty<KK, VV><<<grid, kBlock, 0, st>>>(P, h, w, y, var, logdet, moments, status)
    if (P.K == 4) {
        if (pairs) MPM_UNC(4, 2); else MPM_UNC(4, 1);
    } else {
        if (pairs) MPM_UNC(3, 2); else MPM_UNC(3, 1);
    }
#undef MPM_UNC
    return cudaGetLastError();
}

template <int K, int PRE, int V>
static void grad_hess_batch_v(int echo_dtype, const Batch<GradArgs>& b, cudaStream_t st)
{
    const unsigned grid = b.start[b.n];
    if (echo_dtype == 1)
        k_grad_hess_batch<K, PRE, __nv_bfloat16, V><<<grid, kBlock, 0, st>>>(b);
    else
        k_grad_hess_batch<K, PRE, float, V><<<grid, kBlock, 0, st>>>(b);
}

template <int K, int PRE>
static void grad_hess_batch_dtype(int echo_dtype, const Batch<GradArgs>& b, cudaStream_t st)
{
    bool pairs = true;
    for (int i = 0; i < b.n; ++i) {
        const GradArgs& a = b.a[i];
        pairs = pairs && pairs_ok(a.P.N, echo_dtype, a.x, a.y, a.b1p, a.b1m, a.g, a.h);
    }
    if (pairs)
        grad_hess_batch_v<K, PRE, 2>(echo_dtype, b, st);
    else
        grad_hess_batch_v<K, PRE, 1>(echo_dtype, b, st);
}

template <int K>
static void grad_hess_batch_pre(int precond, int echo_dtype, const Batch<GradArgs>& b, cudaStream_t st)
{
    switch (precond) {
    case 0: grad_hess_batch_dtype<K, 0>(echo_dtype, b, st); break;
    case 1: grad_hess_batch_dtype<K, 1>(echo_dtype, b, st); break;
    default: grad_hess_batch_dtype<K, 2>(echo_dtype, b, st); break;
    }
}

cudaError_t launch_grad_hess_batch(int K, int precond, int echo_dtype, const GradArgs* a,
                                   const unsigned* blocks, int n, cudaStream_t st)
{
    // The staged pass splits its own wave between the subjects; otherwise
    // blocks[s] is sized for one voxel per thread, and with two the blocks'
    // grid-stride loops take half the steps.
    LaunchScope ls(MPM_KERNEL_GRAD_HESS, st);
    cudaError_t e;
    if (launch_grad_hess_tma_batch(K, precond, echo_dtype, a, n, st, &e)) return e;
    Batch<GradArgs> b;
    fill_batch(b, a, blocks, n);
    if (K == 4)
        grad_hess_batch_pre<4>(precond, echo_dtype, b, st);
    else
        grad_hess_batch_pre<3>(precond, echo_dtype, b, st);
    return cudaGetLastError();
}

cudaError_t launch_uncertainty_batch(int K, const UncArgs* a, const unsigned* blocks, int n,
                                     cudaStream_t st)
{
    Batch<UncArgs> b;
    fill_batch(b, a, blocks, n);
    bool pairs = true;
    for (int i = 0; i < n; ++i)
        pairs = pairs && unc_pairs_ok(a[i].P, a[i].h, a[i].w, a[i].y, a[i].var, a[i].logdet, a[i].moments);
    LaunchScope ls(MPM_KERNEL_UNCERTAINTY, st);
    if (K == 4) {
        if (pairs) k_uncertainty_batch<4, 2><<<b.start[n], kBlock, 0, st>>>(b);
        else k_uncertainty_batch<4, 1><<<b.start[n], kBlock, 0, st>>>(b);
    } else {
        if (pairs) k_uncertainty_batch<3, 2><<<b.start[n], kBlock, 0, st>>>(b);
        else k_uncertainty_batch<3, 1><<<b.start[n], kBlock, 0, st>>>(b);
    }
    return cudaGetLastError();
}

cudaError_t launch_image_means(const DevProblem& P, int echo_dtype, const void* x,
                               double* partials, double* means, cudaStream_t st)
{
    long long want = (P.N + kBlock - 1) / kBlock;
    const int nb = (int)(want < kMeanBlocks ? want : kMeanBlocks);
    dim3 grid(nb, P.I);
    {
        LaunchScope ls(MPM_KERNEL_INIT, st);
        if (echo_dtype == 1)
            k_image_means<__nv_bfloat16><<<grid, kBlock, 0, st>>>(
                P, static_cast<const __nv_bfloat16*>(x), partials);
        else
            k_image_means<float><<<grid, kBlock, 0, st>>>(P, static_cast<const float*>(x),
                                                          partials);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    LaunchScope ls(MPM_KERNEL_INIT, st);
    k_means_final<<<P.I, kBlock, 0, st>>>(P, partials, nb, means);
    return cudaGetLastError();
}

cudaError_t launch_init_maps(const DevProblem& P, const double* means, float* y, cudaStream_t st)
{
    LaunchScope ls(MPM_KERNEL_INIT, st);
    k_init_maps<<<voxel_grid(P.N * P.K), kBlock, 0, st>>>(P, means, y);
    return cudaGetLastError();
}

}  // namespace mpm
