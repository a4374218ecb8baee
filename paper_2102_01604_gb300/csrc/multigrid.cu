// multigrid.cu -- conjugate gradient on the Newton system (H + L) delta =
// g + L y (Eq. 42) with an aggregation multigrid V-cycle as the
// preconditioner, an option beside the paper's block preconditioner
// (opts.mg_levels > 0; the paper's solver is the block-Jacobi PCG of
// stencil_kernels.cu / stencil_tma.cu).
//
// The hierarchy, rebuilt for every solve from H and the JTV weights:
//   - level 0 is the volume, with the edge coefficients of L,
//     kappa_a[n] = (w_n + w_{n + e_a}) / h_a^2 for the edge to the +a neighbour
//     (0 at the far face);
//   - level l + 1 merges 2 x 2 x 2 voxels of level l (ceil(n / 2) per axis); a
//     level of at most kMgMinVoxels voxels is the coarsest;
//   - prolongation copies a coarse voxel's value to its children, restriction
//     sums over them; the coarse operator is the Galerkin product P' A P,
//     which keeps the form of A: H summed over the children, and each coarse
//     edge coefficient the sum of the fine edge coefficients crossing it.
// Smoother: damped block-Jacobi x += omega D^-1 (r - A x), with D the 4 x 4
// voxel blocks H + diag(lambda_k sum of the six edge coefficients) (on level 0
// exactly the paper's preconditioner block).  V-cycle from x = 0: nu sweeps,
// coarse correction with the restricted residual, nu sweeps; the coarsest
// level takes coarse_sweeps sweeps.  Equal sweeps on both sides make the
// cycle symmetric, so plain CG may use it.
//
// Vectors are voxel-interleaved (float4 per voxel, the fourth component zero
// for K = 3); H and kappa are planar.  CG scalars stay on the device (last
// block of each reducing launch), so a solve runs without host round trips and
// can be captured in a graph.
#include <utility>

#include "mpm_internal.cuh"
#include "pcg_step.cuh"

namespace mpm {

constexpr long long kMgMinVoxels = 512;
constexpr int kMgMaxLevels = 16;

struct MgLevel {
    int nx, ny, nz;
    long long N;
    const float* h;     // [T][N]
    float* kap;         // [3][N]
    float4* r;          // right-hand side of this level's cycle
    float4* x;          // result of this level's cycle
    float4* t;          // ping-pong partner of x for the sweeps
};

struct MgBufs {
    int L;                       // levels
    MgLevel lv[kMgMaxLevels];
    float4 *cx, *cp[2], *cq;     // CG: delta, directions (ping-pong), (H + L) p; r is lv[0].r, z is lv[0].x
};

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// Level dimensions: ceil(n / 2) per axis until a level has at most
// kMgMinVoxels voxels or `levels` levels exist.
static int mg_dims(const DevProblem& P, int levels, int (*dims)[3])
{
    int n[3] = {P.nx, P.ny, P.nz};
    int L = 0;
    if (levels > kMgMaxLevels) levels = kMgMaxLevels;
    for (;;) {
        dims[L][0] = n[0];
        dims[L][1] = n[1];
        dims[L][2] = n[2];
        ++L;
        if (L >= levels || (long long)n[0] * n[1] * n[2] <= kMgMinVoxels) break;
        for (int a = 0; a < 3; ++a) n[a] = (n[a] + 1) / 2;
    }
    return L;
}

// Carves the multigrid buffers from `ws` (NULL: sizes only); returns bytes.
static size_t mg_carve(const DevProblem& P, int levels, void* ws, MgBufs* B)
{
    int dims[kMgMaxLevels][3];
    const int L = mg_dims(P, levels, dims);
    char* base = static_cast<char*>(ws);
    size_t off = 0;
    auto take = [&](size_t bytes) -> void* {
        void* p = base ? base + off : nullptr;
        off += al256(bytes);
        return p;
    };
    MgBufs b;
    b.L = L;
    for (int l = 0; l < L; ++l) {
        MgLevel& v = b.lv[l];
        v.nx = dims[l][0];
        v.ny = dims[l][1];
        v.nz = dims[l][2];
        v.N = (long long)v.nx * v.ny * v.nz;
        v.h = l == 0 ? nullptr : static_cast<const float*>(take(sizeof(float) * P.T * v.N));
        v.kap = static_cast<float*>(take(sizeof(float) * 3 * v.N));
        v.r = static_cast<float4*>(take(sizeof(float4) * v.N));
        v.x = static_cast<float4*>(take(sizeof(float4) * v.N));
        v.t = static_cast<float4*>(take(sizeof(float4) * v.N));
    }
    b.cx = static_cast<float4*>(take(sizeof(float4) * P.N));
    b.cp[0] = static_cast<float4*>(take(sizeof(float4) * P.N));
    b.cp[1] = static_cast<float4*>(take(sizeof(float4) * P.N));
    b.cq = static_cast<float4*>(take(sizeof(float4) * P.N));
    if (B) *B = b;
    return off;
}

size_t mg_ws_bytes(const DevProblem& P) { return mg_carve(P, kMgMaxLevels, nullptr, nullptr); }

// ------------------------------------------------------------ per voxel

// The six edge coefficients of voxel (x, y, z) of a level (order x-, x+, y-,
// y+, z-, z+; 0 where the neighbour is outside) and the neighbours' offsets.
__device__ __forceinline__ void level_edges(const MgLevel& L, int x, int y, int z, long long n,
                                            float (&c)[6], long long (&off)[6])
{
    const long long sxy = (long long)L.nx * L.ny;
    const float* kx = L.kap;
    const float* ky = L.kap + L.N;
    const float* kz = L.kap + 2 * L.N;
    off[0] = -1;      c[0] = x > 0 ? kx[n - 1] : 0.0f;
    off[1] = 1;       c[1] = x + 1 < L.nx ? kx[n] : 0.0f;
    off[2] = -L.nx;   c[2] = y > 0 ? ky[n - L.nx] : 0.0f;
    off[3] = L.nx;    c[3] = y + 1 < L.ny ? ky[n] : 0.0f;
    off[4] = -sxy;    c[4] = z > 0 ? kz[n - sxy] : 0.0f;
    off[5] = sxy;     c[5] = z + 1 < L.nz ? kz[n] : 0.0f;
}

__device__ __forceinline__ void voxel_xyz(const MgLevel& L, long long n, int& x, int& y, int& z)
{
    x = (int)(n % L.nx);
    y = (int)((n / L.nx) % L.ny);
    z = (int)(n / ((long long)L.nx * L.ny));
}

// (A v)_n on a level: H_n v_n + lambda_k sum_m c_m (v_n - v_m).
template <int K>
__device__ __forceinline__ void level_apply(const DevProblem& P, const float (&hv)[K * (K + 1) / 2],
                                            const float (&c)[6], const long long (&off)[6], long long n,
                                            const float4* __restrict__ v, float (&out)[K])
{
    float vn[K];
    unpack4<K>(v[n], vn);
    float lap[K];
#pragma unroll
    for (int a = 0; a < K; ++a) lap[a] = 0.0f;
#pragma unroll
    for (int m = 0; m < 6; ++m) {
        if (c[m] != 0.0f) {
            float vm[K];
            unpack4<K>(v[n + off[m]], vm);
#pragma unroll
            for (int a = 0; a < K; ++a) lap[a] = fmaf(c[m], vn[a] - vm[a], lap[a]);
        }
    }
#pragma unroll
    for (int a = 0; a < K; ++a) {
        float acc = P.lambda[a] * lap[a];
#pragma unroll
        for (int b = 0; b < K; ++b) acc = fmaf(hv[a < b ? tri(K, a, b) : tri(K, b, a)], vn[b], acc);
        out[a] = acc;
    }
}

template <int K>
__device__ __forceinline__ void load_h(const MgLevel& L, const float* h0, long long n,
                                       float (&hv)[K * (K + 1) / 2])
{
    const float* h = L.h ? L.h : h0;
#pragma unroll
    for (int t = 0; t < K * (K + 1) / 2; ++t) hv[t] = __ldg(h + t * L.N + n);
}

__device__ __forceinline__ bool solve_done(const WsHeader* hdr) { return hdr->sc.done != 0; }

// ------------------------------------------------------------ hierarchy

// Level 0 edge coefficients from the JTV weights.
__global__ void __launch_bounds__(kBlock) k_mg_kappa0(DevProblem P, MgLevel L, const float* __restrict__ w)
{
    const long long sxy = (long long)L.nx * L.ny;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < L.N;
         n += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        voxel_xyz(L, n, x, y, z);
        const float wn = __ldg(w + n);
        L.kap[n] = x + 1 < L.nx ? (wn + __ldg(w + n + 1)) * P.ihx2 : 0.0f;
        L.kap[L.N + n] = y + 1 < L.ny ? (wn + __ldg(w + n + L.nx)) * P.ihy2 : 0.0f;
        L.kap[2 * L.N + n] = z + 1 < L.nz ? (wn + __ldg(w + n + sxy)) * P.ihz2 : 0.0f;
    }
}

// Galerkin coarse level: H summed over the children, each coarse edge the
// sum of the fine edges crossing it (those of the children on the +a side).
__global__ void __launch_bounds__(kBlock) k_mg_coarsen(DevProblem P, MgLevel F, MgLevel C,
                                                       const float* h0)
{
    const int T = P.T;
    const float* fh = F.h ? F.h : h0;
    float* ch = const_cast<float*>(C.h);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < C.N;
         c += (long long)gridDim.x * blockDim.x) {
        int cx, cy, cz;
        voxel_xyz(C, c, cx, cy, cz);
        float hs[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        float ks[3] = {0, 0, 0};
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                    const int fx = 2 * cx + dx, fy = 2 * cy + dy, fz = 2 * cz + dz;
                    if (fx >= F.nx || fy >= F.ny || fz >= F.nz) continue;
                    const long long f = fx + (long long)F.nx * (fy + (long long)F.ny * fz);
                    for (int t = 0; t < T; ++t) hs[t] += __ldg(fh + t * F.N + f);
                    if (dx == 1 && fx + 1 < F.nx) ks[0] += F.kap[f];
                    if (dy == 1 && fy + 1 < F.ny) ks[1] += F.kap[F.N + f];
                    if (dz == 1 && fz + 1 < F.nz) ks[2] += F.kap[2 * F.N + f];
                }
        for (int t = 0; t < T; ++t) ch[t * C.N + c] = hs[t];
        for (int a = 0; a < 3; ++a) C.kap[a * C.N + c] = ks[a];
    }
}

// ------------------------------------------------------------ V-cycle

// One damped block-Jacobi sweep on a level: xout = xin + omega D^-1 (r - A xin)
// (FIRST: xin = 0, so xout = omega D^-1 r).
template <int K, bool FIRST>
__global__ void __launch_bounds__(kBlock) k_mg_sweep(DevProblem P, MgLevel L, const float* h0,
                                                     float omega, const float4* __restrict__ xin,
                                                     float4* __restrict__ xout, const WsHeader* hdr)
{
    constexpr int T = K * (K + 1) / 2;
    if (solve_done(hdr)) return;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < L.N;
         n += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        voxel_xyz(L, n, x, y, z);
        float c[6];
        long long off[6];
        level_edges(L, x, y, z, n, c, off);
        float hv[T];
        load_h<K>(L, h0, n, hv);
        float b[K];
        unpack4<K>(L.r[n], b);
        if (!FIRST) {
            float ax[K];
            level_apply<K>(P, hv, c, off, n, xin, ax);
#pragma unroll
            for (int a = 0; a < K; ++a) b[a] -= ax[a];
        }
        float M[K][K], Lf[T], e[K];
        precond_block<K>(P, hv, edge_sum(c), M);
        cholesky_f32<K>(M, Lf);
        chol_apply<K>(Lf, b, e);
        float xo[K];
        if (FIRST) {
#pragma unroll
            for (int a = 0; a < K; ++a) xo[a] = omega * e[a];
        } else {
            unpack4<K>(xin[n], xo);
#pragma unroll
            for (int a = 0; a < K; ++a) xo[a] = fmaf(omega, e[a], xo[a]);
        }
        xout[n] = pack4<K>(xo);
    }
}

// Restricted residual: C.r = P' (F.r - A_F x), one coarse voxel per thread
// summing its children in a fixed order.
template <int K>
__global__ void __launch_bounds__(kBlock) k_mg_restrict(DevProblem P, MgLevel F, MgLevel C, const float* h0,
                                                        const float4* __restrict__ xf, const WsHeader* hdr)
{
    constexpr int T = K * (K + 1) / 2;
    if (solve_done(hdr)) return;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < C.N;
         c += (long long)gridDim.x * blockDim.x) {
        int cx, cy, cz;
        voxel_xyz(C, c, cx, cy, cz);
        float acc[K];
#pragma unroll
        for (int a = 0; a < K; ++a) acc[a] = 0.0f;
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dx = 0; dx < 2; ++dx) {
                    const int fx = 2 * cx + dx, fy = 2 * cy + dy, fz = 2 * cz + dz;
                    if (fx >= F.nx || fy >= F.ny || fz >= F.nz) continue;
                    const long long f = fx + (long long)F.nx * (fy + (long long)F.ny * fz);
                    float cf[6];
                    long long off[6];
                    level_edges(F, fx, fy, fz, f, cf, off);
                    float hv[T], ax[K], r[K];
                    load_h<K>(F, h0, f, hv);
                    level_apply<K>(P, hv, cf, off, f, xf, ax);
                    unpack4<K>(F.r[f], r);
#pragma unroll
                    for (int a = 0; a < K; ++a) acc[a] += r[a] - ax[a];
                }
        C.r[c] = pack4<K>(acc);
    }
}

// x_F += P x_C: each fine voxel adds its parent's value.
__global__ void __launch_bounds__(kBlock) k_mg_prolong(MgLevel F, MgLevel C, float4* __restrict__ xf,
                                                       const WsHeader* hdr)
{
    if (solve_done(hdr)) return;
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < F.N;
         f += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        voxel_xyz(F, f, x, y, z);
        const long long c = (x / 2) + (long long)C.nx * ((y / 2) + (long long)C.ny * (z / 2));
        const float4 e = C.x[c];
        float4 v = xf[f];
        v.x += e.x;
        v.y += e.y;
        v.z += e.z;
        v.w += e.w;
        xf[f] = v;
    }
}

// The coarsest level in one block: `sweeps` damped block-Jacobi sweeps from
// zero, ping-ponging between L.x and L.t (result in L.x after an even count of
// buffer swaps, else copied there).
template <int K>
__global__ void __launch_bounds__(512) k_mg_coarsest(DevProblem P, MgLevel L, const float* h0, float omega,
                                                      int sweeps, const WsHeader* hdr)
{
    constexpr int T = K * (K + 1) / 2;
    if (solve_done(hdr)) return;
    float4* bufs[2] = {L.x, L.t};
    for (int s = 0; s < sweeps; ++s) {
        const float4* xin = bufs[(s + 1) & 1];
        float4* xout = bufs[s & 1];
        for (long long n = threadIdx.x; n < L.N; n += blockDim.x) {
            int x, y, z;
            voxel_xyz(L, n, x, y, z);
            float c[6];
            long long off[6];
            level_edges(L, x, y, z, n, c, off);
            float hv[T];
            load_h<K>(L, h0, n, hv);
            float b[K];
            unpack4<K>(L.r[n], b);
            float xo[K];
            if (s > 0) {
                float ax[K];
                level_apply<K>(P, hv, c, off, n, xin, ax);
#pragma unroll
                for (int a = 0; a < K; ++a) b[a] -= ax[a];
                unpack4<K>(xin[n], xo);
            } else {
#pragma unroll
                for (int a = 0; a < K; ++a) xo[a] = 0.0f;
            }
            float M[K][K], Lf[T], e[K];
            precond_block<K>(P, hv, edge_sum(c), M);
            cholesky_f32<K>(M, Lf);
            chol_apply<K>(Lf, b, e);
#pragma unroll
            for (int a = 0; a < K; ++a) xo[a] = fmaf(omega, e[a], xo[a]);
            xout[n] = pack4<K>(xo);
        }
        __syncthreads();
    }
    if (sweeps > 0 && ((sweeps - 1) & 1)) {
        for (long long n = threadIdx.x; n < L.N; n += blockDim.x) L.x[n] = L.t[n];
    }
}

// ------------------------------------------------------------ CG

// r = g + L y (L from the JTV weights), |r_0|^2; scalars reset.
template <int K>
__global__ void __launch_bounds__(kBlock) k_mgcg_init(DevProblem P, MgLevel L0, const float* __restrict__ g,
                                                      const float* __restrict__ y, double tol2,
                                                      WsHeader* hdr, double* resid, Reduce red)
{
    Acc rr;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < L0.N;
         n += (long long)gridDim.x * blockDim.x) {
        int x, yy, z;
        voxel_xyz(L0, n, x, yy, z);
        float c[6];
        long long off[6];
        level_edges(L0, x, yy, z, n, c, off);
        float r[K];
        float vr = 0.0f;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float* yk = y + k * P.N;
            const float v = __ldg(yk + n);
            float s = 0.0f;
#pragma unroll
            for (int m = 0; m < 6; ++m)
                if (c[m] != 0.0f) s = fmaf(c[m], v - __ldg(yk + n + off[m]), s);
            r[k] = __ldg(g + k * P.N + n) + P.lambda[k] * s;
            vr = fmaf(r[k], r[k], vr);
        }
        L0.r[n] = pack4<K>(r);
        rr.add(vr);
    }
    Acc v[1] = {rr};
    double out[1];
    if (grid_reduce<1>(v, red, out) && threadIdx.x == 0) {
        SolveScalars& sc = hdr->sc;
        sc.rr0 = out[0];
        sc.rr = out[0];
        sc.rz = 0.0;
        sc.alpha = 0.0;
        sc.alpha_prev = 0.0;
        sc.beta = 0.0;
        sc.it = 0;
        sc.xcount = 0;
        sc.tol2 = tol2;
        const bool bad = !(out[0] == out[0]);
        if (bad) atomicOr(&hdr->status, kStatusNaN);
        sc.done = (bad || !(out[0] > 0.0)) ? 1 : 0;
        if (resid) resid[0] = sqrt(out[0]);
    }
}

// rz = r . z and beta = rz / rz_previous (first: beta unused).
template <int K>
__global__ void __launch_bounds__(kBlock) k_mgcg_rz(long long N, const float4* __restrict__ r,
                                                    const float4* __restrict__ z, int first,
                                                    WsHeader* hdr, Reduce red)
{
    if (solve_done(hdr)) return;
    Acc acc;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        float a[K], b[K];
        unpack4<K>(r[n], a);
        unpack4<K>(z[n], b);
        float s = a[0] * b[0];
#pragma unroll
        for (int k = 1; k < K; ++k) s = fmaf(a[k], b[k], s);
        acc.add(s);
    }
    Acc v[1] = {acc};
    double out[1];
    if (grid_reduce<1>(v, red, out) && threadIdx.x == 0) {
        SolveScalars& sc = hdr->sc;
        if (!(out[0] == out[0])) atomicOr(&hdr->status, kStatusNaN);
        if (!(out[0] > 0.0)) {
            sc.done = 1;
            return;
        }
        sc.beta = first ? 0.0 : out[0] / sc.rz;
        sc.rz = out[0];
    }
}

// p = z + beta p_old (at the voxel and its neighbours), q = (H + L) p, p . q;
// alpha = rz / p.q.
template <int K>
__global__ void __launch_bounds__(kBlock) k_mgcg_matvec(DevProblem P, MgLevel L0, const float* h0,
                                                        const float4* __restrict__ pold,
                                                        float4* __restrict__ pnew, float4* __restrict__ q,
                                                        int first, WsHeader* hdr, Reduce red)
{
    constexpr int T = K * (K + 1) / 2;
    __shared__ float s_beta;
    __shared__ int s_done;
    if (threadIdx.x == 0) {
        s_done = hdr->sc.done;
        s_beta = (float)hdr->sc.beta;
    }
    __syncthreads();
    if (s_done) return;
    const float beta = s_beta;
    const float4* z = L0.x;
    auto dir = [&](long long m, float (&pm)[K]) {
        float zm[K];
        unpack4<K>(z[m], zm);
        if (first) {
#pragma unroll
            for (int a = 0; a < K; ++a) pm[a] = zm[a];
        } else {
            float po[K];
            unpack4<K>(pold[m], po);
#pragma unroll
            for (int a = 0; a < K; ++a) pm[a] = fmaf(beta, po[a], zm[a]);
        }
    };
    Acc acc;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < L0.N;
         n += (long long)gridDim.x * blockDim.x) {
        int x, y, zz;
        voxel_xyz(L0, n, x, y, zz);
        float c[6];
        long long off[6];
        level_edges(L0, x, y, zz, n, c, off);
        float pn[K], lap[K];
        dir(n, pn);
#pragma unroll
        for (int a = 0; a < K; ++a) lap[a] = 0.0f;
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            if (c[m] != 0.0f) {
                float pm[K];
                dir(n + off[m], pm);
#pragma unroll
                for (int a = 0; a < K; ++a) lap[a] = fmaf(c[m], pn[a] - pm[a], lap[a]);
            }
        }
        float hv[T], qn[K];
        load_h<K>(L0, h0, n, hv);
        float s = 0.0f;
#pragma unroll
        for (int a = 0; a < K; ++a) {
            float v = P.lambda[a] * lap[a];
#pragma unroll
            for (int b = 0; b < K; ++b) v = fmaf(hv[a < b ? tri(K, a, b) : tri(K, b, a)], pn[b], v);
            qn[a] = v;
            s = fmaf(pn[a], v, s);
        }
        pnew[n] = pack4<K>(pn);
        q[n] = pack4<K>(qn);
        acc.add(s);
    }
    Acc v[1] = {acc};
    double out[1];
    if (grid_reduce<1>(v, red, out) && threadIdx.x == 0) {
        SolveScalars& sc = hdr->sc;
        if (!(out[0] == out[0])) atomicOr(&hdr->status, kStatusNaN);
        if (!(out[0] > 0.0)) {
            sc.done = 1;                 // no step; the solve keeps its x
            return;
        }
        sc.alpha = sc.rz / out[0];
    }
}

// x += alpha p, r -= alpha q, |r|^2; the iteration counter and the tolerance.
template <int K>
__global__ void __launch_bounds__(kBlock) k_mgcg_update(long long N, int j, float4* __restrict__ xacc,
                                                        const float4* __restrict__ p,
                                                        const float4* __restrict__ q,
                                                        float4* __restrict__ r, WsHeader* hdr,
                                                        double* resid, Reduce red)
{
    __shared__ float s_alpha;
    __shared__ int s_done;
    if (threadIdx.x == 0) {
        s_done = hdr->sc.done;
        s_alpha = (float)hdr->sc.alpha;
    }
    __syncthreads();
    if (s_done) return;
    const float alpha = s_alpha;
    Acc acc;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        float xv[K], pv[K], qv[K], rv[K];
        unpack4<K>(p[n], pv);
        unpack4<K>(q[n], qv);
        unpack4<K>(r[n], rv);
        if (j == 0) {
#pragma unroll
            for (int a = 0; a < K; ++a) xv[a] = 0.0f;
        } else {
            unpack4<K>(xacc[n], xv);
        }
        float s = 0.0f;
#pragma unroll
        for (int a = 0; a < K; ++a) {
            xv[a] = fmaf(alpha, pv[a], xv[a]);
            rv[a] = fmaf(-alpha, qv[a], rv[a]);
            s = fmaf(rv[a], rv[a], s);
        }
        xacc[n] = pack4<K>(xv);
        r[n] = pack4<K>(rv);
        acc.add(s);
    }
    Acc v[1] = {acc};
    double out[1];
    if (grid_reduce<1>(v, red, out) && threadIdx.x == 0) {
        SolveScalars& sc = hdr->sc;
        if (!(out[0] == out[0])) atomicOr(&hdr->status, kStatusNaN);
        sc.rr = out[0];
        sc.it = j + 1;
        if (resid) resid[j + 1] = sqrt(out[0]);
        if (!(out[0] == out[0]) || (sc.tol2 > 0.0 && out[0] <= sc.tol2 * sc.rr0)) sc.done = 1;
    }
}

// delta = x (planar), or y <- y - x; the report.
template <int K>
__global__ void __launch_bounds__(kBlock) k_mgcg_final(long long N, const float4* __restrict__ xacc,
                                                       float* __restrict__ delta,
                                                       float* __restrict__ y_update, const WsHeader* hdr,
                                                       double* report_rel, int* report_it)
{
    const SolveScalars sc = hdr->sc;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        float v[K];
        if (sc.it > 0) {
            unpack4<K>(xacc[n], v);
        } else {
#pragma unroll
            for (int a = 0; a < K; ++a) v[a] = 0.0f;
        }
#pragma unroll
        for (int a = 0; a < K; ++a) {
            if (y_update)
                y_update[a * N + n] -= v[a];
            else
                delta[a * N + n] = v[a];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (report_rel) *report_rel = sc.rr0 > 0.0 ? sqrt(sc.rr / sc.rr0) : 0.0;
        if (report_it) *report_it = sc.it;
    }
}

// ------------------------------------------------------------ host

template <int K>
static void vcycle(const DevProblem& P, const MgBufs& B, int l, const float* h0, const SolveOpts& o,
                   WsHeader* hdr, cudaStream_t st)
{
    const MgLevel& Lv = B.lv[l];
    const int grid = voxel_grid(Lv.N);
    if (l == B.L - 1) {
        if (Lv.N <= 8192) {
            LaunchScope ls(MPM_KERNEL_MG, st);
            k_mg_coarsest<K><<<1, 512, 0, st>>>(P, Lv, h0, o.mg_omega, o.mg_coarse_sweeps, hdr);
        } else {
            // a large coarsest level (few levels asked for): one launch per sweep
            float4* bufs[2] = {Lv.x, Lv.t};
            for (int s = 0; s < o.mg_coarse_sweeps; ++s) {
                LaunchScope ls(MPM_KERNEL_MG, st);
                if (s == 0)
                    k_mg_sweep<K, true><<<grid, kBlock, 0, st>>>(P, Lv, h0, o.mg_omega, Lv.x, bufs[0], hdr);
                else
                    k_mg_sweep<K, false><<<grid, kBlock, 0, st>>>(P, Lv, h0, o.mg_omega, bufs[(s + 1) & 1],
                                                                  bufs[s & 1], hdr);
            }
            if (o.mg_coarse_sweeps > 0 && ((o.mg_coarse_sweeps - 1) & 1))
                cudaMemcpyAsync(Lv.x, Lv.t, sizeof(float4) * Lv.N, cudaMemcpyDeviceToDevice, st);
        }
        return;
    }
    // pre-smoothing: the result ends in `cur`.  The first sweep writes in
    // place and every later sweep swaps, 2 nu - 1 swaps in all, so starting
    // from t the cycle's result lands in x.
    float4* cur = Lv.t;
    float4* other = Lv.x;
    for (int s = 0; s < o.mg_nu; ++s) {
        LaunchScope ls(MPM_KERNEL_MG, st);
        if (s == 0) {
            k_mg_sweep<K, true><<<grid, kBlock, 0, st>>>(P, Lv, h0, o.mg_omega, cur, cur, hdr);
        } else {
            k_mg_sweep<K, false><<<grid, kBlock, 0, st>>>(P, Lv, h0, o.mg_omega, cur, other, hdr);
            std::swap(cur, other);
        }
    }
    const MgLevel& C = B.lv[l + 1];
    {
        LaunchScope ls(MPM_KERNEL_MG, st);
        k_mg_restrict<K><<<voxel_grid(C.N), kBlock, 0, st>>>(P, Lv, C, h0, cur, hdr);
    }
    vcycle<K>(P, B, l + 1, h0, o, hdr, st);
    {
        LaunchScope ls(MPM_KERNEL_MG, st);
        k_mg_prolong<<<grid, kBlock, 0, st>>>(Lv, C, cur, hdr);
    }
    for (int s = 0; s < o.mg_nu; ++s) {
        LaunchScope ls(MPM_KERNEL_MG, st);
        k_mg_sweep<K, false><<<grid, kBlock, 0, st>>>(P, Lv, h0, o.mg_omega, cur, other, hdr);
        std::swap(cur, other);
    }
    if (cur != Lv.x) {
        // the level's result must be in x
        cudaMemcpyAsync(Lv.x, cur, sizeof(float4) * Lv.N, cudaMemcpyDeviceToDevice, st);
    }
}

template <int K>
static cudaError_t solve_mg_k(const DevProblem& P, const SolveOpts& o, const float* h, const float* w,
                              const float* g, const float* y, float* delta, float* y_update,
                              double* resid, double* report_rel, int* report_it, void* solve_ws,
                              WsHeader* hdr, Reduce red, cudaStream_t st)
{
    MgBufs B;
    mg_carve(P, o.mg_levels, solve_ws, &B);
    MgLevel L0 = B.lv[0];
    const int grid = voxel_grid(P.N);
    const double tol2 = o.tol_cg > 0.0 ? o.tol_cg * o.tol_cg : 0.0;
    {
        LaunchScope ls(MPM_KERNEL_MG, st);
        k_mg_kappa0<<<grid, kBlock, 0, st>>>(P, L0, w);
    }
    for (int l = 0; l + 1 < B.L; ++l) {
        LaunchScope ls(MPM_KERNEL_MG, st);
        k_mg_coarsen<<<voxel_grid(B.lv[l + 1].N), kBlock, 0, st>>>(P, B.lv[l], B.lv[l + 1], h);
    }
    {
        LaunchScope ls(MPM_KERNEL_PCG_INIT, st);
        k_mgcg_init<K><<<grid, kBlock, 0, st>>>(P, L0, g, y, tol2, hdr, resid, red);
    }
    vcycle<K>(P, B, 0, h, o, hdr, st);
    {
        LaunchScope ls(MPM_KERNEL_PCG_STEP, st);
        k_mgcg_rz<K><<<grid, kBlock, 0, st>>>(P.N, L0.r, L0.x, 1, hdr, red);
    }
    for (int j = 0; j < o.cg_iters; ++j) {
        float4* pold = B.cp[(j + 1) & 1];
        float4* pnew = B.cp[j & 1];
        {
            LaunchScope ls(MPM_KERNEL_PCG_STEP, st);
            k_mgcg_matvec<K><<<grid, kBlock, 0, st>>>(P, L0, h, pold, pnew, B.cq, j == 0, hdr, red);
        }
        {
            LaunchScope ls(MPM_KERNEL_PCG_STEP, st);
            k_mgcg_update<K><<<grid, kBlock, 0, st>>>(P.N, j, B.cx, pnew, B.cq, L0.r, hdr, resid, red);
        }
        if (j + 1 < o.cg_iters) {
            vcycle<K>(P, B, 0, h, o, hdr, st);
            LaunchScope ls(MPM_KERNEL_PCG_STEP, st);
            k_mgcg_rz<K><<<grid, kBlock, 0, st>>>(P.N, L0.r, L0.x, 0, hdr, red);
        }
    }
    LaunchScope ls(MPM_KERNEL_PCG_FINAL, st);
    k_mgcg_final<K><<<grid, kBlock, 0, st>>>(P.N, B.cx, delta, y_update, hdr, report_rel, report_it);
    return cudaGetLastError();
}

cudaError_t launch_solve_mg(const DevProblem& P, const SolveOpts& o, const float* h, const float* w,
                            const float* g, const float* y, float* delta, float* y_update,
                            double* resid, double* report_rel, int* report_it, void* solve_ws,
                            WsHeader* hdr, Reduce red, cudaStream_t st)
{
    if (P.K == 4)
        return solve_mg_k<4>(P, o, h, w, g, y, delta, y_update, resid, report_rel, report_it,
                             solve_ws, hdr, red, st);
    return solve_mg_k<3>(P, o, h, w, g, y, delta, y_update, resid, report_rel, report_it, solve_ws,
                         hdr, red, st);
}

}  // namespace mpm
