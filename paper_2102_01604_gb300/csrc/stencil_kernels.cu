// stencil_kernels.cu -- the prior and the Newton-system solve (sm_103a):
//   k_jtv          JTV weights w_n = (u_n + eps^2)^-1/2 and JTV_eps (Eqs. 38-40)
//   k_pcg_init     r_0 = g + L y, preconditioner factor, p_0 = z_0 = M^-1 r_0 (Eq. 42)
//   k_pcg_direction p_k = z_k + beta p_{k-1}; every other k also
//                  x += alpha_{k-2} p_{k-2} + alpha_{k-1} p_{k-1}
//   k_pcg_matvec   q = (H + L) p_k; p.q
//   k_pcg_update   r -= alpha q; z = M^-1 r; r.z, r.r
//   k_pcg_final    delta = x + alpha p (or y <- y - delta)
//
// L = G'WG (x) diag(lambda) is applied as the 7-point weighted stencil
//   (L v)_k[n] = lambda_k sum_{m in N(n)} (w_n + w_m)(v_k[n] - v_k[m]) / h^2,
// neighbours outside the volume dropped (Neumann).  Blocks cover a 32 x 8
// (x, y) tile and march along z.  All CG scalars (alpha, beta, |r|) live in
// device memory and are produced by the last block of each reducing launch,
// so the whole PCG runs without a host round trip.
#include <type_traits>

#include "mpm_internal.cuh"

namespace mpm {

// Edge coefficients c_j = (w_n + w_m) / h_j^2 of the six neighbours (0 when
// the neighbour is outside the volume) and their offsets.
struct Edges {
    float c[6];
    long long off[6];
    bool ok[6];
};

__device__ __forceinline__ void make_edges(const DevProblem& P, int x, int y, int z,
                                           long long n, const float* __restrict__ w,
                                           float wn, Edges& e)
{
    const long long sxy = (long long)P.nx * P.ny;
    e.off[0] = -1;        e.ok[0] = x > 0;
    e.off[1] = 1;         e.ok[1] = x < P.nx - 1;
    e.off[2] = -P.nx;     e.ok[2] = y > 0;
    e.off[3] = P.nx;      e.ok[3] = y < P.ny - 1;
    e.off[4] = -sxy;      e.ok[4] = z > 0;
    e.off[5] = sxy;       e.ok[5] = z < P.nz - 1;
    const float ih[6] = {P.ihx2, P.ihx2, P.ihy2, P.ihy2, P.ihz2, P.ihz2};
#pragma unroll
    for (int j = 0; j < 6; ++j)
        e.c[j] = e.ok[j] ? (wn + __ldg(w + n + e.off[j])) * ih[j] : 0.0f;
}

// ------------------------------------------------------------- JTV weights

// Each thread marches up its z range with the centre values of planes z - 1,
// z and z + 1 in registers; the centre of plane z + 2 is loaded one plane
// ahead, so the only far (next-plane) load is in flight while plane z is
// computed.  The x / y neighbours come from the current plane (L1).  The six
// terms are summed in the order x-, x+, y-, y+, z-, z+.
template <int K>
__global__ void __launch_bounds__(kBlock) k_jtv(DevProblem P, int zc, const float* __restrict__ y,
                                                float* __restrict__ w, double* jtv, Reduce red)
{
    const long long N = P.N;
    const long long sxy = (long long)P.nx * P.ny;
    const int x = blockIdx.x * kTileX + threadIdx.x;
    const int yy = blockIdx.y * kTileY + threadIdx.y;
    const int z0 = blockIdx.z * zc;
    const int z1 = min(P.nz, z0 + zc);
    Acc acc;
    if (x < P.nx && yy < P.ny && z0 < z1) {
        const long long base = x + (long long)P.nx * yy;
        const bool okx0 = x > 0, okx1 = x < P.nx - 1, oky0 = yy > 0, oky1 = yy < P.ny - 1;
        float dn[K], cu[K], up[K], nx2[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float* yk = y + k * N + base;
            cu[k] = __ldg(yk + sxy * z0);
            dn[k] = z0 > 0 ? __ldg(yk + sxy * (z0 - 1)) : 0.0f;
            up[k] = z0 + 1 < P.nz ? __ldg(yk + sxy * (z0 + 1)) : 0.0f;
        }
        for (int z = z0; z < z1; ++z) {
            const long long n = base + sxy * z;
            const bool okz0 = z > 0, okz1 = z < P.nz - 1;
            // the centre two planes up, for the next step
#pragma unroll
            for (int k = 0; k < K; ++k)
                nx2[k] = (z + 2 < P.nz && z + 1 < z1) ? __ldg(y + k * N + n + 2 * sxy) : 0.0f;
            float u = 0.0f;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const float* yk = y + k * N + n;
                const float v = cu[k];
                float s = 0.0f;
                float d;
                if (okx0) { d = __ldg(yk - 1) - v; s += d * d * P.ihx2; }
                if (okx1) { d = __ldg(yk + 1) - v; s += d * d * P.ihx2; }
                if (oky0) { d = __ldg(yk - P.nx) - v; s += d * d * P.ihy2; }
                if (oky1) { d = __ldg(yk + P.nx) - v; s += d * d * P.ihy2; }
                if (okz0) { d = dn[k] - v; s += d * d * P.ihz2; }
                if (okz1) { d = up[k] - v; s += d * d * P.ihz2; }
                u += P.lambda[k] * s;
            }
            const float val = u + P.eps2;
            const float sq = sqrtf(val);
            if (w) w[n] = 1.0f / sq;
            acc.add(sq);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                dn[k] = cu[k];
                cu[k] = up[k];
                up[k] = nx2[k];
            }
        }
    }
    Acc v[1] = {acc};
    double out[1];
    if (grid_reduce<1>(v, red, out) && threadIdx.x == 0 && threadIdx.y == 0) *jtv = out[0];
}

// ------------------------------------------------ preconditioner helpers

// Lower Cholesky factor of the K x K block, packed row by row
// (00, 10, 11, 20, 21, 22, 30, 31, 32, 33) with reciprocal diagonal.
__host__ __device__ constexpr int lo(int i, int j) { return i * (i + 1) / 2 + j; }

template <int K>
__device__ __forceinline__ bool cholesky_f32(const float (&M)[K][K], float (&L)[K * (K + 1) / 2])
{
    bool ok = true;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        float s = M[j][j];
#pragma unroll
        for (int k = 0; k < j; ++k) s -= L[lo(j, k)] * L[lo(j, k)];
        if (!(s > 0.0f)) {
            ok = false;
            s = fmaxf(fabsf(M[j][j]), 1e-30f);
        }
        const float dj = sqrtf(s);
        L[lo(j, j)] = 1.0f / dj;
#pragma unroll
        for (int i = j + 1; i < K; ++i) {
            float v = M[i][j];
#pragma unroll
            for (int k = 0; k < j; ++k) v -= L[lo(i, k)] * L[lo(j, k)];
            L[lo(i, j)] = v / dj;
        }
    }
    return ok;
}

// z = (L L')^-1 r with the packed factor.
template <int K>
__device__ __forceinline__ void chol_apply(const float (&L)[K * (K + 1) / 2], const float (&r)[K],
                                           float (&z)[K])
{
    float t[K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        float v = r[i];
#pragma unroll
        for (int k = 0; k < i; ++k) v -= L[lo(i, k)] * t[k];
        t[i] = v * L[lo(i, i)];
    }
#pragma unroll
    for (int i = K - 1; i >= 0; --i) {
        float v = t[i];
#pragma unroll
        for (int k = i + 1; k < K; ++k) v -= L[lo(k, i)] * z[k];
        z[i] = v * L[lo(i, i)];
    }
}

// Per-solve workspace layout (all [.][N] float, 256-byte aligned).
struct SolveBufs {
    float* R;       // [T][N] preconditioner factor
    float* r;       // [K][N]
    float* z;       // [K][N]
    float* p[2];    // [K][N] directions, p_k in p[k & 1]
    float* q;       // [K][N]
};

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t solve_ws_bytes(const DevProblem& P)
{
    const size_t vec = align256(sizeof(float) * (size_t)P.K * P.N);
    return align256(sizeof(float) * (size_t)P.T * P.N) + 5 * vec;
}

static SolveBufs carve(const DevProblem& P, void* ws)
{
    SolveBufs b;
    char* c = static_cast<char*>(ws);
    const size_t vec = align256(sizeof(float) * (size_t)P.K * P.N);
    b.R = reinterpret_cast<float*>(c);
    c += align256(sizeof(float) * (size_t)P.T * P.N);
    b.r = reinterpret_cast<float*>(c); c += vec;
    b.z = reinterpret_cast<float*>(c); c += vec;
    b.p[0] = reinterpret_cast<float*>(c); c += vec;
    b.p[1] = reinterpret_cast<float*>(c); c += vec;
    b.q = reinterpret_cast<float*>(c);
    return b;
}

// --------------------------------------------------------------- PCG init

template <int K>
__global__ void __launch_bounds__(kBlock) k_pcg_init(DevProblem P, int zc, const float* __restrict__ h,
                                                     const float* __restrict__ w,
                                                     const float* __restrict__ g,
                                                     const float* __restrict__ y, SolveBufs B,
                                                     double tol2, WsHeader* hdr, double* resid,
                                                     Reduce red)
{
    constexpr int T = K * (K + 1) / 2;
    const long long N = P.N;
    const long long sxy = (long long)P.nx * P.ny;
    const int x = blockIdx.x * kTileX + threadIdx.x;
    const int yy = blockIdx.y * kTileY + threadIdx.y;
    const int z0 = blockIdx.z * zc;
    const int z1 = min(P.nz, z0 + zc);
    Acc rz, rr;
    bool pd = true;
    if (x < P.nx && yy < P.ny) {
        for (int z = z0; z < z1; ++z) {
            const long long n = x + (long long)P.nx * yy + sxy * z;
            const float wn = __ldg(w + n);
            Edges e;
            make_edges(P, x, yy, z, n, w, wn, e);
            float d = 0.0f;
#pragma unroll
            for (int j = 0; j < 6; ++j) d += e.c[j];
            float r[K], M[K][K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const float* yk = y + k * N;
                const float v = __ldg(yk + n);
                float s = 0.0f;
#pragma unroll
                for (int j = 0; j < 6; ++j)
                    if (e.ok[j]) s += e.c[j] * (v - __ldg(yk + n + e.off[j]));
                r[k] = __ldg(g + k * N + n) + P.lambda[k] * s;
            }
#pragma unroll
            for (int a = 0; a < K; ++a)
#pragma unroll
                for (int b = a; b < K; ++b) M[a][b] = M[b][a] = __ldg(h + tri(K, a, b) * N + n);
#pragma unroll
            for (int a = 0; a < K; ++a) M[a][a] += P.lambda[a] * d;
            float L[T], zz[K];
            pd &= cholesky_f32<K>(M, L);
            chol_apply<K>(L, r, zz);
#pragma unroll
            for (int k = 0; k < T; ++k) B.R[k * N + n] = L[k];
            float vrz = 0.0f, vrr = 0.0f;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                B.r[k * N + n] = r[k];
                B.p[0][k * N + n] = zz[k];                // p_0 = z_0 (z_0 itself is never read again)
                vrz += r[k] * zz[k];
                vrr += r[k] * r[k];
            }
            rz.add(vrz);
            rr.add(vrr);
        }
    }
    if (!pd) atomicOr(&hdr->status, kStatusNotPD);
    Acc v[2] = {rz, rr};
    double out[2];
    if (grid_reduce<2>(v, red, out) && threadIdx.x == 0 && threadIdx.y == 0) {
        SolveScalars& sc = hdr->sc;
        sc.rz = out[0];
        sc.rr0 = out[1];
        sc.rr = out[1];
        sc.alpha = 0.0;
        sc.alpha_prev = 0.0;
        sc.beta = 0.0;
        sc.it = 0;
        sc.xcount = 0;
        sc.tol2 = tol2;
        const bool bad = !(out[0] == out[0]) || !(out[1] == out[1]);
        if (bad) atomicOr(&hdr->status, kStatusNaN);
        sc.done = (bad || !(out[0] > 0.0) || (tol2 > 0.0 && out[1] <= tol2 * out[1])) ? 1 : 0;
        if (resid) resid[0] = sqrt(out[1]);
    }
}

// ---------------------------------------------------------- PCG direction

// p_k = z_k + beta_{k-1} p_{k-1} (k >= 1), a streaming pass over the K*N
// entries (float4 when VPT = 4).  x is brought up to date only at even k:
// x += alpha_{k-2} p_{k-2} + alpha_{k-1} p_{k-1}, with p_{k-2} read from the
// buffer that p_k is about to replace.  The two additions happen in the order
// of two single updates (bit for bit the same x); the odd passes skip x, which
// saves reading and writing it every other iteration.
template <int VPT>
__global__ void __launch_bounds__(kBlock) k_pcg_direction(long long total, int k_it,
                                                          const float* __restrict__ zv,
                                                          const float* __restrict__ pold,
                                                          float* __restrict__ pnew,
                                                          float* __restrict__ xacc,
                                                          WsHeader* hdr)
{
    using V = typename std::conditional<VPT == 4, float4, float>::type;
    __shared__ float s_beta, s_alpha, s_alpha_prev;
    __shared__ int s_done;
    if (threadIdx.x == 0) {
        s_done = hdr->sc.done;
        s_beta = (float)hdr->sc.beta;
        s_alpha = (float)hdr->sc.alpha;
        s_alpha_prev = (float)hdr->sc.alpha_prev;
    }
    __syncthreads();
    if (s_done) return;
    const bool fold = (k_it & 1) == 0;                  // x update at even k (k >= 2)
    if (fold && blockIdx.x == 0 && threadIdx.x == 0) hdr->sc.xcount = k_it;
    const float beta = s_beta, alpha = s_alpha, alpha_prev = s_alpha_prev;
    const long long nv = total / VPT;
    const V* __restrict__ z4 = reinterpret_cast<const V*>(zv);
    const V* __restrict__ o4 = reinterpret_cast<const V*>(pold);
    V* __restrict__ p4 = reinterpret_cast<V*>(pnew);
    V* __restrict__ x4 = reinterpret_cast<V*>(xacc);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nv;
         i += (long long)gridDim.x * blockDim.x) {
        const V zz = __ldg(z4 + i);
        const V o = __ldg(o4 + i);
        V pv;
        if (fold) {
            const V o2 = p4[i];                             // p_{k-2}, before it is replaced
            V xo;
            if (k_it > 2) xo = x4[i];
            V xv;
#pragma unroll
            for (int j = 0; j < VPT; ++j) {
                const float oj = reinterpret_cast<const float*>(&o)[j];
                const float xj = k_it > 2 ? reinterpret_cast<const float*>(&xo)[j] : 0.0f;
                const float t = fmaf(alpha_prev, reinterpret_cast<const float*>(&o2)[j], xj);
                reinterpret_cast<float*>(&xv)[j] = fmaf(alpha, oj, t);
                reinterpret_cast<float*>(&pv)[j] = fmaf(beta, oj, reinterpret_cast<const float*>(&zz)[j]);
            }
            x4[i] = xv;
        } else {
#pragma unroll
            for (int j = 0; j < VPT; ++j)
                reinterpret_cast<float*>(&pv)[j] =
                    fmaf(beta, reinterpret_cast<const float*>(&o)[j], reinterpret_cast<const float*>(&zz)[j]);
        }
        p4[i] = pv;
    }
}

// ------------------------------------------------------------- PCG matvec

// q = (H + L) p with p already formed.  Tiled 2.5-D stencil: a block owns a
// kMvX x kMvY (x, y) tile and marches up a run of z planes; the current plane
// of p (with a one-voxel x / y halo) and of the JTV weights is staged in
// shared memory, the planes below and above live in registers, so each
// operand is read from memory about once per voxel.
constexpr int kMvX = 16, kMvY = 16;

template <int K>
__global__ void __launch_bounds__(kMvX * kMvY, 3) k_pcg_matvec(DevProblem P, int zc, int k_it,
                                                              const float* __restrict__ h,
                                                              const float* __restrict__ w,
                                                              const float* __restrict__ pin,
                                                              float* __restrict__ qout,
                                                              WsHeader* hdr, Reduce red)
{
    constexpr int T = K * (K + 1) / 2;
    __shared__ float sp[K][kMvY + 2][kMvX + 2];
    __shared__ float sw[kMvY + 2][kMvX + 2];
    __shared__ int s_done;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = tx + ty * kMvX;
    if (tid == 0) s_done = hdr->sc.done;
    __syncthreads();
    if (s_done) return;
    const long long N = P.N;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const long long sxy = (long long)nx * ny;
    const int x = blockIdx.x * kMvX + tx;
    const int y = blockIdx.y * kMvY + ty;
    const int z0 = blockIdx.z * zc;
    const int z1 = min(nz, z0 + zc);
    const bool inside = x < nx && y < ny;
    // Halo roles: border threads of the tile also load the neighbour just
    // outside it (one plane ahead, so the loads overlap the compute).
    const bool hx = inside && ((tx == 0 && x > 0) || (tx == kMvX - 1 && x + 1 < nx));
    const bool hy = inside && ((ty == 0 && y > 0) || (ty == kMvY - 1 && y + 1 < ny));
    const long long ox = tx == 0 ? -1 : 1;
    const long long oy = ty == 0 ? -(long long)nx : (long long)nx;
    const int sx = tx == 0 ? 0 : kMvX + 1;
    const int sy = ty == 0 ? 0 : kMvY + 1;

    const long long col = (long long)x + (long long)nx * y;   // (x, y) column offset
    float pc[K], pp[K], pn[K], hxv[K + 1], hyv[K + 1];
    float wc = 0.f, wp = 0.f, wn = 0.f;
    auto load_halo = [&](long long n) {
        if (hx) {
#pragma unroll
            for (int k = 0; k < K; ++k) hxv[k] = __ldg(pin + k * N + n + ox);
            hxv[K] = __ldg(w + n + ox);
        }
        if (hy) {
#pragma unroll
            for (int k = 0; k < K; ++k) hyv[k] = __ldg(pin + k * N + n + oy);
            hyv[K] = __ldg(w + n + oy);
        }
    };
    if (inside) {
        const long long n0 = col + sxy * z0;
#pragma unroll
        for (int k = 0; k < K; ++k) pc[k] = __ldg(pin + k * N + n0);
        wc = __ldg(w + n0);
        load_halo(n0);
        if (z0 > 0) {
#pragma unroll
            for (int k = 0; k < K; ++k) pp[k] = __ldg(pin + k * N + n0 - sxy);
            wp = __ldg(w + n0 - sxy);
        }
        if (z0 + 1 < nz) {
#pragma unroll
            for (int k = 0; k < K; ++k) pn[k] = __ldg(pin + k * N + n0 + sxy);
            wn = __ldg(w + n0 + sxy);
        }
    }
    float Hnext[T];
    if (inside) {
        const long long n0 = col + sxy * z0;
#pragma unroll
        for (int t = 0; t < T; ++t) Hnext[t] = __ldg(h + t * N + n0);
    }
    Acc pq;
    for (int z = z0; z < z1; ++z) {
        const long long n = col + sxy * z;
        float Hn[T];
#pragma unroll
        for (int t = 0; t < T; ++t) Hn[t] = Hnext[t];
        // stage the current plane (own value and x / y halo) in shared memory
        __syncthreads();
        if (inside) {
#pragma unroll
            for (int k = 0; k < K; ++k) sp[k][ty + 1][tx + 1] = pc[k];
            sw[ty + 1][tx + 1] = wc;
            if (hx) {
#pragma unroll
                for (int k = 0; k < K; ++k) sp[k][ty + 1][sx] = hxv[k];
                sw[ty + 1][sx] = hxv[K];
            }
            if (hy) {
#pragma unroll
                for (int k = 0; k < K; ++k) sp[k][sy][tx + 1] = hyv[k];
                sw[sy][tx + 1] = hyv[K];
            }
        }
        __syncthreads();
        if (inside) {
            // prefetch the next plane's halo and the plane after it
            const bool more = z + 1 < z1;
            if (more) load_halo(n + sxy);
            float pn_keep[K];
#pragma unroll
            for (int k = 0; k < K; ++k) pn_keep[k] = pn[k];
            const float wn_keep = wn;
            if (more) {
#pragma unroll
                for (int t = 0; t < T; ++t) Hnext[t] = __ldg(h + t * N + n + sxy);
            }
            if (more && z + 2 < nz) {
                const long long n2 = n + 2 * sxy;
#pragma unroll
                for (int k = 0; k < K; ++k) pn[k] = __ldg(pin + k * N + n2);
                wn = __ldg(w + n2);
            }
            // edge coefficients (w_n + w_m) / h^2 of the six neighbours
            const bool okxm = x > 0, okxp = x + 1 < nx, okym = y > 0, okyp = y + 1 < ny;
            const bool okzm = z > 0, okzp = z + 1 < nz;
            const float cxm = okxm ? (wc + sw[ty + 1][tx]) * P.ihx2 : 0.f;
            const float cxp = okxp ? (wc + sw[ty + 1][tx + 2]) * P.ihx2 : 0.f;
            const float cym = okym ? (wc + sw[ty][tx + 1]) * P.ihy2 : 0.f;
            const float cyp = okyp ? (wc + sw[ty + 2][tx + 1]) * P.ihy2 : 0.f;
            const float czm = okzm ? (wc + wp) * P.ihz2 : 0.f;
            const float czp = okzp ? (wc + wn_keep) * P.ihz2 : 0.f;
            float vpq = 0.0f;
#pragma unroll
            for (int a = 0; a < K; ++a) {
                const float v = pc[a];
                float s = 0.f;
                if (okxm) s += cxm * (v - sp[a][ty + 1][tx]);
                if (okxp) s += cxp * (v - sp[a][ty + 1][tx + 2]);
                if (okym) s += cym * (v - sp[a][ty][tx + 1]);
                if (okyp) s += cyp * (v - sp[a][ty + 2][tx + 1]);
                if (okzm) s += czm * (v - pp[a]);
                if (okzp) s += czp * (v - pn_keep[a]);
                float acc = P.lambda[a] * s;
#pragma unroll
                for (int b = 0; b < K; ++b) acc += Hn[a < b ? tri(K, a, b) : tri(K, b, a)] * pc[b];
                qout[a * N + n] = acc;
                vpq += v * acc;
            }
            pq.add(vpq);
            // march: the plane above becomes current
#pragma unroll
            for (int k = 0; k < K; ++k) {
                pp[k] = pc[k];
                pc[k] = pn_keep[k];
            }
            wp = wc;
            wc = wn_keep;
        }
    }
    Acc v[1] = {pq};
    double out[1];
    if (grid_reduce<1>(v, red, out) && tid == 0) {
        SolveScalars& sc = hdr->sc;
        if (!(out[0] == out[0])) atomicOr(&hdr->status, kStatusNaN);
        if (!(out[0] > 0.0)) {
            sc.done = 1;                 // no further step; the alphas keep their values
        } else {
            sc.alpha_prev = sc.alpha;
            sc.alpha = sc.rz / out[0];
        }
    }
}

// ------------------------------------------------------------- PCG update

// Streaming kernel: VPT consecutive voxels per thread (float4 loads when
// VPT = 4), grid-stride over the volume.
template <int K, int VPT>
__global__ void __launch_bounds__(kBlock) k_pcg_update(DevProblem P, int k_it, SolveBufs B,
                                                       WsHeader* hdr, double* resid, Reduce red)
{
    constexpr int T = K * (K + 1) / 2;
    using V = typename std::conditional<VPT == 4, float4, float>::type;
    __shared__ float s_alpha;
    __shared__ int s_done;
    if (threadIdx.x == 0) {
        s_done = hdr->sc.done;
        s_alpha = (float)hdr->sc.alpha;
    }
    __syncthreads();
    if (s_done) return;
    const float alpha = s_alpha;
    const long long N = P.N;
    const long long NV = N / VPT;           // vectors per map (N % VPT == 0)
    const V* __restrict__ r4 = reinterpret_cast<const V*>(B.r);
    const V* __restrict__ q4 = reinterpret_cast<const V*>(B.q);
    const V* __restrict__ R4 = reinterpret_cast<const V*>(B.R);
    V* __restrict__ rw = reinterpret_cast<V*>(B.r);
    V* __restrict__ zw = reinterpret_cast<V*>(B.z);
    Acc rz, rr;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < NV;
         i += (long long)gridDim.x * blockDim.x) {
        V rv[K], qv[K], Lv[T];
#pragma unroll
        for (int k = 0; k < K; ++k) rv[k] = r4[k * NV + i];
#pragma unroll
        for (int k = 0; k < K; ++k) qv[k] = __ldg(q4 + k * NV + i);
#pragma unroll
        for (int t = 0; t < T; ++t) Lv[t] = __ldg(R4 + t * NV + i);
        V zo[K];
#pragma unroll
        for (int j = 0; j < VPT; ++j) {
            float r[K], L[T], zz[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                r[k] = reinterpret_cast<const float*>(&rv[k])[j] -
                       alpha * reinterpret_cast<const float*>(&qv[k])[j];
                reinterpret_cast<float*>(&rv[k])[j] = r[k];
            }
#pragma unroll
            for (int t = 0; t < T; ++t) L[t] = reinterpret_cast<const float*>(&Lv[t])[j];
            chol_apply<K>(L, r, zz);
            float vrz = 0.0f, vrr = 0.0f;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                reinterpret_cast<float*>(&zo[k])[j] = zz[k];
                vrz += r[k] * zz[k];
                vrr += r[k] * r[k];
            }
            rz.add(vrz);
            rr.add(vrr);
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            rw[k * NV + i] = rv[k];
            zw[k * NV + i] = zo[k];
        }
    }
    Acc v[2] = {rz, rr};
    double out[2];
    if (grid_reduce<2>(v, red, out) && threadIdx.x == 0) {
        SolveScalars& sc = hdr->sc;
        const bool bad = !(out[0] == out[0]) || !(out[1] == out[1]);
        if (bad) atomicOr(&hdr->status, kStatusNaN);
        sc.beta = out[0] / sc.rz;
        sc.rz = out[0];
        sc.rr = out[1];
        sc.it = k_it + 1;
        if (resid) resid[k_it + 1] = sqrt(out[1]);
        if (bad || !(out[0] > 0.0) || (sc.tol2 > 0.0 && out[1] <= sc.tol2 * sc.rr0)) sc.done = 1;
    }
}

// -------------------------------------------------------------- PCG final

__global__ void __launch_bounds__(kBlock) k_pcg_final(long long total, SolveBufs B,
                                                      const float* __restrict__ xacc,
                                                      float* __restrict__ delta,
                                                      float* __restrict__ y_update,
                                                      const WsHeader* hdr, double* report_rel,
                                                      int* report_it)
{
    const SolveScalars sc = hdr->sc;
    const bool have_x = sc.xcount > 0;
    const int pend = sc.it - sc.xcount;        // directions not yet in x: 0, 1 or 2
    const float alpha = (float)sc.alpha, alpha_prev = (float)sc.alpha_prev;
    const float* __restrict__ pp = B.p[(sc.it - 1) & 1];
    const float* __restrict__ pp2 = B.p[sc.it & 1];   // p_{it-2} when pend == 2
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        float v = have_x ? xacc[i] : 0.0f;
        if (pend == 2) v = fmaf(alpha_prev, pp2[i], v);
        if (pend >= 1) v = fmaf(alpha, pp[i], v);
        if (y_update)
            y_update[i] -= v;
        else
            delta[i] = v;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (report_rel) *report_rel = sc.rr0 > 0.0 ? sqrt(sc.rr / sc.rr0) : 0.0;
        if (report_it) *report_it = sc.it;
    }
}

// ------------------------------------------------------------- launchers

// One wave of resident blocks for a grid-stride streaming kernel.
template <int K, int VPT>
static int update_grid(long long units)
{
    static int per_sm = 0;
    if (per_sm == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pcg_update<K, VPT>, kBlock, 0) !=
                cudaSuccess || b < 1)
            b = 1;
        per_sm = b;
    }
    long long g = (units + kBlock - 1) / kBlock;
    const long long cap = (long long)per_sm * kNumSm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

StencilGrid stencil_grid(const DevProblem& P, int tx, int ty)
{
    StencilGrid sg;
    sg.block = dim3(tx, ty, 1);
    const int gx = (P.nx + tx - 1) / tx;
    const int gy = (P.ny + ty - 1) / ty;
    const long long tiles = (long long)gx * gy;
    // about two waves of 8 resident blocks per SM, at most kMaxBlocks blocks
    const long long target = 2LL * 8 * kNumSm;
    long long gz = target / (tiles > 0 ? tiles : 1);
    if (gz < 1) gz = 1;
    if (gz > P.nz) gz = P.nz;
    while (tiles * gz > kMaxBlocks && gz > 1) --gz;
    sg.zc = (int)((P.nz + gz - 1) / gz);
    gz = (P.nz + sg.zc - 1) / sg.zc;
    sg.grid = dim3(gx, gy, (unsigned)gz);
    return sg;
}

cudaError_t launch_jtv(const DevProblem& P, const float* y, float* w, double* jtv, Reduce red,
                       cudaStream_t st)
{
    const StencilGrid sg = stencil_grid(P, kTileX, kTileY);
    LaunchScope ls(MPM_KERNEL_JTV, st);
    if (P.K == 4)
        k_jtv<4><<<sg.grid, sg.block, 0, st>>>(P, sg.zc, y, w, jtv, red);
    else
        k_jtv<3><<<sg.grid, sg.block, 0, st>>>(P, sg.zc, y, w, jtv, red);
    return cudaGetLastError();
}

template <int K>
static cudaError_t solve_k(const DevProblem& P, int cg_iters, double tol_cg, const float* h,
                           const float* w, const float* g, const float* y, float* delta,
                           float* y_update, double* resid, double* report_rel, int* report_it,
                           void* solve_ws, WsHeader* hdr, Reduce red, cudaStream_t st)
{
    const StencilGrid sg = stencil_grid(P, kTileX, kTileY);
    SolveBufs B = carve(P, solve_ws);
    // x accumulates in `delta` (the caller's output when solving alone, a
    // workspace buffer inside the fit, which then passes y_update).
    float* xacc = delta;
    const double tol2 = tol_cg > 0.0 ? tol_cg * tol_cg : 0.0;
    {
        LaunchScope ls(MPM_KERNEL_PCG_INIT, st);
        k_pcg_init<K><<<sg.grid, sg.block, 0, st>>>(P, sg.zc, h, w, g, y, B, tol2, hdr, resid, red);
    }
    const StencilGrid mg = stencil_grid(P, kMvX, kMvY);
    TmaMaps maps;
    const int tile = tma_tile_choice(P);
    const bool tma = tile >= 0 && make_tma_maps(P, h, w, B.p[0], B.p[1], tile, &maps);
    const StencilGrid tg = tma ? tma_grid(P, tile) : mg;
    // float4 streaming needs whole vectors per map and 16-byte aligned rows
    const bool vec4 = (P.N % 4 == 0) &&
                      ((reinterpret_cast<uintptr_t>(B.r) | reinterpret_cast<uintptr_t>(B.q) |
                        reinterpret_cast<uintptr_t>(B.z) | reinterpret_cast<uintptr_t>(B.R) |
                        reinterpret_cast<uintptr_t>(B.p[0]) | reinterpret_cast<uintptr_t>(B.p[1]) |
                        reinterpret_cast<uintptr_t>(xacc)) % 16 == 0);
    const int ugrid = vec4 ? update_grid<K, 4>(P.N / 4) : update_grid<K, 1>(P.N);
    const long long KN = (long long)K * P.N;
    const int dgrid = voxel_grid(vec4 ? KN / 4 : KN);
    for (int k = 0; k < cg_iters; ++k) {
        float* pk = B.p[k & 1];
        if (k > 0) {
            LaunchScope ls(MPM_KERNEL_PCG_DIRECTION, st);
            if (vec4)
                k_pcg_direction<4><<<dgrid, kBlock, 0, st>>>(KN, k, B.z, B.p[(k + 1) & 1], pk, xacc, hdr);
            else
                k_pcg_direction<1><<<dgrid, kBlock, 0, st>>>(KN, k, B.z, B.p[(k + 1) & 1], pk, xacc, hdr);
        }
        {
            LaunchScope ls(MPM_KERNEL_PCG_MATVEC, st);
            if (tma) {
                cudaError_t e = launch_matvec_tma(P, tg, maps, k, B.q, hdr, red, st);
                if (e != cudaSuccess) return e;
            } else {
                k_pcg_matvec<K><<<mg.grid, mg.block, 0, st>>>(P, mg.zc, k, h, w, pk, B.q, hdr, red);
            }
        }
        LaunchScope ls(MPM_KERNEL_PCG_UPDATE, st);
        if (vec4)
            k_pcg_update<K, 4><<<ugrid, kBlock, 0, st>>>(P, k, B, hdr, resid, red);
        else
            k_pcg_update<K, 1><<<ugrid, kBlock, 0, st>>>(P, k, B, hdr, resid, red);
    }
    LaunchScope ls(MPM_KERNEL_PCG_FINAL, st);
    k_pcg_final<<<voxel_grid(P.N * K), kBlock, 0, st>>>(P.N * K, B, xacc, delta, y_update, hdr,
                                                        report_rel, report_it);
    return cudaGetLastError();
}

cudaError_t tma_autotune(const DevProblem& P, void* solve_ws, WsHeader* hdr, Reduce red,
                         cudaStream_t st, int* best, float* ms)
{
    SolveBufs B = carve(P, solve_ws);
    *best = -1;
    // operands: R stands in for H (same size), r for w; all zero
    const size_t vec = sizeof(float) * (size_t)P.K * P.N;
    cudaError_t e;
    if ((e = cudaMemsetAsync(B.R, 0, sizeof(float) * (size_t)P.T * P.N, st)) != cudaSuccess) return e;
    for (float* v : {B.r, B.p[0], B.p[1]})
        if ((e = cudaMemsetAsync(v, 0, vec, st)) != cudaSuccess) return e;
    cudaEvent_t a, b;
    if ((e = cudaEventCreate(&a)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&b)) != cudaSuccess) {
        cudaEventDestroy(a);
        return e;
    }
    float best_ms = 0.0f;
    for (int t = 0; t < tma_tile_count(); ++t) {
        ms[t] = -1.0f;
        TmaMaps m;
        if (!make_tma_maps(P, B.R, B.r, B.p[0], B.p[1], t, &m)) continue;
        const StencilGrid g = tma_grid(P, t);
        constexpr int reps = 5;
        for (int i = 0; i <= reps && e == cudaSuccess; ++i) {
            if (i == 1) e = cudaEventRecord(a, st);
            if (e == cudaSuccess) e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st);
            if (e == cudaSuccess) e = launch_matvec_tma(P, g, m, 2, B.q, hdr, red, st);
        }
        if (e == cudaSuccess) e = cudaEventRecord(b, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float t_ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t_ms, a, b);
        if (e != cudaSuccess) break;
        ms[t] = t_ms / reps;
        if (*best < 0 || ms[t] < best_ms) {
            best_ms = ms[t];
            *best = t;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e == cudaSuccess && *best >= 0) tma_tile_set(P, *best);
    return e;
}

cudaError_t launch_solve(const DevProblem& P, int cg_iters, double tol_cg, const float* h,
                         const float* w, const float* g, const float* y, float* delta,
                         float* y_update, double* resid, double* report_rel, int* report_it,
                         void* solve_ws, WsHeader* hdr, Reduce red, cudaStream_t st)
{
    if (P.K == 4)
        return solve_k<4>(P, cg_iters, tol_cg, h, w, g, y, delta, y_update, resid, report_rel,
                          report_it, solve_ws, hdr, red, st);
    return solve_k<3>(P, cg_iters, tol_cg, h, w, g, y, delta, y_update, resid, report_rel,
                      report_it, solve_ws, hdr, red, st);
}

}  // namespace mpm
