// stencil_kernels.cu -- the prior and the Newton-system solve (sm_103a):
//   k_jtv          JTV weights w_n = (u_n + eps^2)^-1/2 and JTV_eps (Eqs. 38-40)
//   k_pcg_init     r_0 = g + L y, z_0 = M^-1 r_0 (Eq. 42)
//   k_pcg_step     one PCG iteration (pcg_step.cuh): z_j, p_j from the previous
//                  iteration, q = (H + L) p_j, v = M^-1 q, the x fold and the
//                  sums for alpha_j and beta_j -- the plain kernel used when the
//                  TMA-staged one (stencil_tma.cu) does not apply
//   k_pcg_final    delta = x + pending directions (or y <- y - delta)
//
// L = G'WG (x) diag(lambda) is applied as the 7-point weighted stencil
//   (L v)_k[n] = lambda_k sum_{m in N(n)} (w_n + w_m)(v_k[n] - v_k[m]) / h^2,
// neighbours outside the volume dropped (Neumann).  Blocks cover a 32 x 8
// (x, y) tile and march along z.  All CG scalars (alpha, beta, |r|) live in
// device memory and are produced by the last block of each reducing launch,
// so the whole PCG runs without a host round trip.
#include <algorithm>

#include "mpm_internal.cuh"
#include "pcg_step.cuh"

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

// Whether every index the JTV kernel forms for this volume (K arrays of N
// values, with room to spare) fits in a signed 32-bit int: its address
// arithmetic is then 32-bit (114 -> 111 us at 176x240x256).
static bool index32(const DevProblem& P)
{
    return P.N * (long long)(P.K * (P.K + 1) / 2 + 1) < 0x7fffffffLL;
}

constexpr int kInitAhead = 2;     // planes between the PCG start's L2 hint and the use

// Each thread marches up its z range with the centre values of planes z - 1,
// z and z + 1 in registers; the centre of plane z + 2 is loaded one plane
// ahead.  The x / y neighbours come from the plane's tile in shared memory
// (double-buffered, one barrier per plane): every thread writes its centre,
// and 80 threads the tile's halo (rows y0 - 1 and y0 + 8, columns x0 - 1 and
// x0 + 32), which they too load two planes ahead.  The six terms are summed in
// the order x-, x+, y-, y+, z-, z+.
template <int K, typename IT>
__device__ __forceinline__ void jtv_body(const DevProblem& P, int zc, const float* __restrict__ y,
                                         float* __restrict__ w, double* jtv, Reduce red, const VGrid& vg)
{
    constexpr int TW = kTileX + 2, TH = kTileY + 2;
    __shared__ float tile[2][K][TH][TW];
    const IT N = (IT)P.N;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const IT sxy = (IT)nx * ny;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x = vg.bx * kTileX + tx;
    const int yy = vg.by * kTileY + ty;
    const int z0 = vg.bz * zc;
    const int z1 = min(nz, z0 + zc);
    // this thread's halo point, if any: its place in the tile and the volume
    const int t = ty * kTileX + tx;
    int hx = -1, hy = -1, hr = 0, hc = 0;
    if (t < 2 * kTileX) {                       // rows above and below the tile
        hr = t < kTileX ? 0 : TH - 1;
        hc = 1 + t % kTileX;
    } else if (t < 2 * kTileX + 2 * kTileY) {   // columns left and right
        const int u = t - 2 * kTileX;
        hr = 1 + u % kTileY;
        hc = u < kTileY ? 0 : TW - 1;
    }
    if (t < 2 * kTileX + 2 * kTileY) {
        hx = vg.bx * kTileX + hc - 1;
        hy = vg.by * kTileY + hr - 1;
    }
    const bool halo = hx >= 0 && hx < nx && hy >= 0 && hy < ny;
    const bool inside = x < nx && yy < ny;
    Acc acc;
    if (z0 < z1) {
        const IT base = inside ? x + (IT)nx * yy : 0;
        const IT hbase = halo ? hx + (IT)nx * hy : 0;
        const bool okx0 = x > 0, okx1 = x < nx - 1, oky0 = yy > 0, oky1 = yy < ny - 1;
        float dn[K], cu[K], up[K], nx2[K], h0[K], h1[K], h2[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float* yk = y + k * N + base;
            const float* hk = y + k * N + hbase;
            cu[k] = inside ? __ldg(yk + sxy * z0) : 0.0f;
            dn[k] = inside && z0 > 0 ? __ldg(yk + sxy * (z0 - 1)) : 0.0f;
            up[k] = inside && z0 + 1 < nz ? __ldg(yk + sxy * (z0 + 1)) : 0.0f;
            h0[k] = halo ? __ldg(hk + sxy * z0) : 0.0f;
            h1[k] = halo && z0 + 1 < z1 ? __ldg(hk + sxy * (z0 + 1)) : 0.0f;
        }
        for (int z = z0; z < z1; ++z) {
            const int b = z & 1;
            const IT n = base + sxy * z;
            const bool okz0 = z > 0, okz1 = z < nz - 1;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                tile[b][k][ty + 1][tx + 1] = cu[k];
                if (t < 2 * kTileX + 2 * kTileY) tile[b][k][hr][hc] = h0[k];
            }
            // the centre two planes up, and the halo two planes up, for later steps
#pragma unroll
            for (int k = 0; k < K; ++k) {
                nx2[k] = inside && z + 2 < nz && z + 1 < z1 ? __ldg(y + k * N + n + 2 * sxy) : 0.0f;
                h2[k] = halo && z + 2 < z1 ? __ldg(y + k * N + hbase + sxy * (z + 2)) : 0.0f;
            }
            __syncthreads();
            if (inside) {
                float u = 0.0f;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const float v = cu[k];
                    float s = 0.0f;
                    float d;
                    if (okx0) { d = tile[b][k][ty + 1][tx] - v; s += d * d * P.ihx2; }
                    if (okx1) { d = tile[b][k][ty + 1][tx + 2] - v; s += d * d * P.ihx2; }
                    if (oky0) { d = tile[b][k][ty][tx + 1] - v; s += d * d * P.ihy2; }
                    if (oky1) { d = tile[b][k][ty + 2][tx + 1] - v; s += d * d * P.ihy2; }
                    if (okz0) { d = dn[k] - v; s += d * d * P.ihz2; }
                    if (okz1) { d = up[k] - v; s += d * d * P.ihz2; }
                    u += P.lambda[k] * s;
                }
                const float val = u + P.eps2;
                const float sq = sqrtf(val);
                if (w) w[n] = 1.0f / sq;
                acc.add(sq);
            }
#pragma unroll
            for (int k = 0; k < K; ++k) {
                dn[k] = cu[k];
                cu[k] = up[k];
                up[k] = nx2[k];
                h0[k] = h1[k];
                h1[k] = h2[k];
            }
        }
    }
    Acc v[1] = {acc};
    double out[1];
    if (grid_reduce<1>(v, red, out, vg) && threadIdx.x == 0 && threadIdx.y == 0) *jtv = out[0];
}

template <int K, typename IT>
__global__ void __launch_bounds__(kBlock) k_jtv(DevProblem P, int zc, const float* __restrict__ y,
                                                float* __restrict__ w, double* jtv, Reduce red)
{
    jtv_body<K, IT>(P, zc, y, w, jtv, red, hw_grid());
}

template <int K, typename IT>
__global__ void __launch_bounds__(kBlock) k_jtv_batch(const __grid_constant__ Batch<JtvArgs> b)
{
    const int s = batch_subject(b.start, b.n);
    const JtvArgs& a = b.a[s];
    jtv_body<K, IT>(a.P, a.zc, a.y, a.w, a.jtv, a.red, batch_grid(b.start[s], a.gx, a.gy, a.gz));
}

// ------------------------------------------------------ solve workspace

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// z[2], v[2], p[3] and x, each [N] float4; or the multigrid solver's
// buffers (multigrid.cu), whichever is larger.
size_t solve_ws_bytes(const DevProblem& P)
{
    const size_t pcg = 8 * align256(sizeof(float4) * (size_t)P.N);
    const size_t mg = mg_ws_bytes(P);
    return pcg > mg ? pcg : mg;
}

SolveOpts solve_opts(const mpm_opts& o)
{
    SolveOpts s;
    s.cg_iters = o.cg_iters;
    s.tol_cg = o.tol_cg;
    s.mg_levels = o.mg_levels;
    s.mg_nu = o.mg_nu > 0 ? o.mg_nu : 1;
    s.mg_omega = o.mg_omega > 0.0 ? (float)o.mg_omega : 0.7f;
    s.mg_coarse_sweeps = o.mg_coarse_sweeps > 0 ? o.mg_coarse_sweeps : 20;
    return s;
}

static SolveBufs carve(const DevProblem& P, void* ws)
{
    SolveBufs b;
    char* c = static_cast<char*>(ws);
    const size_t vec = align256(sizeof(float4) * (size_t)P.N);
    for (float4*& v : b.z) { v = reinterpret_cast<float4*>(c); c += vec; }
    for (float4*& v : b.v) { v = reinterpret_cast<float4*>(c); c += vec; }
    for (float4*& v : b.p) { v = reinterpret_cast<float4*>(c); c += vec; }
    b.x = reinterpret_cast<float4*>(c);
    return b;
}

// --------------------------------------------------------------- PCG init

template <int K>
__device__ __forceinline__ void pcg_init_body(const DevProblem& P, int zc, const float* __restrict__ h,
                                              const float* __restrict__ w, const float* __restrict__ g,
                                              const float* __restrict__ y, float4* __restrict__ z0,
                                              double tol2, WsHeader* hdr, double* resid, Reduce red,
                                              const VGrid& vg)
{
    constexpr int T = K * (K + 1) / 2;
    const long long N = P.N;
    const long long sxy = (long long)P.nx * P.ny;
    const int x = vg.bx * kTileX + threadIdx.x;
    const int yy = vg.by * kTileY + threadIdx.y;
    const int z0p = vg.bz * zc;
    const int z1p = min(P.nz, z0p + zc);
    Acc rz, rr;
    bool pd = true;
    if (x < P.nx && yy < P.ny) {
        for (int z = z0p; z < z1p; ++z) {
            const long long n = x + (long long)P.nx * yy + sxy * z;
            // the operands of plane z + kInitAhead into L2 while plane z is computed
            if (z + kInitAhead < z1p) {
                const long long na = n + kInitAhead * sxy;
                prefetch_l2(w + na);
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    prefetch_l2(y + k * N + na);
                    prefetch_l2(g + k * N + na);
                }
#pragma unroll
                for (int t = 0; t < T; ++t) prefetch_l2(h + t * N + na);
            }
            const float wn = __ldg(w + n);
            Edges e;
            make_edges(P, x, yy, z, n, w, wn, e);
            float r[K];
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
            float hv[T], M[K][K];
#pragma unroll
            for (int t = 0; t < T; ++t) hv[t] = __ldg(h + t * N + n);
            precond_block<K>(P, hv, edge_sum(e.c), M);
            float L[T], zz[K];
            pd &= cholesky_f32<K>(M, L);
            chol_apply<K>(L, r, zz);
            z0[n] = pack4<K>(zz);
            float vrz = 0.0f, vrr = 0.0f;
#pragma unroll
            for (int k = 0; k < K; ++k) {
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
    if (grid_reduce<2>(v, red, out, vg) && threadIdx.x == 0 && threadIdx.y == 0) {
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

template <int K>
__global__ void __launch_bounds__(kBlock) k_pcg_init(DevProblem P, int zc, const float* __restrict__ h,
                                                     const float* __restrict__ w,
                                                     const float* __restrict__ g,
                                                     const float* __restrict__ y, float4* __restrict__ z0,
                                                     double tol2, WsHeader* hdr, double* resid,
                                                     Reduce red)
{
    pcg_init_body<K>(P, zc, h, w, g, y, z0, tol2, hdr, resid, red, hw_grid());
}

template <int K>
__global__ void __launch_bounds__(kBlock) k_pcg_init_batch(const __grid_constant__ Batch<InitArgs> b)
{
    const int s = batch_subject(b.start, b.n);
    const InitArgs& a = b.a[s];
    pcg_init_body<K>(a.P, a.zc, a.h, a.w, a.g, a.y, a.z0, a.tol2, a.hdr, a.resid, a.red,
                     batch_grid(b.start[s], a.gx, a.gy, a.gz));
}

// -------------------------------------------------------- PCG iteration

// Plain form of one PCG iteration (pcg_step.cuh): a thread per (x, y) column
// marching a run of z planes; each neighbour's p_j is formed from its own
// (z, v, p) read from memory.  Used for volumes or pointers the TMA kernel
// cannot take (nx not a multiple of 4, a volume smaller than a tile).
template <int K, int MODE>
__global__ void __launch_bounds__(kBlock) k_pcg_step(DevProblem P, int zc, int j, int want_rr,
                                                     const float* __restrict__ h,
                                                     const float* __restrict__ w,
                                                     const float4* __restrict__ zin,
                                                     const float4* __restrict__ vin,
                                                     const float4* __restrict__ pin,
                                                     const float4* __restrict__ p2,
                                                     float4* __restrict__ zout, float4* __restrict__ vout,
                                                     float4* __restrict__ pout, float4* __restrict__ xacc,
                                                     WsHeader* hdr, double* resid, Reduce red)
{
    constexpr int T = K * (K + 1) / 2;
    constexpr bool first = MODE == kModeFirst;
    __shared__ float s_alpha, s_alpha_prev, s_beta;
    __shared__ int s_done;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    if (tid == 0) {
        s_done = hdr->sc.done;
        s_alpha = (float)hdr->sc.alpha;
        s_alpha_prev = (float)hdr->sc.alpha_prev;
        s_beta = (float)hdr->sc.beta;
    }
    __syncthreads();
    if (s_done) return;
    if (MODE >= kModeFold && tid == 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0)
        hdr->sc.xcount = j;
    const float alpha = s_alpha, alpha_prev = s_alpha_prev, beta = s_beta;
    const long long sxy = (long long)P.nx * P.ny;
    const int x = blockIdx.x * kTileX + threadIdx.x;
    const int yy = blockIdx.y * kTileY + threadIdx.y;
    const int z0p = blockIdx.z * zc;
    const int z1p = min(P.nz, z0p + zc);
    float part[kStepSums] = {};
    auto point = [&](long long m, float (&zj)[K], float (&pj)[K]) {
        const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
        step_point<K, first>(alpha, beta, zin[m], first ? zero : vin[m], first ? zero : pin[m], zj, pj);
    };
    if (x < P.nx && yy < P.ny) {
        for (int z = z0p; z < z1p; ++z) {
            const long long n = x + (long long)P.nx * yy + sxy * z;
            const float wn = __ldg(w + n);
            Edges e;
            make_edges(P, x, yy, z, n, w, wn, e);
            float zj[K], pj[K], nb[6][K];
            point(n, zj, pj);
#pragma unroll
            for (int m = 0; m < 6; ++m) {
                float zm[K];
                if (e.ok[m]) {
                    point(n + e.off[m], zm, nb[m]);
                } else {
#pragma unroll
                    for (int a = 0; a < K; ++a) nb[m][a] = pj[a];
                }
            }
            float hv[T];
#pragma unroll
            for (int t = 0; t < T; ++t) hv[t] = __ldg(h + t * P.N + n);
            float v[K], sums[kStepSums];
            step_voxel<K>(P, e.c, zj, pj, [&](int m, int a) { return nb[m][a]; }, hv, want_rr, v, sums);
            if (!first) zout[n] = pack4<K>(zj);
            pout[n] = pack4<K>(pj);
            vout[n] = pack4<K>(v);
            if (MODE >= kModeFold) {
                const float4 x0 = MODE == kModeFoldX ? xacc[n] : make_float4(0.f, 0.f, 0.f, 0.f);
                xacc[n] = fold_x(x0, alpha_prev, p2[n], alpha, pin[n]);
            }
#pragma unroll
            for (int i = 0; i < kStepSums; ++i) part[i] += sums[i];
        }
    }
    Acc acc[kStepSums];
#pragma unroll
    for (int i = 0; i < kStepSums; ++i) acc[i].add(part[i]);
    double out[kStepSums];
    if (grid_reduce<kStepSums>(acc, red, out) && tid == 0) step_scalars(out, j, want_rr, hdr, resid);
}

// -------------------------------------------------------------- PCG final

// Grid-stride voxels whose operands a thread of the final kernel loads
// together: two in the solo kernel (171 -> 134 us at 176x240x256), one in the
// batched kernel, whose share of blocks per subject counts on the occupancy of
// its 40 registers (two voxels: 76 registers, phase-batched fits 2% slower).
constexpr int kFinalUnroll = 2;

// delta = x + the directions not yet folded into x (none, p_{it-1}, or
// p_{it-2} and p_{it-1}), written planar, or y <- y - delta.  Each thread
// loads the operands of U voxels (one grid stride apart) before it combines
// and stores them, so that more reads are in flight per thread.
template <int K, int U>
__device__ __forceinline__ void pcg_final_body(long long N, const SolveBufs& B, float* __restrict__ delta,
                                               float* __restrict__ y_update, const WsHeader* hdr,
                                               double* report_rel, int* report_it, const VGrid& vg)
{
    const SolveScalars sc = hdr->sc;
    const bool have_x = sc.xcount > 0;
    const int pend = sc.it - sc.xcount;        // directions not yet in x: 0, 1 or 2
    const float alpha = (float)sc.alpha, alpha_prev = (float)sc.alpha_prev;
    const float4* __restrict__ pp = B.p[(sc.it + 2) % 3];    // p_{it-1}
    const float4* __restrict__ pp2 = B.p[(sc.it + 1) % 3];   // p_{it-2} when pend == 2
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const long long stride = (long long)vg.gx * blockDim.x;
    for (long long n0 = vg.bx * (long long)blockDim.x + threadIdx.x; n0 < N; n0 += U * stride) {
        float4 xv[U], p1[U], p2[U];
        float yv[U][K];
#pragma unroll
        for (int i = 0; i < U; ++i) {
            const long long n = n0 + i * stride;
            const bool in = n < N;
            xv[i] = in && have_x ? B.x[n] : zero4;
            p2[i] = in && pend == 2 ? pp2[n] : zero4;
            p1[i] = in && pend >= 1 ? pp[n] : zero4;
#pragma unroll
            for (int a = 0; a < K; ++a) yv[i][a] = in && y_update ? y_update[a * N + n] : 0.0f;
        }
#pragma unroll
        for (int i = 0; i < U; ++i) {
            const long long n = n0 + i * stride;
            if (n >= N) break;
            float v[K], t[K];
            if (have_x) {
                unpack4<K>(xv[i], v);
            } else {
#pragma unroll
                for (int a = 0; a < K; ++a) v[a] = 0.0f;
            }
            if (pend == 2) {
                unpack4<K>(p2[i], t);
#pragma unroll
                for (int a = 0; a < K; ++a) v[a] = fmaf(alpha_prev, t[a], v[a]);
            }
            if (pend >= 1) {
                unpack4<K>(p1[i], t);
#pragma unroll
                for (int a = 0; a < K; ++a) v[a] = fmaf(alpha, t[a], v[a]);
            }
#pragma unroll
            for (int a = 0; a < K; ++a) {
                if (y_update)
                    y_update[a * N + n] = yv[i][a] - v[a];
                else
                    delta[a * N + n] = v[a];
            }
        }
    }
    if (vg.bx == 0 && threadIdx.x == 0) {
        if (report_rel) *report_rel = sc.rr0 > 0.0 ? sqrt(sc.rr / sc.rr0) : 0.0;
        if (report_it) *report_it = sc.it;
    }
}

template <int K>
__global__ void __launch_bounds__(kBlock) k_pcg_final(long long N, SolveBufs B,
                                                      float* __restrict__ delta,
                                                      float* __restrict__ y_update,
                                                      const WsHeader* hdr, double* report_rel,
                                                      int* report_it)
{
    pcg_final_body<K, kFinalUnroll>(N, B, delta, y_update, hdr, report_rel, report_it, hw_grid());
}

template <int K>
__global__ void __launch_bounds__(kBlock) k_pcg_final_batch(const __grid_constant__ Batch<FinalArgs> b)
{
    const int s = batch_subject(b.start, b.n);
    const FinalArgs& a = b.a[s];
    pcg_final_body<K, 1>(a.N, a.B, a.delta, a.y_update, a.hdr, a.report_rel, a.report_it,
                      batch_grid(b.start[s], b.start[s + 1] - b.start[s], 1, 1));
}

// ------------------------------------------------------------- launchers

StencilGrid stencil_grid(const DevProblem& P, int tx, int ty, int waves, double share)
{
    StencilGrid sg;
    sg.block = dim3(tx, ty, 1);
    const int gx = (P.nx + tx - 1) / tx;
    const int gy = (P.ny + ty - 1) / ty;
    const long long tiles = (long long)gx * gy;
    // about `waves` waves of 8 resident blocks per SM (times this volume's
    // share of a launch serving several), at most kMaxBlocks blocks
    const long long target = std::max(1LL, (long long)(share * waves * 8 * kNumSm));
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
    const bool i32 = index32(P);
    if (P.K == 4) {
        if (i32) k_jtv<4, int><<<sg.grid, sg.block, 0, st>>>(P, sg.zc, y, w, jtv, red);
        else k_jtv<4, long long><<<sg.grid, sg.block, 0, st>>>(P, sg.zc, y, w, jtv, red);
    } else {
        if (i32) k_jtv<3, int><<<sg.grid, sg.block, 0, st>>>(P, sg.zc, y, w, jtv, red);
        else k_jtv<3, long long><<<sg.grid, sg.block, 0, st>>>(P, sg.zc, y, w, jtv, red);
    }
    return cudaGetLastError();
}

// What iteration j of a solve does besides the common work.
int step_mode(int j)
{
    if (j == 0) return kModeFirst;
    if (j % 2) return kModeStep;
    return j == 2 ? kModeFold : kModeFoldX;
}

template <int K>
static void launch_step_plain(const DevProblem& P, const StencilGrid& sg, int j, int want_rr,
                              const float* h, const float* w, const SolveBufs& B, WsHeader* hdr,
                              double* resid, Reduce red, cudaStream_t st)
{
    const int jm = j > 0 ? j - 1 : 0;
    const float4 *zin = B.z[jm & 1], *vin = B.v[jm & 1], *pin = B.p[(j + 2) % 3], *p2 = B.p[(j + 1) % 3];
    float4 *zout = B.z[j & 1], *vout = B.v[j & 1], *pout = B.p[j % 3];
#define MPM_STEP_PLAIN(M)                                                                          \
    k_pcg_step<K, M><<<sg.grid, sg.block, 0, st>>>(P, sg.zc, j, want_rr, h, w, zin, vin, pin, p2, zout, \
                                                   vout, pout, B.x, hdr, resid, red)
    switch (step_mode(j)) {
    case kModeFirst: MPM_STEP_PLAIN(kModeFirst); break;
    case kModeStep: MPM_STEP_PLAIN(kModeStep); break;
    case kModeFold: MPM_STEP_PLAIN(kModeFold); break;
    default: MPM_STEP_PLAIN(kModeFoldX); break;
    }
#undef MPM_STEP_PLAIN
}

template <int K>
static cudaError_t solve_k(const DevProblem& P, int cg_iters, double tol_cg, const float* h,
                           const float* w, const float* g, const float* y, float* delta,
                           float* y_update, double* resid, double* report_rel, int* report_it,
                           void* solve_ws, WsHeader* hdr, Reduce red, cudaStream_t st)
{
    const StencilGrid sg = stencil_grid(P, kTileX, kTileY);
    const StencilGrid ig = stencil_grid(P, kTileX, kTileY, kInitWaves);
    SolveBufs B = carve(P, solve_ws);
    const double tol2 = tol_cg > 0.0 ? tol_cg * tol_cg : 0.0;
    {
        LaunchScope ls(MPM_KERNEL_PCG_INIT, st);
        k_pcg_init<K><<<ig.grid, ig.block, 0, st>>>(P, ig.zc, h, w, g, y, B.z[0], tol2, hdr, resid, red);
    }
    StepMaps maps;
    const int tile = tma_tile_choice(P);
    const bool tma = tile >= 0 && make_step_maps(P, h, w, B, tile, &maps);
    const StencilGrid tg = tma ? tma_grid(P, tile) : sg;
    const bool want_resid = resid != nullptr || tol2 > 0.0;
    for (int j = 0; j < cg_iters; ++j) {
        const int rr = (want_resid || j == cg_iters - 1) ? 1 : 0;
        LaunchScope ls(MPM_KERNEL_PCG_STEP, st);
        if (tma) {
            cudaError_t e = launch_step_tma(P, tg, maps, j, step_mode(j), rr, hdr, resid, red, st);
            if (e != cudaSuccess) return e;
        } else {
            launch_step_plain<K>(P, sg, j, rr, h, w, B, hdr, resid, red, st);
        }
    }
    LaunchScope ls(MPM_KERNEL_PCG_FINAL, st);
    k_pcg_final<K><<<voxel_grid(P.N), kBlock, 0, st>>>(P.N, B, delta, y_update, hdr, report_rel,
                                                       report_it);
    return cudaGetLastError();
}

cudaError_t tma_autotune(const DevProblem& P, void* solve_ws, WsHeader* hdr, Reduce red,
                         cudaStream_t st, int* best, float* ms)
{
    *best = -1;
    // Timed on zeroed operands carved from the solve workspace's eight vectors
    // so that no buffer the launch writes is also read: iteration 3 reads z, v
    // and p from vectors 0-2, writes z, v, p to 4-6; H and w alias the
    // read-only vectors 0-3 (T N floats fit in 0-2 for K = 3, 4).
    const size_t vec = align256(sizeof(float4) * (size_t)P.N);
    char* c = static_cast<char*>(solve_ws);
    auto at = [&](int i) { return reinterpret_cast<float4*>(c + i * vec); };
    SolveBufs B;
    B.z[0] = at(0); B.z[1] = at(4);
    B.v[0] = at(1); B.v[1] = at(5);
    B.p[2] = at(2); B.p[1] = at(3); B.p[0] = at(6);
    B.x = at(7);
    const float* h = reinterpret_cast<const float*>(at(0));
    const float* w = reinterpret_cast<const float*>(at(3));
    cudaError_t e;
    if ((e = cudaMemsetAsync(solve_ws, 0, solve_ws_bytes(P), st)) != cudaSuccess) return e;
    cudaEvent_t a, b;
    if ((e = cudaEventCreate(&a)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&b)) != cudaSuccess) {
        cudaEventDestroy(a);
        return e;
    }
    float best_ms = 0.0f;
    for (int t = 0; t < tma_tile_count(); ++t) {
        ms[t] = -1.0f;
        StepMaps m;
        if (!make_step_maps(P, h, w, B, t, &m)) continue;
        const StencilGrid g = tma_grid(P, t);
        constexpr int reps = 5;
        for (int i = 0; i <= reps && e == cudaSuccess; ++i) {
            if (i == 1) e = cudaEventRecord(a, st);
            if (e == cudaSuccess) e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st);
            if (e == cudaSuccess) e = launch_step_tma(P, g, m, 3, kModeStep, 0, hdr, nullptr, red, st);
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

// ------------------------------------------------- batched launches

SolveBufs solve_bufs(const DevProblem& P, void* solve_ws) { return carve(P, solve_ws); }

cudaError_t launch_jtv_batch(int K, const JtvArgs* a, const unsigned* blocks, int n, cudaStream_t st)
{
    Batch<JtvArgs> b;
    fill_batch(b, a, blocks, n);
    bool i32 = true;
    for (int i = 0; i < n; ++i) i32 = i32 && index32(a[i].P);
    LaunchScope ls(MPM_KERNEL_JTV, st);
    const dim3 blk(kTileX, kTileY, 1);
    if (K == 4) {
        if (i32) k_jtv_batch<4, int><<<b.start[n], blk, 0, st>>>(b);
        else k_jtv_batch<4, long long><<<b.start[n], blk, 0, st>>>(b);
    } else {
        if (i32) k_jtv_batch<3, int><<<b.start[n], blk, 0, st>>>(b);
        else k_jtv_batch<3, long long><<<b.start[n], blk, 0, st>>>(b);
    }
    return cudaGetLastError();
}

cudaError_t launch_pcg_init_batch(int K, const InitArgs* a, const unsigned* blocks, int n,
                                  cudaStream_t st)
{
    Batch<InitArgs> b;
    fill_batch(b, a, blocks, n);
    LaunchScope ls(MPM_KERNEL_PCG_INIT, st);
    const dim3 blk(kTileX, kTileY, 1);
    if (K == 4)
        k_pcg_init_batch<4><<<b.start[n], blk, 0, st>>>(b);
    else
        k_pcg_init_batch<3><<<b.start[n], blk, 0, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_pcg_final_batch(int K, const FinalArgs* a, const unsigned* blocks, int n,
                                   cudaStream_t st)
{
    Batch<FinalArgs> b;
    fill_batch(b, a, blocks, n);
    LaunchScope ls(MPM_KERNEL_PCG_FINAL, st);
    if (K == 4)
        k_pcg_final_batch<4><<<b.start[n], kBlock, 0, st>>>(b);
    else
        k_pcg_final_batch<3><<<b.start[n], kBlock, 0, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_solve(const DevProblem& P, const SolveOpts& so, const float* h,
                         const float* w, const float* g, const float* y, float* delta,
                         float* y_update, double* resid, double* report_rel, int* report_it,
                         void* solve_ws, WsHeader* hdr, Reduce red, cudaStream_t st)
{
    if (so.mg_levels > 0)
        return launch_solve_mg(P, so, h, w, g, y, delta, y_update, resid, report_rel, report_it,
                               solve_ws, hdr, red, st);
    if (P.K == 4)
        return solve_k<4>(P, so.cg_iters, so.tol_cg, h, w, g, y, delta, y_update, resid, report_rel,
                          report_it, solve_ws, hdr, red, st);
    return solve_k<3>(P, so.cg_iters, so.tol_cg, h, w, g, y, delta, y_update, resid, report_rel,
                      report_it, solve_ws, hdr, red, st);
}

}  // namespace mpm
