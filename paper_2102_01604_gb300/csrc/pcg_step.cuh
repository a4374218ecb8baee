// pcg_step.cuh -- per-voxel arithmetic of the block-Jacobi PCG of the Newton
// system (H + L) delta = g + L y (Eq. 42, Sec. 2.6), shared by the TMA-staged
// iteration kernel (stencil_tma.cu) and the plain one (stencil_kernels.cu) so
// that both compute every voxel with the same operations in the same order.
//
// One kernel per PCG iteration.  The textbook recurrence keeps r and z = M^-1 r
// and needs two grid-wide reductions per iteration (p.q for alpha, r.z for
// beta).  Here the preconditioned residual is carried instead and updated as
//     z_{j+1} = z_j - alpha_j v_j,   v_j = M^-1 q_j,   q_j = (H + L) p_j,
// which is the same vector as M^-1 (r_j - alpha_j q_j) (M is linear), and the
// next r.z is expanded from quantities of iteration j alone:
//     r_{j+1}.z_{j+1} = r_j.z_j - 2 alpha_j q_j.z_j + alpha_j^2 q_j.v_j
// with r_j = M z_j formed per voxel (M symmetric, so r_j.v_j = z_j.q_j).  All
// four sums are reduced in the same launch as q_j, so alpha_j and beta_j are
// known when iteration j + 1 starts: it forms z_{j+1} and p_{j+1} = z_{j+1} +
// beta_j p_j for its tile and halo from (z_j, v_j, p_j), applies the operator
// and writes z, v and p once.  |r_{j+1}|^2 is expanded the same way when the
// residual norm is wanted.  r.z is recomputed directly (z_j.M z_j) in every
// iteration, so the expansion spans one step and errors do not accumulate.
//
// The preconditioner block M_n = H_n + diag(lambda_k d_n), d_n = sum of the
// six edge coefficients, is factorised in every iteration from H and the JTV
// weights (its float32 Cholesky factor is the same each time), so the solve
// stores no factor.
//
// The solve's own vectors (z, v, p and the accumulated x) are stored voxel
// by voxel, four floats per voxel (K = 3 leaves the fourth zero), so one
// 16-byte access moves all maps of a voxel; H, w and the caller's arrays stay
// planar [component][N].
#pragma once

#include "device_common.cuh"

namespace mpm {

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
        for (int k = 0; k < j; ++k) s = fmaf(-L[lo(j, k)], L[lo(j, k)], s);
        if (!(s > 0.0f)) {
            ok = false;
            s = fmaxf(fabsf(M[j][j]), 1e-30f);
        }
        const float rj = rsqrtf(s);      // 1 / L_jj
        L[lo(j, j)] = rj;
#pragma unroll
        for (int i = j + 1; i < K; ++i) {
            float v = M[i][j];
#pragma unroll
            for (int k = 0; k < j; ++k) v = fmaf(-L[lo(i, k)], L[lo(j, k)], v);
            L[lo(i, j)] = v * rj;
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
        for (int k = 0; k < i; ++k) v = fmaf(-L[lo(i, k)], t[k], v);
        t[i] = v * L[lo(i, i)];
    }
#pragma unroll
    for (int i = K - 1; i >= 0; --i) {
        float v = t[i];
#pragma unroll
        for (int k = i + 1; k < K; ++k) v = fmaf(-L[lo(k, i)], z[k], v);
        z[i] = v * L[lo(i, i)];
    }
}

// Preconditioner block M = H + diag(lambda_k d) from the packed H.
template <int K>
__device__ __forceinline__ void precond_block(const DevProblem& P, const float (&hv)[K * (K + 1) / 2],
                                              float d, float (&M)[K][K])
{
#pragma unroll
    for (int a = 0; a < K; ++a)
#pragma unroll
        for (int b = a; b < K; ++b) M[a][b] = M[b][a] = hv[tri(K, a, b)];
#pragma unroll
    for (int a = 0; a < K; ++a) M[a][a] = fmaf(P.lambda[a], d, M[a][a]);
}

// Sum of the six edge coefficients (order x-, x+, y-, y+, z-, z+).
__device__ __forceinline__ float edge_sum(const float (&c)[6])
{
    return ((((c[0] + c[1]) + c[2]) + c[3]) + c[4]) + c[5];
}

// Per-solve workspace buffers: [N] float4 each (voxel-interleaved maps),
// 256-byte aligned.
struct SolveBufs {
    float4* z[2];    // preconditioned residual z_j in z[j & 1]
    float4* v[2];    // v_j = M^-1 q_j in v[j & 1]
    float4* p[3];    // direction p_j in p[j % 3]
    float4* x;       // sum of the directions folded so far, alpha_i p_i
};

template <int K>
__device__ __forceinline__ void unpack4(const float4& a, float (&o)[K])
{
    o[0] = a.x;
    o[1] = a.y;
    o[2] = a.z;
    if constexpr (K > 3) o[3] = a.w;
}

template <int K>
__device__ __forceinline__ float4 pack4(const float (&o)[K])
{
    if constexpr (K > 3) return make_float4(o[0], o[1], o[2], o[3]);
    else return make_float4(o[0], o[1], o[2], 0.0f);
}

// What one iteration's launch does besides the common work.
enum : int {
    kModeFirst = 0,    // j = 0: z_0 comes from the init kernel, p_0 = z_0
    kModeStep = 1,     // odd j
    kModeFold = 2,     // j = 2: also x = alpha_0 p_0 + alpha_1 p_1
    kModeFoldX = 3     // even j > 2: also x += alpha_{j-2} p_{j-2} + alpha_{j-1} p_{j-1}
};

// Sums reduced by every iteration, in this order.
enum : int { kSumPQ, kSumZQ, kSumVQ, kSumZR, kSumRR, kSumRQ, kSumQQ, kStepSums };

// z_j and p_j of one point from the previous iteration's z, v, p (at j = 0,
// z is z_0 and v, p are not read).
template <int K, bool FIRST>
__device__ __forceinline__ void step_point(float alpha, float beta, const float4& z4, const float4& v4,
                                           const float4& p4, float (&zj)[K], float (&pj)[K])
{
    float z[K], v[K], p[K];
    unpack4<K>(z4, z);
    unpack4<K>(v4, v);
    unpack4<K>(p4, p);
#pragma unroll
    for (int a = 0; a < K; ++a) {
        zj[a] = FIRST ? z[a] : fmaf(-alpha, v[a], z[a]);
        pj[a] = FIRST ? zj[a] : fmaf(beta, p[a], zj[a]);
    }
}

// x after folding in the two latest directions, in the order of two single
// updates: x + alpha_{j-2} p_{j-2}, then + alpha_{j-1} p_{j-1} (all four
// components; the padding of K = 3 stays zero).
__device__ __forceinline__ float4 fold_x(const float4& x, float alpha_prev, const float4& p2, float alpha,
                                         const float4& p1)
{
    return make_float4(fmaf(alpha, p1.x, fmaf(alpha_prev, p2.x, x.x)),
                       fmaf(alpha, p1.y, fmaf(alpha_prev, p2.y, x.y)),
                       fmaf(alpha, p1.z, fmaf(alpha_prev, p2.z, x.z)),
                       fmaf(alpha, p1.w, fmaf(alpha_prev, p2.w, x.w)));
}

// One voxel of iteration j: q = (H + L) p_j with the weighted 7-point stencil
//     (L p)_k = lambda_k sum_m c_m (p_k[n] - p_k[m]),  c_m = (w_n + w_m) / h^2
// (c_m = 0 for neighbours outside the volume, whose values nb then only need
// to be finite), v = M^-1 q, r = M z_j, and the voxel's terms of the sums.
// nb(m, a) returns p_j of map a at neighbour m (order x-, x+, y-, y+, z-, z+).
template <int K, class NB>
__device__ __forceinline__ void step_voxel(const DevProblem& P, const float (&c)[6],
                                           const float (&zj)[K], const float (&pj)[K], NB nb,
                                           const float (&hv)[K * (K + 1) / 2], bool resid,
                                           float (&v)[K], float (&sums)[kStepSums])
{
    float M[K][K];
    precond_block<K>(P, hv, edge_sum(c), M);
    float q[K];
#pragma unroll
    for (int a = 0; a < K; ++a) {
        const float pa = pj[a];
        float s = c[0] * (pa - nb(0, a));
#pragma unroll
        for (int m = 1; m < 6; ++m) s = fmaf(c[m], pa - nb(m, a), s);
        float acc = P.lambda[a] * s;
#pragma unroll
        for (int b = 0; b < K; ++b) acc = fmaf(hv[a < b ? tri(K, a, b) : tri(K, b, a)], pj[b], acc);
        q[a] = acc;
    }
    float L[K * (K + 1) / 2];
    cholesky_f32<K>(M, L);
    chol_apply<K>(L, q, v);
    float r[K];
#pragma unroll
    for (int a = 0; a < K; ++a) {
        float acc = M[a][0] * zj[0];
#pragma unroll
        for (int b = 1; b < K; ++b) acc = fmaf(M[a][b], zj[b], acc);
        r[a] = acc;
    }
    float pq = pj[0] * q[0], zq = zj[0] * q[0], vq = v[0] * q[0], zr = zj[0] * r[0];
#pragma unroll
    for (int a = 1; a < K; ++a) {
        pq = fmaf(pj[a], q[a], pq);
        zq = fmaf(zj[a], q[a], zq);
        vq = fmaf(v[a], q[a], vq);
        zr = fmaf(zj[a], r[a], zr);
    }
    sums[kSumPQ] = pq;
    sums[kSumZQ] = zq;
    sums[kSumVQ] = vq;
    sums[kSumZR] = zr;
    float rr = 0.0f, rq = 0.0f, qq = 0.0f;
    if (resid) {
        rr = r[0] * r[0];
        rq = r[0] * q[0];
        qq = q[0] * q[0];
#pragma unroll
        for (int a = 1; a < K; ++a) {
            rr = fmaf(r[a], r[a], rr);
            rq = fmaf(r[a], q[a], rq);
            qq = fmaf(q[a], q[a], qq);
        }
    }
    sums[kSumRR] = rr;
    sums[kSumRQ] = rq;
    sums[kSumQQ] = qq;
}

// Scalars of iteration j from its reduced sums (the last block of the launch):
// alpha_j = r_j.z_j / p_j.q_j, the expanded r_{j+1}.z_{j+1} and |r_{j+1}|^2,
// beta_j and the stopping tests.  A breakdown (p.q or r.z not positive, or a
// NaN) stops the solve without a step.
__device__ __forceinline__ void step_scalars(const double (&s)[kStepSums], int j, bool resid_sums,
                                             WsHeader* hdr, double* resid)
{
    SolveScalars& sc = hdr->sc;
    bool bad = false;
#pragma unroll
    for (int i = 0; i < kStepSums; ++i) bad |= !(s[i] == s[i]);
    if (bad) atomicOr(&hdr->status, kStatusNaN);
    const double pq = s[kSumPQ], rz = s[kSumZR];
    if (bad || !(pq > 0.0) || !(rz > 0.0)) {
        sc.done = 1;                       // no further step; the alphas keep their values
        return;
    }
    const double alpha = rz / pq;
    const double rz_next = rz - 2.0 * alpha * s[kSumZQ] + alpha * alpha * s[kSumVQ];
    sc.alpha_prev = sc.alpha;
    sc.alpha = alpha;
    sc.beta = rz_next / rz;
    sc.rz = rz_next;
    sc.it = j + 1;
    if (resid_sums) {
        const double rr = s[kSumRR] - 2.0 * alpha * s[kSumRQ] + alpha * alpha * s[kSumQQ];
        sc.rr = rr > 0.0 ? rr : 0.0;
        if (resid) resid[j + 1] = sqrt(sc.rr);
        if (sc.tol2 > 0.0 && sc.rr <= sc.tol2 * sc.rr0) sc.done = 1;
    }
    if (!(rz_next > 0.0)) sc.done = 1;
}

}  // namespace mpm
