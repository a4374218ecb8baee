// voxel_model.cuh -- the per-voxel signal model shared by the voxel passes
// (voxel_kernels.cu: k_forward, k_grad_hess; projection.cu: the projected
// voxel pass).  Eq. 26 with the B1 footnote, its derivatives (Eqs. 27-34)
// and the per-contrast accumulation of Eqs. 6, 24 and 25.
#pragma once

#include "mpm_internal.cuh"

namespace mpm {

// Per-contrast factors shared by every echo of contrast c in one voxel.  With
// q_k = (ds/dy_k) / s  (Eqs. 27-30):
//   q_A = 1, q_R1 = q1, q_R2* = -TE r2 (echo dependent), q_delta = qd,
// and the diagonal second derivatives (Eqs. 31-34) are
//   d2s/dA2 = s, d2s/dR1^2 = h1 q1 s, d2s/dR2*^2 = (1 + q2) q2 s, d2s/ddelta^2 = hd qd s.
// `cross` is the extra term of d2s/dR1 ddelta = (q1 qd + cross) s.
// Cancellation-free forms in float32: 1 - E = -expm1(-r1 TR),
// 1 - cos(a) = sin(a)^2 / (1 + cos(a)), 1 - (1-delta) cos(a) = (1 - cos a) + delta cos a,
// D = 1 - (1-delta) cos(a) E = (1 - E) + E (1 - (1-delta) cos a).
struct ContrastTerms {
    float s0, q1, qd, h1, hd, cross;
};

// Longitudinal relaxation over one TR: tt = r1 TR, E = exp(-tt), omE = 1 - E.
struct Relax {
    float tt, E, omE;
};

__device__ __forceinline__ Relax relax(float tr, float r1)
{
    Relax R;
    R.tt = tr * r1;
    R.E = expf(-R.tt);
    R.omE = -expm1f(-R.tt);
    return R;
}

// The local flip angle's factors: sa = sin(a), ca = cos(a), omc = 1 - cos(a).
struct Flip {
    float sa, ca, omc;
};

__device__ __forceinline__ Flip flip(float angle)
{
    Flip f;
    sincosf(angle, &f.sa, &f.ca);
    f.omc = __fdividef(f.sa * f.sa, 1.0f + f.ca);
    return f;
}

// ContrastTerms of contrast c from the flip factors of its local angle
// alpha_c b1+.
__device__ __forceinline__ ContrastTerms contrast_terms_f(const DevProblem& P, int c, float a,
                                                          const Relax& R, float dl, float m,
                                                          const Flip& f, float bm)
{
    ContrastTerms t;
    const float sa = f.sa, ca = f.ca, omc = f.omc;
    const float tt = R.tt, E = R.E, omE = R.omE;
    const bool mt = P.mt[c] != 0;
    const float d = mt ? dl : 0.0f;
    const float mm = mt ? m : 1.0f;
    const float omcm = omc + d * ca;                 // 1 - m cos(a)
    const float D = omE + E * omcm;                  // 1 - m cos(a) E
    const float iD = 1.0f / D;
    t.s0 = bm * a * sa * mm * omE * iD;
    t.q1 = __fdividef(tt * E * omcm * iD, omE);
    t.qd = mt ? -d * iD : 0.0f;
    t.h1 = 1.0f - tt * (2.0f - D) * iD;              // 1 + m cos(a) E = 2 - D
    t.hd = 2.0f * mm * (omE + E * omc) * iD - 1.0f;  // 1 - cos(a) E = (1-E) + E (1 - cos a)
    t.cross = mt ? tt * E * ca * d * mm * iD * iD : 0.0f;
    return t;
}

__device__ __forceinline__ ContrastTerms contrast_terms(const DevProblem& P, int c, float a,
                                                        const Relax& R, float dl, float m,
                                                        float bp, float bm)
{
    return contrast_terms_f(P, c, a, R, dl, m, flip(P.alpha[c] * bp), bm);
}

// exp of the log-parameters; delta = logistic(y_delta) and m = 1 - delta from
// one exponential of -|y_delta| (no overflow, no cancellation).
__device__ __forceinline__ void map_params(const float* __restrict__ y, long long N,
                                           long long n, int K, float& a, float& r1,
                                           float& r2, float& dl, float& m)
{
    a = expf(__ldg(y + n));
    r1 = expf(__ldg(y + N + n));
    r2 = expf(__ldg(y + 2 * N + n));
    dl = 0.0f;
    m = 1.0f;
    if (K == 4) {
        const float yd = __ldg(y + 3 * N + n);
        const float e = expf(-fabsf(yd));
        const float i1 = 1.0f / (1.0f + e);
        const float big = i1, small = e * i1;
        dl = yd >= 0.0f ? big : small;
        m = yd >= 0.0f ? small : big;
    }
}

// exp of the log-parameters from values already in registers (same
// arithmetic as map_params).
__device__ __forceinline__ void map_params_v(const float* yv, int K, float& a, float& r1,
                                             float& r2, float& dl, float& m)
{
    a = expf(yv[0]);
    r1 = expf(yv[1]);
    r2 = expf(yv[2]);
    dl = 0.0f;
    m = 1.0f;
    if (K == 4) {
        const float yd = yv[3];
        const float e = expf(-fabsf(yd));
        const float i1 = 1.0f / (1.0f + e);
        const float big = i1, small = e * i1;
        dl = yd >= 0.0f ? big : small;
        m = yd >= 0.0f ? small : big;
    }
}

// Per contrast the echo sums
//   S0 = sum s^2, S1 = sum s^2 q2, S2 = sum s^2 q2^2,
//   R0 = sum r s, R1 = sum r s q2, N2 = sum r^2,
//   A0 = sum |r s|, A2 = sum |r s| |(1 + q2) q2|, B1 = sum |r s| |q2|
// give, with v = (1, q1, 0, qd) and e2 the log R2* axis,
//   g += (R0 v + R1 e2) / sigma^2
//   P += (S0 v v' + S1 (v e2' + e2 v') + S2 e2 e2' + loading) / sigma^2
// which is Eq. 24 summed over the echoes of the contrast.  xp points at the
// first echo of contrast c in this voxel; echo e is at xp[e * stride].
template <int PRE>
struct EchoSums {
    float S0 = 0.f, S1 = 0.f, S2 = 0.f, R0 = 0.f, R1 = 0.f, N2 = 0.f;
    float A0 = 0.f, A2 = 0.f, B1 = 0.f;
    // One echo: signal s, q2 = -TE r2, measured value xv.  Every rounding is
    // spelled out (no contraction left to the compiler), so EchoSums2 below
    // gives each of its two voxels exactly these sums.  (1 + q2) q2 is taken
    // as fma(q2, q2, q2).
    __device__ __forceinline__ void add(float s, float q2, float xv)
    {
        const float r = __fadd_rn(s, -xv);
        const float rs = __fmul_rn(r, s);
        R0 = __fmaf_rn(r, s, R0);
        R1 = __fmaf_rn(rs, q2, R1);
        N2 = __fmaf_rn(r, r, N2);
        const float ss = __fmul_rn(s, s);
        S0 = __fmaf_rn(s, s, S0);
        S1 = __fmaf_rn(ss, q2, S1);
        S2 = __fmaf_rn(__fmul_rn(ss, q2), q2, S2);
        if (PRE != 2) {
            const float ars = fabsf(rs);
            A0 = __fadd_rn(A0, ars);
            A2 = __fmaf_rn(ars, fabsf(__fmaf_rn(q2, q2, q2)), A2);
            if (PRE == 1) B1 = __fmaf_rn(ars, fabsf(q2), B1);
        }
    }
};

__device__ __forceinline__ float2 abs2(float2 v) { return make_float2(fabsf(v.x), fabsf(v.y)); }
__device__ __forceinline__ float2 neg2(float2 v) { return make_float2(-v.x, -v.y); }

// EchoSums of two voxels at once, in paired float32 instructions (each lane
// rounds as its scalar counterpart in EchoSums::add).
template <int PRE>
struct EchoSums2 {
    float2 S0 = {0.f, 0.f}, S1 = {0.f, 0.f}, S2 = {0.f, 0.f}, R0 = {0.f, 0.f}, R1 = {0.f, 0.f};
    float2 N2 = {0.f, 0.f}, A0 = {0.f, 0.f}, A2 = {0.f, 0.f}, B1 = {0.f, 0.f};
    __device__ __forceinline__ void add(float2 s, float2 q2, float2 xv)
    {
        const float2 r = __fadd2_rn(s, neg2(xv));
        const float2 rs = __fmul2_rn(r, s);
        R0 = __ffma2_rn(r, s, R0);
        R1 = __ffma2_rn(rs, q2, R1);
        N2 = __ffma2_rn(r, r, N2);
        const float2 ss = __fmul2_rn(s, s);
        S0 = __ffma2_rn(s, s, S0);
        S1 = __ffma2_rn(ss, q2, S1);
        S2 = __ffma2_rn(__fmul2_rn(ss, q2), q2, S2);
        if (PRE != 2) {
            const float2 ars = abs2(rs);
            A0 = __fadd2_rn(A0, ars);
            A2 = __ffma2_rn(ars, abs2(__ffma2_rn(q2, q2, q2)), A2);
            if (PRE == 1) B1 = __ffma2_rn(ars, abs2(q2), B1);
        }
    }
    // the sums of voxel v (0: x lanes, 1: y lanes)
    __device__ __forceinline__ EchoSums<PRE> lane(int v) const
    {
        EchoSums<PRE> e;
        auto pick = [v](float2 a) { return v == 0 ? a.x : a.y; };
        e.S0 = pick(S0), e.S1 = pick(S1), e.S2 = pick(S2), e.R0 = pick(R0), e.R1 = pick(R1);
        e.N2 = pick(N2), e.A0 = pick(A0), e.A2 = pick(A2), e.B1 = pick(B1);
        return e;
    }
};

// Elementwise float32 arithmetic on one voxel (float) or on two at once
// (float2, paired instructions), every rounding explicit, so that each lane
// of the paired form rounds exactly as the single form.
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float vabs(float a) { return fabsf(a); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vabs(float2 a) { return abs2(a); }
template <typename F>
__device__ __forceinline__ F vsplat(float v);
template <>
__device__ __forceinline__ float vsplat<float>(float v) { return v; }
template <>
__device__ __forceinline__ float2 vsplat<float2>(float v) { return make_float2(v, v); }

// Eq. 24 of contrast c from its echo sums (S0 .. B1) and factors (q1, qd,
// h1, hd, cross of ContrastTerms): the gradient, Hessian and NLL terms added
// to G, H and nll, for one voxel (F = float) or two (F = float2).
template <int K, int PRE, typename F>
__device__ __forceinline__ void finish_terms(float is2s, F q1, F qd, F h1, F hd, F cross, F S0, F S1,
                                             F S2, F R0, F R1, F N2, F A0, F A2, F B1, F (&G)[K],
                                             F (&H)[K * (K + 1) / 2], F& nll)
{
    const F is2 = vsplat<F>(is2s);
    const F is2R0 = vmul(is2, R0), is2S0 = vmul(is2, S0), is2S1 = vmul(is2, S1);
    const F is2S0q1 = vmul(is2S0, q1);
    G[0] = vadd(G[0], is2R0);
    G[1] = vfma(is2R0, q1, G[1]);
    G[2] = vfma(is2, R1, G[2]);
    H[tri(K, 0, 0)] = vadd(H[tri(K, 0, 0)], is2S0);
    H[tri(K, 0, 1)] = vadd(H[tri(K, 0, 1)], is2S0q1);
    H[tri(K, 0, 2)] = vadd(H[tri(K, 0, 2)], is2S1);
    H[tri(K, 1, 1)] = vfma(is2S0q1, q1, H[tri(K, 1, 1)]);
    H[tri(K, 1, 2)] = vfma(is2S1, q1, H[tri(K, 1, 2)]);
    H[tri(K, 2, 2)] = vfma(is2, S2, H[tri(K, 2, 2)]);
    if (K == 4) {
        G[K - 1] = vfma(is2R0, qd, G[K - 1]);
        H[tri(K, 0, K - 1)] = vfma(is2S0, qd, H[tri(K, 0, K - 1)]);
        H[tri(K, 1, K - 1)] = vfma(is2S0q1, qd, H[tri(K, 1, K - 1)]);
        H[tri(K, 2, K - 1)] = vfma(is2S1, qd, H[tri(K, 2, K - 1)]);
        H[tri(K, K - 1, K - 1)] = vfma(vmul(is2S0, qd), qd, H[tri(K, K - 1, K - 1)]);
    }
    if (PRE == 0) {
        const F is2A0 = vmul(is2, A0);
        H[tri(K, 0, 0)] = vadd(H[tri(K, 0, 0)], is2A0);
        H[tri(K, 1, 1)] = vfma(is2A0, vabs(vmul(h1, q1)), H[tri(K, 1, 1)]);
        H[tri(K, 2, 2)] = vfma(is2, A2, H[tri(K, 2, 2)]);
        if (K == 4) H[tri(K, K - 1, K - 1)] = vfma(is2A0, vabs(vmul(hd, qd)), H[tri(K, K - 1, K - 1)]);
    } else if (PRE == 1) {
        const F aq1 = vabs(q1), aqd = vabs(qd);
        const F c13 = vabs(vfma(q1, qd, cross));
        const F t1 = vadd(vadd(vsplat<F>(1.0f), aq1), aqd);      // 1 + |q1| + |qd|
        H[tri(K, 0, 0)] = vfma(is2, vfma(A0, t1, B1), H[tri(K, 0, 0)]);
        const F u1 = vadd(vadd(vabs(vmul(h1, q1)), aq1), c13);
        H[tri(K, 1, 1)] = vfma(is2, vfma(aq1, B1, vmul(A0, u1)), H[tri(K, 1, 1)]);
        H[tri(K, 2, 2)] = vfma(is2, vfma(B1, t1, A2), H[tri(K, 2, 2)]);
        if (K == 4) {
            const F ud = vadd(vadd(vabs(vmul(hd, qd)), aqd), c13);
            H[tri(K, K - 1, K - 1)] = vfma(is2, vfma(aqd, B1, vmul(A0, ud)), H[tri(K, K - 1, K - 1)]);
        }
    }
    nll = vfma(vmul(vsplat<F>(0.5f), is2), N2, nll);
}

// finish_terms for one voxel from its EchoSums.
template <int K, int PRE>
__device__ __forceinline__ void finish_contrast(const DevProblem& P, int c, const ContrastTerms& t,
                                                const EchoSums<PRE>& es, float (&G)[K],
                                                float (&H)[K * (K + 1) / 2], float& nll_v)
{
    finish_terms<K, PRE, float>(P.isig2[c], t.q1, t.qd, t.h1, t.hd, t.cross, es.S0, es.S1, es.S2, es.R0,
                                es.R1, es.N2, es.A0, es.A2, es.B1, G, H, nll_v);
}

// finish_terms for two voxels at once from their paired sums.
template <int K, int PRE>
__device__ __forceinline__ void finish_contrast2(const DevProblem& P, int c, const ContrastTerms& t0,
                                                 const ContrastTerms& t1, const EchoSums2<PRE>& es,
                                                 float2 (&G)[K], float2 (&H)[K * (K + 1) / 2],
                                                 float2& nll)
{
    finish_terms<K, PRE, float2>(P.isig2[c], make_float2(t0.q1, t1.q1), make_float2(t0.qd, t1.qd),
                                 make_float2(t0.h1, t1.h1), make_float2(t0.hd, t1.hd),
                                 make_float2(t0.cross, t1.cross), es.S0, es.S1, es.S2, es.R0, es.R1,
                                 es.N2, es.A0, es.A2, es.B1, G, H, nll);
}

template <int K, int PRE, typename XT>
__device__ __forceinline__ void accumulate_contrast(const DevProblem& P, int c,
                                                    const ContrastTerms& t, float r2,
                                                    const XT* xp, long long stride,
                                                    float (&G)[K], float (&H)[K * (K + 1) / 2],
                                                    float& nll_v)
{
    EchoSums<PRE> es;
    const int i0 = P.echo0[c];
    const int ne = P.n_echoes[c];
    float q2 = -P.te[i0] * r2;
    float s = t.s0 * expf(q2);
    if (P.te_uniform[c] != 0) {
        // equally spaced echoes: s_e = s_0 exp(-TE_0 r2) rho^e, rho = exp(-dTE r2)
        const float dq = -P.dte[c] * r2;
        const float rho = expf(dq);
#pragma unroll 4
        for (int e = 0; e < ne; ++e) {
            es.add(s, q2, load_echo<XT>(xp, e * stride));
            q2 = __fadd_rn(q2, dq);
            s = __fmul_rn(s, rho);
        }
    } else {
        es.add(s, q2, load_echo<XT>(xp, 0));
#pragma unroll 4
        for (int e = 1; e < ne; ++e) {
            q2 = -P.te[i0 + e] * r2;
            es.add(t.s0 * expf(q2), q2, load_echo<XT>(xp, e * stride));
        }
    }
    finish_contrast<K, PRE>(P, c, t, es, G, H, nll_v);
}

// V consecutive values from p (p aligned to V elements), as floats.
template <int V, typename T>
__device__ __forceinline__ void load_vec(const T* __restrict__ p, float (&o)[V]);

template <>
__device__ __forceinline__ void load_vec<1, float>(const float* __restrict__ p, float (&o)[1])
{
    o[0] = __ldg(p);
}

template <>
__device__ __forceinline__ void load_vec<2, float>(const float* __restrict__ p, float (&o)[2])
{
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    o[0] = v.x;
    o[1] = v.y;
}

template <>
__device__ __forceinline__ void load_vec<1, __nv_bfloat16>(const __nv_bfloat16* __restrict__ p,
                                                           float (&o)[1])
{
    o[0] = __bfloat162float(p[0]);
}

template <>
__device__ __forceinline__ void load_vec<2, __nv_bfloat16>(const __nv_bfloat16* __restrict__ p,
                                                           float (&o)[2])
{
    const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(p);
    o[0] = __low2float(v);
    o[1] = __high2float(v);
}

// V consecutive floats to p (p aligned to V elements).
template <int V>
__device__ __forceinline__ void store_vec(float* p, const float (&v)[V])
{
    if (V == 2)
        *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
    else
        p[0] = v[0];
}

// accumulate_contrast for V neighbouring voxels at once: one vector load per
// echo serves all V, and their echo recurrences run side by side.  Each
// voxel's arithmetic is that of accumulate_contrast, in the same order.
template <int K, int PRE, typename XT, int V>
__device__ __forceinline__ void accumulate_contrast_v(const DevProblem& P, int c,
                                                      const ContrastTerms (&t)[V],
                                                      const float (&r2)[V], const XT* xp,
                                                      long long stride, float (&G)[V][K],
                                                      float (&H)[V][K * (K + 1) / 2],
                                                      float (&nll_v)[V])
{
    static_assert(V == 1 || V == 2, "one or two voxels per thread");
    if (V == 1) {
        accumulate_contrast<K, PRE, XT>(P, c, t[0], r2[0], xp, stride, G[0], H[0], nll_v[0]);
        return;
    }
    EchoSums2<PRE> es;
    const int i0 = P.echo0[c];
    const int ne = P.n_echoes[c];
    const float2 r22 = make_float2(r2[0], r2[V - 1]);
    const float te0 = -P.te[i0];
    float2 q2 = make_float2(te0 * r22.x, te0 * r22.y);
    float2 s = make_float2(t[0].s0 * expf(q2.x), t[V - 1].s0 * expf(q2.y));
    if (P.te_uniform[c] != 0) {
        const float dte = -P.dte[c];
        const float2 dq = make_float2(dte * r22.x, dte * r22.y);
        const float2 rho = make_float2(expf(dq.x), expf(dq.y));
#pragma unroll 4
        for (int e = 0; e < ne; ++e) {
            float xv[2];
            load_vec<2, XT>(xp + e * stride, xv);
            es.add(s, q2, make_float2(xv[0], xv[1]));
            q2 = __fadd2_rn(q2, dq);
            s = __fmul2_rn(s, rho);
        }
    } else {
        float xv[2];
        load_vec<2, XT>(xp, xv);
        es.add(s, q2, make_float2(xv[0], xv[1]));
#pragma unroll 4
        for (int e = 1; e < ne; ++e) {
            load_vec<2, XT>(xp + e * stride, xv);
            const float te = -P.te[i0 + e];
            q2 = make_float2(te * r22.x, te * r22.y);
            s = make_float2(t[0].s0 * expf(q2.x), t[V - 1].s0 * expf(q2.y));
            es.add(s, q2, make_float2(xv[0], xv[1]));
        }
    }
    constexpr int T = K * (K + 1) / 2;
    float2 G2[K], H2[T], n2 = make_float2(nll_v[0], nll_v[V - 1]);
#pragma unroll
    for (int k = 0; k < K; ++k) G2[k] = make_float2(G[0][k], G[V - 1][k]);
#pragma unroll
    for (int k = 0; k < T; ++k) H2[k] = make_float2(H[0][k], H[V - 1][k]);
    finish_contrast2<K, PRE>(P, c, t[0], t[V - 1], es, G2, H2, n2);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        G[0][k] = G2[k].x;
        G[V - 1][k] = G2[k].y;
    }
#pragma unroll
    for (int k = 0; k < T; ++k) {
        H[0][k] = H2[k].x;
        H[V - 1][k] = H2[k].y;
    }
    nll_v[0] = n2.x;
    nll_v[V - 1] = n2.y;
}

}  // namespace mpm
