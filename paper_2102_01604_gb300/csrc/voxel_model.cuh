// voxel_model.cuh -- the per-voxel signal model shared by the voxel passes
// (voxel_kernels.cu: k_forward, k_grad_hess; projection.cu: the projected
// voxel pass).  Eq. 26 with the B1 footnote, its derivatives (Eqs. 27-34)
// and the per-contrast accumulation of Eqs. 6, 24 and 25.
#pragma once

#include "mpm_internal.cuh"

namespace mpm {

// Hint the line holding p into L2 (the voxel passes fetch their next voxel's
// operands this way while they compute the current one).
__device__ __forceinline__ void prefetch_l2(const void* p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

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

__device__ __forceinline__ ContrastTerms contrast_terms(const DevProblem& P, int c, float a,
                                                        const Relax& R, float dl, float m,
                                                        float bp, float bm)
{
    ContrastTerms t;
    float sa, ca;
    sincosf(P.alpha[c] * bp, &sa, &ca);
    const float omc = __fdividef(sa * sa, 1.0f + ca);
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
    // one echo: signal s, q2 = -TE r2, measured value xv
    __device__ __forceinline__ void add(float s, float q2, float xv)
    {
        const float r = s - xv;
        const float ss = s * s;
        S0 += ss;
        S1 += ss * q2;
        S2 += ss * q2 * q2;
        const float rs = r * s;
        R0 += rs;
        R1 += rs * q2;
        N2 += r * r;
        if (PRE != 2) {
            const float ars = fabsf(rs);
            A0 += ars;
            A2 += ars * fabsf((1.0f + q2) * q2);
            if (PRE == 1) B1 += ars * fabsf(q2);
        }
    }
};

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
            q2 += dq;
            s *= rho;
        }
    } else {
        es.add(s, q2, load_echo<XT>(xp, 0));
#pragma unroll 4
        for (int e = 1; e < ne; ++e) {
            q2 = -P.te[i0 + e] * r2;
            es.add(t.s0 * expf(q2), q2, load_echo<XT>(xp, e * stride));
        }
    }
    const float S0 = es.S0, S1 = es.S1, S2 = es.S2, R0 = es.R0, R1 = es.R1, N2 = es.N2;
    const float A0 = es.A0, A2 = es.A2, B1 = es.B1;
    const float is2 = P.isig2[c];
    const float q1 = t.q1, qd = t.qd;
    G[0] += is2 * R0;
    G[1] += is2 * R0 * q1;
    G[2] += is2 * R1;
    H[tri(K, 0, 0)] += is2 * S0;
    H[tri(K, 0, 1)] += is2 * S0 * q1;
    H[tri(K, 0, 2)] += is2 * S1;
    H[tri(K, 1, 1)] += is2 * S0 * q1 * q1;
    H[tri(K, 1, 2)] += is2 * S1 * q1;
    H[tri(K, 2, 2)] += is2 * S2;
    if (K == 4) {
        G[K - 1] += is2 * R0 * qd;
        H[tri(K, 0, K - 1)] += is2 * S0 * qd;
        H[tri(K, 1, K - 1)] += is2 * S0 * q1 * qd;
        H[tri(K, 2, K - 1)] += is2 * S1 * qd;
        H[tri(K, K - 1, K - 1)] += is2 * S0 * qd * qd;
    }
    if (PRE == 0) {
        H[tri(K, 0, 0)] += is2 * A0;
        H[tri(K, 1, 1)] += is2 * A0 * fabsf(t.h1 * q1);
        H[tri(K, 2, 2)] += is2 * A2;
        if (K == 4) H[tri(K, K - 1, K - 1)] += is2 * A0 * fabsf(t.hd * qd);
    } else if (PRE == 1) {
        const float aq1 = fabsf(q1), aqd = fabsf(qd);
        const float c13 = fabsf(q1 * qd + t.cross);
        H[tri(K, 0, 0)] += is2 * (A0 * (1.0f + aq1 + aqd) + B1);
        H[tri(K, 1, 1)] += is2 * (A0 * (fabsf(t.h1 * q1) + aq1 + c13) + aq1 * B1);
        H[tri(K, 2, 2)] += is2 * (A2 + B1 * (1.0f + aq1 + aqd));
        if (K == 4)
            H[tri(K, K - 1, K - 1)] +=
                is2 * (A0 * (fabsf(t.hd * qd) + aqd + c13) + aqd * B1);
    }
    nll_v += 0.5f * is2 * N2;
}

}  // namespace mpm
