// init_maps.cuh -- the constant initial maps of a fit from the mean intensity
// of every image (k_init_maps derives them on the device for mpm_fit and the
// server; the function also compiles for the host).  Internal.
#pragma once

#include <math.h>

#include "device_common.cuh"

namespace mpm {

// Constant starting maps from the image means (Sec. 2.7 starts from constant
// maps derived from the mean intensity of every volume; the formulas are this
// library's reading of Eqs. 1 and 3):
//  - one R2* shared by all contrasts and one TE = 0 intercept per contrast
//    from least squares on log(mean) against TE;
//  - the non-MT intercepts lie on the line S/sin a = E (S/tan a) + A (1 - E):
//    slope E (at the mean TR of those contrasts), intercept A (1 - E);
//  - MT contrasts give 1 - delta = S / (A sin a (1 - E) + S cos a E), averaged;
//  - clamps R2* >= 1e-3, E in [1e-6, 1 - 1e-6], delta in [1e-4, 0.5];
//    fallbacks R1 = 1/s and A from the first contrast when fewer than two
//    distinct non-MT flip angles exist, R2* = 20/s without multi-echo data.
__host__ __device__ inline void initial_map_values(const DevProblem& P, const double* mean, float out[4])
{
    const int C = P.C;
    double lm[MPM_MAX_IMAGES];
    for (int i = 0; i < P.I; ++i) lm[i] = log(mean[i] > 1e-30 ? mean[i] : 1e-30);
    double tbar[MPM_MAX_CONTRASTS], lbar[MPM_MAX_CONTRASTS];
    double sxy = 0.0, sxx = 0.0;
    for (int c = 0; c < C; ++c) {
        const int E = P.n_echoes[c], i0 = P.echo0[c];
        double st = 0.0, sl = 0.0;
        for (int e = 0; e < E; ++e) {
            st += P.te[i0 + e];
            sl += lm[i0 + e];
        }
        tbar[c] = st / E;
        lbar[c] = sl / E;
        for (int e = 0; e < E; ++e) {
            const double dt = P.te[i0 + e] - tbar[c];
            sxy += dt * (lm[i0 + e] - lbar[c]);
            sxx += dt * dt;
        }
    }
    double r2 = sxx > 0.0 ? -sxy / sxx : 20.0;
    if (r2 < 1e-3) r2 = 1e-3;
    double S0[MPM_MAX_CONTRASTS];
    for (int c = 0; c < C; ++c) S0[c] = exp(lbar[c] + r2 * tbar[c]);

    int first = -1, cnt = 0;
    double mx = 0, my = 0, mxx = 0, mxy = 0, trsum = 0;
    for (int c = 0; c < C; ++c) {
        if (P.mt[c]) continue;
        if (first < 0) first = c;
        const double X = S0[c] / tan((double)P.alpha[c]);
        const double Y = S0[c] / sin((double)P.alpha[c]);
        mx += X; my += Y; mxx += X * X; mxy += X * Y; trsum += P.tr[c];
        ++cnt;
    }
    if (first < 0) first = 0;
    const double varx = cnt > 0 ? mxx - mx * mx / cnt : 0.0;
    double A, r1;
    const double af = P.alpha[first];
    if (cnt >= 2 && varx > 1e-12 * mxx) {
        double E = (mxy - mx * my / cnt) / varx;
        E = fmin(fmax(E, 1e-6), 1.0 - 1e-6);
        r1 = -log(E) / (trsum / cnt);
        A = ((my - E * mx) / cnt) / (1.0 - E);
        if (!(A > 0.0)) A = S0[first] * (1.0 - cos(af) * E) / (sin(af) * (1.0 - E));
    } else {
        r1 = 1.0;
        const double E = exp(-r1 * P.tr[first]);
        A = S0[first] * (1.0 - cos(af) * E) / (sin(af) * (1.0 - E));
    }
    double dsum = 0.0;
    int nmt = 0;
    for (int c = 0; c < C; ++c) {
        if (!P.mt[c]) continue;
        const double E = exp(-r1 * P.tr[c]);
        const double ac = P.alpha[c];
        const double mfac = S0[c] / (A * sin(ac) * (1.0 - E) + S0[c] * cos(ac) * E);
        dsum += 1.0 - mfac;
        ++nmt;
    }
    double delta = nmt ? dsum / nmt : 0.01;
    if (!(delta >= 1e-4)) delta = 1e-4;
    if (delta > 0.5) delta = 0.5;
    out[0] = (float)log(A);
    out[1] = (float)log(r1);
    out[2] = (float)log(r2);
    out[3] = (float)log(delta / (1.0 - delta));
}

}  // namespace mpm
