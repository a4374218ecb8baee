/*
 * mpm_oracle.c -- FP64 CPU oracle of the model-based multi-parameter-mapping
 * fit (Balbastre et al., "Model-Based Multi-Parameter Mapping", 2021).
 *
 * TEST INFRASTRUCTURE.  This is the slow, plain, double-precision reference
 * that the CUDA library is checked against.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark load it; the CUDA library
 * never does, and the two share no code, header, table or constant.
 *
 * Every function is plain loops over voxels in the paper's order and
 * notation: the signal and its derivatives are the printed closed forms, the
 * likelihood gradient and approximate Hessian are summed image by image, the
 * prior is the explicit 6-neighbour stencil, and PCG is the textbook
 * recurrence.  No blocking, fusion or reordering.
 *
 * What pins it (tests/test_oracle_*.py):
 *   orc_signal        steady-state Bloch recursion simulated pulse by pulse;
 *                     the Ernst angle; the DESPOT1 straight line.
 *   orc_signal_jet    central finite differences of orc_signal.
 *   orc_grad_hess     likelihood computed from the planted residuals; finite
 *                     differences of the likelihood; Jacobian built by finite
 *                     differences of orc_forward; positive definiteness; the
 *                     row-sum loading majorises the true Hessian.
 *   orc_jtv, orc_membrane, orc_membrane_diag
 *                     the finite-difference matrix G materialised densely.
 *   orc_pcg/orc_solve dense Cholesky solve of H + L.
 *   orc_uncertainty   dense inverse / log-determinant; Monte-Carlo moments.
 *   orc_init          exact on a single noise-free voxel.
 *   orc_pull/orc_push exact shifts and 90-degree rotations (index
 *                     permutations); affine functions reproduced exactly by
 *                     the interpolation; <Psi u, v> = <u, Psi' v>.
 *   orc_grad_hess_proj
 *                     identity reslicing gives orc_grad_hess; finite
 *                     differences of the projected likelihood; the pushed
 *                     Hessian majorises Psi' H Psi (Psi materialised).
 *   orc_fit           exact recovery from noise-free data (no prior); the
 *                     likelihood never increases over 1000 simulated voxels
 *                     (Sec. 3.1 protocol); the objective decreases under the
 *                     JTV majorise-minimise loop with accurate inner solves;
 *                     with the prior, constant noise-free maps are recovered
 *                     from a perturbed start with F = N eps (the closed-form
 *                     optimum); the fit commutes with mirroring any axis and
 *                     with swapping x and y together with their voxel sizes.
 *   The prior-regularised fit of noisy data after a fixed iteration count has
 *   no value printed in the paper: beyond the pins above it is "parity
 *   unpinned".
 *
 * Threads.  The same source builds serial and, with -fopenmp, threaded over
 * voxels (the timing host's cores).  Every volume-wide sum is taken in fixed
 * chunks of ORC_CHUNK voxels, each chunk summed in voxel order and the chunk
 * sums added in chunk order, so both builds round identically for any thread
 * count.  Per-voxel arithmetic is the same statement in both.  The spatial
 * projection functions stay serial.
 */
#include "mpm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- helpers */

static long n_vox(const orc_problem* p) { return (long)p->nx * p->ny * p->nz; }

/* Volume-wide sums: chunks of ORC_CHUNK voxels summed in order, then the
 * chunk sums in chunk order (the same rounding with or without threads). */
#define ORC_CHUNK 4096L

static long n_chunks(long n) { return (n + ORC_CHUNK - 1) / ORC_CHUNK; }

static long chunk_end(long c, long n)
{
    long e = (c + 1) * ORC_CHUNK;
    return e < n ? e : n;
}

static double sum_chunks(const double* part, long nc)
{
    double s = 0.0;
    for (long c = 0; c < nc; ++c) s += part[c];
    return s;
}

int orc_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

static int n_images(const orc_problem* p)
{
    int i = 0;
    for (int c = 0; c < p->n_contrasts; ++c) i += p->n_echoes[c];
    return i;
}

static int n_tri(int K) { return K * (K + 1) / 2; }

/* Position of (k, j), k <= j, in the packed upper triangle. */
static int tri_index(int K, int k, int j)
{
    if (k > j) { int t = k; k = j; j = t; }
    int idx = 0;
    for (int r = 0; r < k; ++r) idx += K - r;
    return idx + (j - k);
}

/* The 6 neighbours of voxel n used by the finite-difference operator G
 * (Sec. 2.5: forward and backward differences along x, y and z).  Neighbours
 * outside the volume are dropped (Neumann boundary).  Returns the count and
 * fills the neighbour index and 1/h^2 of the axis. */
static int neighbours(const orc_problem* p, long n, long* m, double* ih2)
{
    long nx = p->nx, ny = p->ny, nz = p->nz;
    long x = n % nx, yy = (n / nx) % ny, z = n / (nx * ny);
    int c = 0;
    double hx = 1.0 / (p->vx[0] * p->vx[0]);
    double hy = 1.0 / (p->vx[1] * p->vx[1]);
    double hz = 1.0 / (p->vx[2] * p->vx[2]);
    if (x > 0)      { m[c] = n - 1;       ih2[c++] = hx; }
    if (x < nx - 1) { m[c] = n + 1;       ih2[c++] = hx; }
    if (yy > 0)     { m[c] = n - nx;      ih2[c++] = hy; }
    if (yy < ny - 1){ m[c] = n + nx;      ih2[c++] = hy; }
    if (z > 0)      { m[c] = n - nx * ny; ih2[c++] = hz; }
    if (z < nz - 1) { m[c] = n + nx * ny; ih2[c++] = hz; }
    return c;
}

/* Cholesky A = L L^T of a K x K symmetric matrix (lower triangle used).
 * Returns 0, or -1 if A is not positive definite. */
static int cholesky(int K, double A[4][4], double L[4][4])
{
    memset(L, 0, sizeof(double) * 16);
    for (int j = 0; j < K; ++j) {
        double d = A[j][j];
        for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
        if (!(d > 0.0)) return -1;
        L[j][j] = sqrt(d);
        for (int i = j + 1; i < K; ++i) {
            double v = A[i][j];
            for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
            L[i][j] = v / L[j][j];
        }
    }
    return 0;
}

static void chol_solve(int K, double L[4][4], const double* b, double* x)
{
    double t[4];
    for (int i = 0; i < K; ++i) {
        double v = b[i];
        for (int k = 0; k < i; ++k) v -= L[i][k] * t[k];
        t[i] = v / L[i][i];
    }
    for (int i = K - 1; i >= 0; --i) {
        double v = t[i];
        for (int k = i + 1; k < K; ++k) v -= L[k][i] * x[k];
        x[i] = v / L[i][i];
    }
}

/* Block n of the preconditioner  H_n + diag_k(lambda_k d_n)  (Sec. 2.6). */
static void precond_block(const orc_problem* p, const double* h, const double* d,
                          long n, double M[4][4])
{
    int K = p->n_maps;
    long N = n_vox(p);
    for (int k = 0; k < K; ++k)
        for (int j = 0; j < K; ++j)
            M[k][j] = h[(long)tri_index(K, k, j) * N + n];
    for (int k = 0; k < K; ++k) M[k][k] += p->lambda[k] * d[n];
}

/* ------------------------------------------------------- forward model */

/* Eq. 26 with the B1 footnote: alpha_n = alpha * b1p, signal scaled by b1m.
 * delta = 0 for contrasts without MT pulse (Sec. 2.4). */
double orc_signal(const double y[4], double alpha, double tr, double te,
                  int mt, double b1p, double b1m)
{
    double a = exp(y[0]);
    double r1 = exp(y[1]);
    double r2 = exp(y[2]);
    double delta = mt ? 1.0 / (1.0 + exp(-y[3])) : 0.0;
    double al = alpha * b1p;
    double E = exp(-r1 * tr);
    return b1m * a * sin(al) * (1.0 - delta) * (1.0 - E)
           / (1.0 - (1.0 - delta) * cos(al) * E) * exp(-r2 * te);
}

void orc_signal_jet(const double y[4], double alpha, double tr, double te,
                    int mt, double b1p, double b1m,
                    double* s_out, double ds[4], double d2s[16])
{
    double r1 = exp(y[1]);
    double r2 = exp(y[2]);
    double delta = mt ? 1.0 / (1.0 + exp(-y[3])) : 0.0;
    double al = alpha * b1p;
    double ca = cos(al);
    double E = exp(-r1 * tr);
    double m = 1.0 - delta;
    double D = 1.0 - m * ca * E;
    double s = orc_signal(y, alpha, tr, te, mt, b1p, b1m);

    /* Gradient, Eqs. 27-30, written as q_k s. */
    double q[4];
    q[0] = 1.0;
    q[1] = -tr * r1 * ((m * ca - 1.0) * E) / (D * (1.0 - E));
    q[2] = -te * r2;
    q[3] = mt ? delta / (m * ca * E - 1.0) : 0.0;
    for (int k = 0; k < 4; ++k) ds[k] = q[k] * s;

    /* Off-diagonal second derivatives: d2s/dk dj = s (q_k q_j + dq_j/dk).
     * q_0 and q_2 depend only on their own parameter; q_1 and q_3 both
     * depend on log R1 and logit delta through E and (1 - delta), with
     * dq_1/d(logit delta) = dq_3/d(log R1) = tr r1 E cos(alpha) delta (1-delta) / D^2. */
    for (int k = 0; k < 4; ++k)
        for (int j = 0; j < 4; ++j)
            d2s[4 * k + j] = s * q[k] * q[j];
    if (mt) {
        double cross = tr * r1 * E * ca * delta * m / (D * D);
        d2s[4 * 1 + 3] += s * cross;
        d2s[4 * 3 + 1] += s * cross;
    }
    /* Diagonal: Eqs. 31-34 as printed. */
    d2s[0] = ds[0];
    d2s[5] = (1.0 - tr * r1 * (1.0 + m * ca * E) / (1.0 - m * ca * E)) * ds[1];
    d2s[10] = (1.0 - te * r2) * ds[2];
    d2s[15] = mt ? (2.0 * m * (1.0 - ca * E) / (1.0 - m * ca * E) - 1.0) * ds[3] : 0.0;
    *s_out = s;
}

void orc_forward(const orc_problem* p, const double* y, const double* b1p,
                 const double* b1m, double* s)
{
    long N = n_vox(p);
    int K = p->n_maps;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        double yn[4] = {0, 0, 0, 0};
        for (int k = 0; k < K; ++k) yn[k] = y[(long)k * N + n];
        int i = 0;
        for (int c = 0; c < p->n_contrasts; ++c) {
            double bp = b1p ? b1p[n] : 1.0;
            double bm = b1m ? b1m[(long)c * N + n] : 1.0;
            for (int e = 0; e < p->n_echoes[c]; ++e, ++i)
                s[(long)i * N + n] = orc_signal(yn, p->alpha[c], p->tr[c], p->te[i],
                                                p->mt[c], bp, bm);
        }
    }
}

/* ------------------------------------------- likelihood, Eqs. 6, 24, 25 */

/* Contribution of the echoes of contrast c in one voxel (Eqs. 6, 24, 25):
 * adds to *nll, gn and P.  xv[e * xstride] is the observed echo e. */
static void contrast_terms(const orc_problem* p, int c, int i0, const double yn[4], double bp,
                           double bm, const double* xv, long xstride, double* nll, double gn[4],
                           double P[4][4])
{
    int K = p->n_maps;
    double is2 = 1.0 / p->sigma2[c];
    for (int e = 0; e < p->n_echoes[c]; ++e) {
        double s, ds[4], d2s[16];
        orc_signal_jet(yn, p->alpha[c], p->tr[c], p->te[i0 + e], p->mt[c], bp, bm, &s, ds, d2s);
        double r = s - xv[(long)e * xstride];
        *nll += 0.5 * r * r * is2;
        for (int k = 0; k < K; ++k) gn[k] += r * ds[k] * is2;
        for (int k = 0; k < K; ++k)
            for (int j = 0; j < K; ++j) P[k][j] += ds[k] * ds[j] * is2;
        /* Loading of Eq. 24: |r| |H_f| (.) I (precond 0), or the
         * row sums |H_f| 1 ("Proposed+", precond 1), or none (2). */
        for (int k = 0; k < K; ++k) {
            double load = 0.0;
            if (p->precond == 0) {
                load = fabs(d2s[4 * k + k]);
            } else if (p->precond == 1) {
                for (int j = 0; j < K; ++j) load += fabs(d2s[4 * k + j]);
            }
            P[k][k] += fabs(r) * load * is2;
        }
    }
}

double orc_grad_hess(const orc_problem* p, const double* x, const double* y,
                     const double* b1p, const double* b1m, double* g, double* h)
{
    long N = n_vox(p);
    int K = p->n_maps;
    long nc = n_chunks(N);
    double* part = malloc(sizeof(double) * (nc > 0 ? nc : 1));
#pragma omp parallel for schedule(static)
    for (long ch = 0; ch < nc; ++ch) {
        double nll = 0.0;
        for (long n = ch * ORC_CHUNK; n < chunk_end(ch, N); ++n) {
            double yn[4] = {0, 0, 0, 0};
            for (int k = 0; k < K; ++k) yn[k] = y[(long)k * N + n];
            double gn[4] = {0, 0, 0, 0};
            double P[4][4];
            memset(P, 0, sizeof P);
            int i = 0;
            for (int c = 0; c < p->n_contrasts; ++c) {
                double bp = b1p ? b1p[n] : 1.0;
                double bm = b1m ? b1m[(long)c * N + n] : 1.0;
                contrast_terms(p, c, i, yn, bp, bm, x + (long)i * N + n, N, &nll, gn, P);
                i += p->n_echoes[c];
            }
            for (int k = 0; k < K; ++k) g[(long)k * N + n] = gn[k];
            for (int k = 0; k < K; ++k)
                for (int j = k; j < K; ++j)
                    h[(long)tri_index(K, k, j) * N + n] = P[k][j];
        }
        part[ch] = nll;
    }
    double nll = sum_chunks(part, nc);
    free(part);
    return nll;
}

/* ------------------------------------------- spatial projection, Sec. 2.4 */

/* Reconstruction-space coordinate r = A (i, j, k, 1) of acquisition voxel
 * (i, j, k); returns 1 when r lies inside the reconstruction grid,
 * 0 <= r_d <= n_d - 1 on every axis (the voxel then has data that the model
 * explains), else 0. */
static int reslice_coord(const orc_problem* p, const double A[12], long i, long j, long k,
                         double r[3])
{
    for (int d = 0; d < 3; ++d)
        r[d] = A[4 * d + 0] * (double)i + A[4 * d + 1] * (double)j + A[4 * d + 2] * (double)k +
               A[4 * d + 3];
    return r[0] >= 0.0 && r[0] <= p->nx - 1 && r[1] >= 0.0 && r[1] <= p->ny - 1 &&
           r[2] >= 0.0 && r[2] <= p->nz - 1;
}

/* The trilinear interpolation weights of r: up to 8 reconstruction voxels
 * (corners of the cell holding r) and their weights; corners past the last
 * voxel (which have weight 0) are left out.  Returns the count. */
static int trilinear(const orc_problem* p, const double r[3], long idx[8], double wt[8])
{
    long b[3];
    double f[3];
    long n[3] = {p->nx, p->ny, p->nz};
    for (int d = 0; d < 3; ++d) {
        b[d] = (long)floor(r[d]);
        f[d] = r[d] - (double)b[d];
    }
    int cnt = 0;
    for (int cz = 0; cz < 2; ++cz)
        for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx) {
                long ix = b[0] + cx, iy = b[1] + cy, iz = b[2] + cz;
                if (ix > n[0] - 1 || iy > n[1] - 1 || iz > n[2] - 1) continue;
                idx[cnt] = ix + n[0] * (iy + n[1] * iz);
                wt[cnt] = (cx ? f[0] : 1.0 - f[0]) * (cy ? f[1] : 1.0 - f[1]) *
                          (cz ? f[2] : 1.0 - f[2]);
                ++cnt;
            }
    return cnt;
}

void orc_pull(const orc_problem* p, const int dims[3], const double A[12], int channels,
              const double* u, double* out, unsigned char* inside)
{
    long N = n_vox(p);
    long M = (long)dims[0] * dims[1] * dims[2];
    long m = 0;
    for (long k = 0; k < dims[2]; ++k)
        for (long j = 0; j < dims[1]; ++j)
            for (long i = 0; i < dims[0]; ++i, ++m) {
                double r[3];
                int in = reslice_coord(p, A, i, j, k, r);
                if (inside) inside[m] = (unsigned char)in;
                for (int ch = 0; ch < channels; ++ch) out[(long)ch * M + m] = 0.0;
                if (!in) continue;
                long idx[8];
                double wt[8];
                int cnt = trilinear(p, r, idx, wt);
                for (int ch = 0; ch < channels; ++ch)
                    for (int q = 0; q < cnt; ++q)
                        out[(long)ch * M + m] += wt[q] * u[(long)ch * N + idx[q]];
            }
}

void orc_push(const orc_problem* p, const int dims[3], const double A[12], int channels,
              const double* u, double* out)
{
    long N = n_vox(p);
    long M = (long)dims[0] * dims[1] * dims[2];
    long m = 0;
    for (long k = 0; k < dims[2]; ++k)
        for (long j = 0; j < dims[1]; ++j)
            for (long i = 0; i < dims[0]; ++i, ++m) {
                double r[3];
                if (!reslice_coord(p, A, i, j, k, r)) continue;
                long idx[8];
                double wt[8];
                int cnt = trilinear(p, r, idx, wt);
                for (int ch = 0; ch < channels; ++ch)
                    for (int q = 0; q < cnt; ++q)
                        out[(long)ch * N + idx[q]] += wt[q] * u[(long)ch * M + m];
            }
}

/* Sec. 2.4: l_psi(y) = sum_c l_c(Psi_c y).  Per contrast the maps are pulled
 * to its acquisition grid, the gradient and loaded Hessian of the contrast's
 * echoes are formed there voxel by voxel (as in orc_grad_hess, acquisition
 * voxels outside the reconstruction grid contribute nothing), and both are
 * pushed back: g = sum_c Psi_c' g_c, h = sum_c Psi_c' h_c.  The latter is the
 * block-diagonal majoriser of Psi_c' H_c Psi_c: with non-negative weights that
 * sum to one per acquisition voxel, Jensen's inequality on each voxel's
 * quadratic form bounds Psi' H Psi by diag(Psi' H) (the result the paper takes
 * from Ashburner et al. 2018). */
double orc_grad_hess_proj(const orc_problem* p, const orc_projection* q,
                          const double* const* x, const double* const* b1p,
                          const double* const* b1m, const double* y, double* g, double* h)
{
    long N = n_vox(p);
    int K = p->n_maps, T = n_tri(K);
    for (long i = 0; i < (long)K * N; ++i) g[i] = 0.0;
    for (long i = 0; i < (long)T * N; ++i) h[i] = 0.0;
    double nll = 0.0;
    int i0 = 0;
    for (int c = 0; c < p->n_contrasts; ++c) {
        const int* dims = q->dims[c];
        long M = (long)dims[0] * dims[1] * dims[2];
        double* yc = malloc(sizeof(double) * K * M);
        unsigned char* in = malloc(M);
        double* gc = calloc((size_t)K * M, sizeof(double));
        double* hc = calloc((size_t)T * M, sizeof(double));
        orc_pull(p, dims, q->affine[c], K, y, yc, in);
        for (long m = 0; m < M; ++m) {
            if (!in[m]) continue;
            double yn[4] = {0, 0, 0, 0};
            for (int k = 0; k < K; ++k) yn[k] = yc[(long)k * M + m];
            double gn[4] = {0, 0, 0, 0};
            double P[4][4];
            memset(P, 0, sizeof P);
            double bp = b1p && b1p[c] ? b1p[c][m] : 1.0;
            double bm = b1m && b1m[c] ? b1m[c][m] : 1.0;
            contrast_terms(p, c, i0, yn, bp, bm, x[c] + m, M, &nll, gn, P);
            for (int k = 0; k < K; ++k) gc[(long)k * M + m] = gn[k];
            for (int k = 0; k < K; ++k)
                for (int j = k; j < K; ++j) hc[(long)tri_index(K, k, j) * M + m] = P[k][j];
        }
        orc_push(p, dims, q->affine[c], K, gc, g);
        orc_push(p, dims, q->affine[c], T, hc, h);
        free(yc); free(in); free(gc); free(hc);
        i0 += p->n_echoes[c];
    }
    return nll;
}

/* ------------------------------------------------------ prior, Sec. 2.5 */

/* u_n = sum_k lambda_k |G_n y_k|^2 (Eq. 38); w_n = (u_n + eps^2)^-1/2
 * (Eq. 40 with the eps smoothing); returns sum_n sqrt(u_n + eps^2). */
double orc_jtv(const orc_problem* p, const double* y, double* w)
{
    long N = n_vox(p);
    int K = p->n_maps;
    long nc = n_chunks(N);
    double* part = malloc(sizeof(double) * (nc > 0 ? nc : 1));
#pragma omp parallel for schedule(static)
    for (long ch = 0; ch < nc; ++ch) {
        double jtv = 0.0;
        for (long n = ch * ORC_CHUNK; n < chunk_end(ch, N); ++n) {
            long m[6];
            double ih2[6];
            int cnt = neighbours(p, n, m, ih2);
            double u = 0.0;
            for (int k = 0; k < K; ++k) {
                double acc = 0.0;
                for (int j = 0; j < cnt; ++j) {
                    double dlt = y[(long)k * N + m[j]] - y[(long)k * N + n];
                    acc += dlt * dlt * ih2[j];
                }
                u += p->lambda[k] * acc;
            }
            double v = u + p->eps * p->eps;
            if (w) w[n] = 1.0 / sqrt(v);
            jtv += sqrt(v);
        }
        part[ch] = jtv;
    }
    double jtv = sum_chunks(part, nc);
    free(part);
    return jtv;
}

/* (G'WG v)_n = sum_{m in N(n)} (w_n + w_m)(v_n - v_m) / h^2, times lambda_k. */
void orc_membrane(const orc_problem* p, const double* w, const double* v, double* out)
{
    long N = n_vox(p);
    int K = p->n_maps;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        long m[6];
        double ih2[6];
        int cnt = neighbours(p, n, m, ih2);
        for (int k = 0; k < K; ++k) {
            double acc = 0.0;
            for (int j = 0; j < cnt; ++j)
                acc += (w[n] + w[m[j]]) * (v[(long)k * N + n] - v[(long)k * N + m[j]]) * ih2[j];
            out[(long)k * N + n] = p->lambda[k] * acc;
        }
    }
}

void orc_membrane_diag(const orc_problem* p, const double* w, double* d)
{
    long N = n_vox(p);
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        long m[6];
        double ih2[6];
        int cnt = neighbours(p, n, m, ih2);
        double acc = 0.0;
        for (int j = 0; j < cnt; ++j) acc += (w[n] + w[m[j]]) * ih2[j];
        d[n] = acc;
    }
}

/* -------------------------------------------- Newton system, Sec. 2.6 */

static void apply_system(const orc_problem* p, const double* h, const double* w,
                         const double* v, double* out)
{
    long N = n_vox(p);
    int K = p->n_maps;
    orc_membrane(p, w, v, out);
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n)
        for (int k = 0; k < K; ++k) {
            double acc = 0.0;
            for (int j = 0; j < K; ++j)
                acc += h[(long)tri_index(K, k, j) * N + n] * v[(long)j * N + n];
            out[(long)k * N + n] += acc;
        }
}

static int apply_precond_inverse(const orc_problem* p, const double* h, const double* d,
                                 const double* r, double* z)
{
    long N = n_vox(p);
    int K = p->n_maps;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(|:bad)
    for (long n = 0; n < N; ++n) {
        double M[4][4], L[4][4], b[4], x[4];
        precond_block(p, h, d, n, M);
        if (cholesky(K, M, L)) { bad = 1; continue; }
        for (int k = 0; k < K; ++k) b[k] = r[(long)k * N + n];
        chol_solve(K, L, b, x);
        for (int k = 0; k < K; ++k) z[(long)k * N + n] = x[k];
    }
    return bad ? -1 : 0;
}

static double dot(long n, const double* a, const double* b)
{
    long nc = n_chunks(n);
    double* part = malloc(sizeof(double) * (nc > 0 ? nc : 1));
#pragma omp parallel for schedule(static)
    for (long c = 0; c < nc; ++c) {
        double s = 0.0;
        for (long i = c * ORC_CHUNK; i < chunk_end(c, n); ++i) s += a[i] * b[i];
        part[c] = s;
    }
    double s = sum_chunks(part, nc);
    free(part);
    return s;
}

int orc_pcg(const orc_problem* p, const double* h, const double* w, const double* b,
            double* x, int max_iters, double tol, double* resid)
{
    long N = n_vox(p);
    long L = (long)p->n_maps * N;
    double* r = malloc(sizeof(double) * L);
    double* z = malloc(sizeof(double) * L);
    double* pv = malloc(sizeof(double) * L);
    double* q = malloc(sizeof(double) * L);
    double* d = malloc(sizeof(double) * N);
    int it = 0;

    orc_membrane_diag(p, w, d);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < L; ++i) { x[i] = 0.0; r[i] = b[i]; }
    if (apply_precond_inverse(p, h, d, r, z)) { it = -1; goto done; }
    memcpy(pv, z, sizeof(double) * L);
    double rz = dot(L, r, z);
    double rr0 = dot(L, r, r);
    if (resid) resid[0] = sqrt(rr0);
    for (it = 0; it < max_iters; ++it) {
        if (!(rz > 0.0)) break;                             /* r = 0: solved */
        if (tol > 0.0 && sqrt(dot(L, r, r)) <= tol * sqrt(rr0)) break;
        apply_system(p, h, w, pv, q);
        double pq = dot(L, pv, q);
        if (!(pq > 0.0)) break;
        double alpha = rz / pq;
#pragma omp parallel for schedule(static)
        for (long i = 0; i < L; ++i) { x[i] += alpha * pv[i]; r[i] -= alpha * q[i]; }
        if (apply_precond_inverse(p, h, d, r, z)) { it = -1; goto done; }
        double rz_new = dot(L, r, z);
        double beta = rz_new / rz;
        rz = rz_new;
#pragma omp parallel for schedule(static)
        for (long i = 0; i < L; ++i) pv[i] = z[i] + beta * pv[i];
        if (resid) resid[it + 1] = sqrt(dot(L, r, r));
    }
done:
    free(r); free(z); free(pv); free(q); free(d);
    return it;
}

int orc_solve(const orc_problem* p, const double* h, const double* w, const double* g,
              const double* y, double* delta, int max_iters, double tol, double* resid)
{
    long L = (long)p->n_maps * n_vox(p);
    double* b = malloc(sizeof(double) * L);
    orc_membrane(p, w, y, b);                       /* b = g + L y (Eq. 42) */
#pragma omp parallel for schedule(static)
    for (long i = 0; i < L; ++i) b[i] += g[i];
    int it = orc_pcg(p, h, w, b, delta, max_iters, tol, resid);
    free(b);
    return it;
}

/* ---------------------------------- multigrid preconditioner (an option) */

/* Not part of the paper's solver (Sec. 2.6 uses the block preconditioner of
 * orc_pcg).  An aggregation multigrid V-cycle for A = H + L, used as the
 * preconditioner of the same conjugate-gradient recurrence:
 *   - levels: level l + 1 merges 2 x 2 x 2 voxels of level l (ceil(n / 2) per
 *     axis); a level of at most ORC_MG_MIN_VOXELS voxels is the coarsest;
 *   - prolongation P: a coarse voxel's value copied to its children;
 *     restriction P' (sum over the children);
 *   - coarse operators by the Galerkin product A_c = P' A P, which keeps the
 *     form of A: H_c = sum of the children's blocks, and the coefficient of a
 *     coarse edge = sum of the coefficients of the fine edges crossing it
 *     (edges inside a coarse voxel drop out); level 0 has the coefficients
 *     (w_n + w_m) / h^2 of L;
 *   - smoother: damped block-Jacobi, x += omega D^-1 (r - A x), D the 4 x 4
 *     voxel blocks of A (on level 0 exactly the block preconditioner of Eq. 42);
 *   - V-cycle from x = 0: nu sweeps, coarse correction with the restricted
 *     residual, nu sweeps; coarse_sweeps sweeps on the coarsest level.  Equal
 *     sweeps before and after make the cycle a symmetric operator. */

#define ORC_MG_MIN_VOXELS 512L
#define ORC_MG_MAX_LEVELS 16

typedef struct {
    int n[3];
    long N;
    double* h;      /* [T][N] */
    double* kap;    /* [3][N]: edge from voxel v to v + e_a, 0 where it leaves the level */
    long* parent;   /* [N]: voxel of level l + 1 holding v (NULL on the coarsest) */
} orc_level;

int orc_mg_levels(const orc_problem* p, const orc_mg* mg, int dims[][3])
{
    int n[3] = {p->nx, p->ny, p->nz};
    int L = 0;
    int max_l = mg->levels < ORC_MG_MAX_LEVELS ? mg->levels : ORC_MG_MAX_LEVELS;
    for (;;) {
        if (dims) { dims[L][0] = n[0]; dims[L][1] = n[1]; dims[L][2] = n[2]; }
        ++L;
        if (L >= max_l || (long)n[0] * n[1] * n[2] <= ORC_MG_MIN_VOXELS) break;
        for (int a = 0; a < 3; ++a) n[a] = (n[a] + 1) / 2;
    }
    return L;
}

static long lvox(const int n[3], int x, int y, int z) { return x + (long)n[0] * (y + (long)n[1] * z); }

/* Level 0 from H and w; every coarser level by the Galerkin product. */
static int mg_build(const orc_problem* p, const double* h, const double* w, const orc_mg* mg,
                    orc_level* lv)
{
    int dims[ORC_MG_MAX_LEVELS][3];
    int L = orc_mg_levels(p, mg, dims);
    int T = n_tri(p->n_maps);
    double ih2[3] = {1.0 / (p->vx[0] * p->vx[0]), 1.0 / (p->vx[1] * p->vx[1]),
                     1.0 / (p->vx[2] * p->vx[2])};
    for (int l = 0; l < L; ++l) {
        for (int a = 0; a < 3; ++a) lv[l].n[a] = dims[l][a];
        lv[l].N = (long)dims[l][0] * dims[l][1] * dims[l][2];
        lv[l].h = calloc((size_t)T * lv[l].N, sizeof(double));
        lv[l].kap = calloc((size_t)3 * lv[l].N, sizeof(double));
        lv[l].parent = l + 1 < L ? malloc(sizeof(long) * lv[l].N) : NULL;
    }
    /* level 0 */
    long N = lv[0].N;
    memcpy(lv[0].h, h, sizeof(double) * T * N);
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long v = lvox(lv[0].n, x, y, z);
                if (x + 1 < p->nx) lv[0].kap[0 * N + v] = (w[v] + w[v + 1]) * ih2[0];
                if (y + 1 < p->ny) lv[0].kap[1 * N + v] = (w[v] + w[v + p->nx]) * ih2[1];
                if (z + 1 < p->nz) lv[0].kap[2 * N + v] = (w[v] + w[v + (long)p->nx * p->ny]) * ih2[2];
            }
    /* coarser levels */
    for (int l = 0; l + 1 < L; ++l) {
        orc_level* f = &lv[l];
        orc_level* c = &lv[l + 1];
        for (int z = 0; z < f->n[2]; ++z)
            for (int y = 0; y < f->n[1]; ++y)
                for (int x = 0; x < f->n[0]; ++x) {
                    long v = lvox(f->n, x, y, z);
                    long pv = lvox(c->n, x / 2, y / 2, z / 2);
                    f->parent[v] = pv;
                    for (int t = 0; t < T; ++t) c->h[(long)t * c->N + pv] += f->h[(long)t * f->N + v];
                    int q[3] = {x, y, z};
                    for (int a = 0; a < 3; ++a) {
                        /* the fine edge v -> v + e_a crosses into the next coarse voxel */
                        if (q[a] + 1 < f->n[a] && (q[a] + 1) / 2 != q[a] / 2)
                            c->kap[(long)a * c->N + pv] += f->kap[(long)a * f->N + v];
                    }
                }
    }
    return L;
}

static void mg_free(orc_level* lv, int L)
{
    for (int l = 0; l < L; ++l) { free(lv[l].h); free(lv[l].kap); free(lv[l].parent); }
}

/* out = A_l x on one level. */
static void mg_apply(const orc_problem* p, const orc_level* lv, const double* x, double* out)
{
    int K = p->n_maps;
    long N = lv->N;
    long st[3] = {1, lv->n[0], (long)lv->n[0] * lv->n[1]};
#pragma omp parallel for schedule(static)
    for (long v = 0; v < N; ++v) {
        long q[3] = {v % lv->n[0], (v / lv->n[0]) % lv->n[1], v / ((long)lv->n[0] * lv->n[1])};
        for (int k = 0; k < K; ++k) {
            double acc = 0.0;
            for (int j = 0; j < K; ++j) acc += lv->h[(long)tri_index(K, k, j) * N + v] * x[(long)j * N + v];
            double lap = 0.0;
            for (int a = 0; a < 3; ++a) {
                if (q[a] + 1 < lv->n[a])
                    lap += lv->kap[(long)a * N + v] * (x[(long)k * N + v] - x[(long)k * N + v + st[a]]);
                if (q[a] > 0)
                    lap += lv->kap[(long)a * N + v - st[a]] * (x[(long)k * N + v] - x[(long)k * N + v - st[a]]);
            }
            out[(long)k * N + v] = acc + p->lambda[k] * lap;
        }
    }
}

/* x += omega D^-1 (r - A x), D the voxel blocks of A_l. */
static int mg_sweep(const orc_problem* p, const orc_level* lv, double omega, const double* r,
                    double* x, double* t)
{
    int K = p->n_maps;
    long N = lv->N;
    long st[3] = {1, lv->n[0], (long)lv->n[0] * lv->n[1]};
    mg_apply(p, lv, x, t);
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(|:bad)
    for (long v = 0; v < N; ++v) {
        long q[3] = {v % lv->n[0], (v / lv->n[0]) % lv->n[1], v / ((long)lv->n[0] * lv->n[1])};
        double d = 0.0;
        for (int a = 0; a < 3; ++a) {
            if (q[a] + 1 < lv->n[a]) d += lv->kap[(long)a * N + v];
            if (q[a] > 0) d += lv->kap[(long)a * N + v - st[a]];
        }
        double M[4][4], Lc[4][4], b[4], e[4];
        for (int k = 0; k < K; ++k)
            for (int j = 0; j < K; ++j) M[k][j] = lv->h[(long)tri_index(K, k, j) * N + v];
        for (int k = 0; k < K; ++k) M[k][k] += p->lambda[k] * d;
        if (cholesky(K, M, Lc)) { bad = 1; continue; }
        for (int k = 0; k < K; ++k) b[k] = r[(long)k * N + v] - t[(long)k * N + v];
        chol_solve(K, Lc, b, e);
        for (int k = 0; k < K; ++k) x[(long)k * N + v] += omega * e[k];
    }
    return bad ? -1 : 0;
}

/* x = V-cycle applied to r on level l (x starts at zero). */
static int mg_cycle(const orc_problem* p, orc_level* lv, int l, int L, const orc_mg* mg,
                    const double* r, double* x)
{
    int K = p->n_maps;
    long N = lv[l].N;
    double* t = malloc(sizeof(double) * K * N);
    int st = 0;
    for (long i = 0; i < (long)K * N; ++i) x[i] = 0.0;
    if (l == L - 1) {
        for (int s = 0; s < mg->coarse_sweeps && !st; ++s) st = mg_sweep(p, &lv[l], mg->omega, r, x, t);
        free(t);
        return st;
    }
    for (int s = 0; s < mg->nu && !st; ++s) st = mg_sweep(p, &lv[l], mg->omega, r, x, t);
    long Nc = lv[l + 1].N;
    double* rc = calloc((size_t)K * Nc, sizeof(double));
    double* ec = malloc(sizeof(double) * K * Nc);
    mg_apply(p, &lv[l], x, t);                          /* restricted residual P'(r - A x) */
    for (long v = 0; v < N; ++v)
        for (int k = 0; k < K; ++k)
            rc[(long)k * Nc + lv[l].parent[v]] += r[(long)k * N + v] - t[(long)k * N + v];
    if (!st) st = mg_cycle(p, lv, l + 1, L, mg, rc, ec);
    for (long v = 0; v < N; ++v)                       /* x += P e_c */
        for (int k = 0; k < K; ++k) x[(long)k * N + v] += ec[(long)k * Nc + lv[l].parent[v]];
    for (int s = 0; s < mg->nu && !st; ++s) st = mg_sweep(p, &lv[l], mg->omega, r, x, t);
    free(rc); free(ec); free(t);
    return st;
}

void orc_mg_vcycle(const orc_problem* p, const double* h, const double* w, const orc_mg* mg,
                   const double* r, double* z)
{
    orc_level lv[ORC_MG_MAX_LEVELS];
    int L = mg_build(p, h, w, mg, lv);
    mg_cycle(p, lv, 0, L, mg, r, z);
    mg_free(lv, L);
}

double orc_mg_energy(const orc_problem* p, const double* h, const double* w, const orc_mg* mg,
                     int level, const double* e)
{
    orc_level lv[ORC_MG_MAX_LEVELS];
    int L = mg_build(p, h, w, mg, lv);
    double en = 0.0;
    if (level >= 0 && level < L) {
        long n = (long)p->n_maps * lv[level].N;
        double* t = malloc(sizeof(double) * n);
        mg_apply(p, &lv[level], e, t);
        for (long i = 0; i < n; ++i) en += e[i] * t[i];
        free(t);
    }
    mg_free(lv, L);
    return en;
}

/* The conjugate-gradient recurrence of orc_pcg with z = V-cycle(r). */
int orc_mg_pcg(const orc_problem* p, const double* h, const double* w, const double* b,
               double* x, int max_iters, double tol, const orc_mg* mg, double* resid)
{
    long N = n_vox(p);
    long L = (long)p->n_maps * N;
    double* r = malloc(sizeof(double) * L);
    double* z = malloc(sizeof(double) * L);
    double* pv = malloc(sizeof(double) * L);
    double* q = malloc(sizeof(double) * L);
    orc_level lv[ORC_MG_MAX_LEVELS];
    int nl = mg_build(p, h, w, mg, lv);
    int it = 0;

    for (long i = 0; i < L; ++i) { x[i] = 0.0; r[i] = b[i]; }
    if (mg_cycle(p, lv, 0, nl, mg, r, z)) { it = -1; goto done; }
    memcpy(pv, z, sizeof(double) * L);
    double rz = dot(L, r, z);
    double rr0 = dot(L, r, r);
    if (resid) resid[0] = sqrt(rr0);
    for (it = 0; it < max_iters; ++it) {
        if (!(rz > 0.0)) break;
        if (tol > 0.0 && sqrt(dot(L, r, r)) <= tol * sqrt(rr0)) break;
        apply_system(p, h, w, pv, q);
        double pq = dot(L, pv, q);
        if (!(pq > 0.0)) break;
        double alpha = rz / pq;
        for (long i = 0; i < L; ++i) { x[i] += alpha * pv[i]; r[i] -= alpha * q[i]; }
        if (mg_cycle(p, lv, 0, nl, mg, r, z)) { it = -1; goto done; }
        double rz_new = dot(L, r, z);
        double beta = rz_new / rz;
        rz = rz_new;
        for (long i = 0; i < L; ++i) pv[i] = z[i] + beta * pv[i];
        if (resid) resid[it + 1] = sqrt(dot(L, r, r));
    }
done:
    mg_free(lv, nl);
    free(r); free(z); free(pv); free(q);
    return it;
}

int orc_mg_solve(const orc_problem* p, const double* h, const double* w, const double* g,
                 const double* y, double* delta, int max_iters, double tol, const orc_mg* mg,
                 double* resid)
{
    long L = (long)p->n_maps * n_vox(p);
    double* b = malloc(sizeof(double) * L);
    orc_membrane(p, w, y, b);                       /* b = g + L y (Eq. 42) */
    for (long i = 0; i < L; ++i) b[i] += g[i];
    int it = orc_mg_pcg(p, h, w, b, delta, max_iters, tol, mg, resid);
    free(b);
    return it;
}

/* ------------------------------------------------ uncertainty, Sec. 3.6 */

int orc_uncertainty(const orc_problem* p, const double* h, const double* w,
                    const double* y, double* var, double* logdet, double* moments)
{
    long N = n_vox(p);
    int K = p->n_maps;
    double* d = malloc(sizeof(double) * N);
    int bad = 0;
    orc_membrane_diag(p, w, d);
#pragma omp parallel for schedule(static) reduction(|:bad)
    for (long n = 0; n < N; ++n) {
        double M[4][4], L[4][4];
        precond_block(p, h, d, n, M);
        if (cholesky(K, M, L)) { bad = 1; continue; }
        for (int k = 0; k < K; ++k) {
            double e[4] = {0, 0, 0, 0}, col[4];
            e[k] = 1.0;
            chol_solve(K, L, e, col);
            var[(long)k * N + n] = col[k];
        }
        if (logdet) {
            double ld = 0.0;
            for (int k = 0; k < K; ++k) ld += log(L[k][k]);
            logdet[n] = -2.0 * ld;                  /* log det of M^-1 */
        }
        if (moments && y) {
            /* Eqs. 44-47: log-normal moments of r1 = exp(log R1) and t1 = 1/r1. */
            double s2 = var[1 * N + n];
            double lr1 = y[1 * N + n];
            moments[0 * N + n] = sqrt(exp(s2)) * exp(lr1);
            moments[1 * N + n] = (exp(s2) - 1.0) * exp(s2) * exp(lr1) * exp(lr1);
            moments[2 * N + n] = sqrt(exp(s2)) * exp(-lr1);
            moments[3 * N + n] = (exp(s2) - 1.0) * exp(s2) * exp(-lr1) * exp(-lr1);
        }
    }
    free(d);
    return bad ? -1 : 0;
}

/* ---------------------------------------------------- initial maps */

/* Sec. 2.7 starts from constant maps computed from the mean intensity of each
 * volume.  The paper does not give the formulas; this reading inverts its own
 * signal equations on the means, ignoring B1:
 *   1. mu_i = mean of image i over all voxels;
 *   2. one R2* shared by all contrasts and one intercept S_c per contrast from
 *      the least-squares line  log mu_ce = log S_c - R2* TE_ce;
 *   3. without MT (Eq. 1) S / sin(a) = E S / tan(a) + A (1 - E), a straight line
 *      in the non-MT contrasts: its slope is E (at their mean TR) and its
 *      intercept A (1 - E);
 *   4. with MT (Eq. 3) solved for 1 - delta:
 *         1 - delta = S / (A sin(a) (1 - E) + S cos(a) E), averaged over MT contrasts;
 *   5. clamps: R2* >= 1e-3, E in [1e-6, 1 - 1e-6], delta in [1e-4, 0.5].
 * Fallbacks: fewer than two distinct non-MT flip angles -> R1 = 1/s and A from
 * the first contrast; no multi-echo contrast -> R2* = 20/s. */
static void init_from_log_means(const orc_problem* p, const double* lmu, long N, double* y);

void orc_init(const orc_problem* p, const double* x, double* y)
{
    long N = n_vox(p);
    int I = n_images(p);
    double lmu[ORC_MAX_IMAGES];
    long nc = n_chunks(N);
    double* part = malloc(sizeof(double) * (nc > 0 ? nc : 1));
    for (int i = 0; i < I; ++i) {
#pragma omp parallel for schedule(static)
        for (long c = 0; c < nc; ++c) {
            double s = 0.0;
            for (long n = c * ORC_CHUNK; n < chunk_end(c, N); ++n) s += x[(long)i * N + n];
            part[c] = s;
        }
        double mu = sum_chunks(part, nc) / (double)N;
        lmu[i] = log(mu > 1e-30 ? mu : 1e-30);
    }
    free(part);
    init_from_log_means(p, lmu, N, y);
}

/* The same rule with each image's mean taken over its own acquisition grid. */
void orc_init_proj(const orc_problem* p, const orc_projection* q, const double* const* x,
                   double* y)
{
    double lmu[ORC_MAX_IMAGES];
    int i = 0;
    for (int c = 0; c < p->n_contrasts; ++c) {
        long M = (long)q->dims[c][0] * q->dims[c][1] * q->dims[c][2];
        for (int e = 0; e < p->n_echoes[c]; ++e, ++i) {
            double s = 0.0;
            for (long m = 0; m < M; ++m) s += x[c][(long)e * M + m];
            double mu = s / (double)M;
            lmu[i] = log(mu > 1e-30 ? mu : 1e-30);
        }
    }
    init_from_log_means(p, lmu, n_vox(p), y);
}

static void init_from_log_means(const orc_problem* p, const double* lmu, long N, double* y)
{
    int C = p->n_contrasts, K = p->n_maps;
    /* 2. shared slope, per-contrast intercepts */
    double te_mean[ORC_MAX_CONTRASTS], l_mean[ORC_MAX_CONTRASTS];
    double num = 0.0, den = 0.0;
    int i0 = 0;
    for (int c = 0; c < C; ++c) {
        int E = p->n_echoes[c];
        double st = 0.0, sl = 0.0;
        for (int e = 0; e < E; ++e) { st += p->te[i0 + e]; sl += lmu[i0 + e]; }
        te_mean[c] = st / E;
        l_mean[c] = sl / E;
        for (int e = 0; e < E; ++e) {
            num += (p->te[i0 + e] - te_mean[c]) * (lmu[i0 + e] - l_mean[c]);
            den += (p->te[i0 + e] - te_mean[c]) * (p->te[i0 + e] - te_mean[c]);
        }
        i0 += E;
    }
    double R2 = den > 0.0 ? -num / den : 20.0;
    if (R2 < 1e-3) R2 = 1e-3;
    double S[ORC_MAX_CONTRASTS];
    for (int c = 0; c < C; ++c) S[c] = exp(l_mean[c] + R2 * te_mean[c]);

    /* 3. DESPOT1 line over the non-MT contrasts */
    double sx = 0, sy = 0, sxx = 0, sxy = 0, trs = 0;
    int nn = 0, first = -1;
    for (int c = 0; c < C; ++c) {
        if (p->mt[c]) continue;
        if (first < 0) first = c;
        double X = S[c] / tan(p->alpha[c]);
        double Y = S[c] / sin(p->alpha[c]);
        sx += X; sy += Y; sxx += X * X; sxy += X * Y; trs += p->tr[c];
        ++nn;
    }
    if (first < 0) first = 0;
    double A, R1;
    double vx_ = nn > 0 ? sxx - sx * sx / nn : 0.0;
    if (nn >= 2 && vx_ > 1e-12 * sxx) {
        double tr_ref = trs / nn;
        double Ee = (sxy - sx * sy / nn) / vx_;
        if (Ee < 1e-6) Ee = 1e-6;
        if (Ee > 1.0 - 1e-6) Ee = 1.0 - 1e-6;
        double icpt = (sy - Ee * sx) / nn;
        R1 = -log(Ee) / tr_ref;
        A = icpt / (1.0 - Ee);
        if (!(A > 0.0)) A = S[first] * (1.0 - cos(p->alpha[first]) * Ee)
                            / (sin(p->alpha[first]) * (1.0 - Ee));
    } else {
        R1 = 1.0;
        double Ee = exp(-R1 * p->tr[first]);
        A = S[first] * (1.0 - cos(p->alpha[first]) * Ee) / (sin(p->alpha[first]) * (1.0 - Ee));
    }
    /* 4. MT saturation */
    double dsum = 0.0;
    int nmt = 0;
    for (int c = 0; c < C; ++c) {
        if (!p->mt[c]) continue;
        double Ec = exp(-R1 * p->tr[c]);
        double mfac = S[c] / (A * sin(p->alpha[c]) * (1.0 - Ec) + S[c] * cos(p->alpha[c]) * Ec);
        dsum += 1.0 - mfac;
        ++nmt;
    }
    double delta = nmt ? dsum / nmt : 0.01;
    if (!(delta >= 1e-4)) delta = 1e-4;
    if (delta > 0.5) delta = 0.5;

    double c0 = log(A), c1 = log(R1), c2 = log(R2), c3 = log(delta / (1.0 - delta));
    for (long n = 0; n < N; ++n) {
        y[0 * N + n] = c0;
        y[1 * N + n] = c1;
        y[2 * N + n] = c2;
        if (K == 4) y[3 * N + n] = c3;
    }
}

/* ----------------------------------------------------------- the fit */

/* Sec. 2.6-2.7: alternate the JTV weights (Eq. 40) and Newton updates
 * y <- y - (H + L)^-1 (g + L y) (Eq. 42) with the approximate Hessian of
 * Eq. 24, solved by PCG.  The objective is F = NLL (Eq. 25) + JTV_eps. */
static int fit_loop(const orc_problem* p, const orc_projection* q, const orc_opts* o,
                    const double* x, const double* b1p, const double* b1m,
                    const double* const* xs, const double* const* b1ps, const double* const* b1ms,
                    double* y, double* F, double* nll_out, double* jtv_out, double* cg_rel)
{
    long N = n_vox(p);
    int K = p->n_maps;
    long L = (long)K * N;
    double* w = malloc(sizeof(double) * N);
    double* g = malloc(sizeof(double) * L);
    double* h = malloc(sizeof(double) * (long)n_tri(K) * N);
    double* delta = malloc(sizeof(double) * L);
    double* resid = malloc(sizeof(double) * (o->cg_iters + 1));
    int npi = o->newton_per_irls > 0 ? o->newton_per_irls : 1;
    double F_prev = 0.0;
    int it;

    if (o->init) {
        if (q) orc_init_proj(p, q, xs, y);
        else orc_init(p, x, y);
    }
    for (it = 0;; ++it) {
        double jtv = orc_jtv(p, y, (it % npi == 0) ? w : NULL);
        double nll = q ? orc_grad_hess_proj(p, q, xs, b1ps, b1ms, y, g, h)
                       : orc_grad_hess(p, x, y, b1p, b1m, g, h);
        double Fi = nll + jtv;
        if (F) F[it] = Fi;
        if (nll_out) nll_out[it] = nll;
        if (jtv_out) jtv_out[it] = jtv;
        if (it >= o->gn_iters) break;
        if (it > 0 && o->tol_gn > 0.0 && fabs(F_prev - Fi) < o->tol_gn * fabs(F_prev)) break;
        F_prev = Fi;
        int cg;
        if (o->mg_levels > 0) {
            orc_mg mg = {o->mg_levels, o->mg_nu, o->mg_omega, o->mg_coarse_sweeps};
            cg = orc_mg_solve(p, h, w, g, y, delta, o->cg_iters, o->tol_cg, &mg, resid);
        } else {
            cg = orc_solve(p, h, w, g, y, delta, o->cg_iters, o->tol_cg, resid);
        }
        if (cg < 0) { it = -1; break; }
        if (cg_rel) cg_rel[it] = resid[0] > 0.0 ? resid[cg] / resid[0] : 0.0;
#pragma omp parallel for schedule(static)
        for (long i = 0; i < L; ++i) y[i] -= delta[i];
    }
    free(w); free(g); free(h); free(delta); free(resid);
    return it;
}

int orc_fit(const orc_problem* p, const orc_opts* o, const double* x,
            const double* b1p, const double* b1m, double* y,
            double* F, double* nll_out, double* jtv_out, double* cg_rel)
{
    return fit_loop(p, NULL, o, x, b1p, b1m, NULL, NULL, NULL, y, F, nll_out, jtv_out, cg_rel);
}

int orc_fit_proj(const orc_problem* p, const orc_projection* q, const orc_opts* o,
                 const double* const* x, const double* const* b1p, const double* const* b1m,
                 double* y, double* F, double* nll_out, double* jtv_out, double* cg_rel)
{
    return fit_loop(p, q, o, NULL, NULL, NULL, x, b1p, b1m, y, F, nll_out, jtv_out, cg_rel);
}
