/*
 * mpm_oracle.h -- FP64 CPU oracle of the model-based multi-parameter-mapping
 * fit (Balbastre et al., "Model-Based Multi-Parameter Mapping", 2021).
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA library it checks.
 *
 * Conventions (all arrays are caller-owned, double precision, voxel index
 * n = x + nx*(y + ny*z), x fastest):
 *   y     [K][N]   log-parameter maps (log A, log R1, log R2*, logit delta),
 *                  Sec. 2.4; K = 4 when any contrast has an MT pulse, else 3.
 *   x     [I][N]   observed images, contrast-major (all echoes of contrast 0,
 *                  then contrast 1, ...), I = sum of n_echoes.
 *   b1p   [N]      transmit efficiency, NULL = 1 (footnote to Eq. 26).
 *   b1m   [C][N]   receive modulation per contrast, NULL = 1.
 *   g     [K][N]   gradient of the negative log-likelihood (Eq. 6).
 *   h     [T][N]   approximate Hessian (Eq. 24), T = K(K+1)/2, upper triangle
 *                  row by row: 00,01,02,03,11,12,13,22,23,33 (K = 4) or
 *                  00,01,02,11,12,22 (K = 3).
 *   w     [N]      JTV weights (Eq. 40).
 */
#ifndef MPM_ORACLE_H
#define MPM_ORACLE_H

#define ORC_MAX_CONTRASTS 8
#define ORC_MAX_IMAGES 128

typedef struct {
    int nx, ny, nz;
    double vx[3];                       /* voxel size (mm) along x, y, z */
    int n_contrasts;
    int n_echoes[ORC_MAX_CONTRASTS];
    double alpha[ORC_MAX_CONTRASTS];    /* nominal flip angle (rad) */
    double tr[ORC_MAX_CONTRASTS];       /* repetition time (s) */
    int mt[ORC_MAX_CONTRASTS];          /* 1 = off-resonance MT pulse */
    double sigma2[ORC_MAX_CONTRASTS];   /* noise variance per contrast */
    double te[ORC_MAX_IMAGES];          /* echo times (s), contrast-major */
    int n_maps;                         /* K: 4 with an MT contrast, else 3 */
    double lambda[4];                   /* JTV factor per map (Eq. 38) */
    double eps;                         /* JTV smoothing, w = (u+eps^2)^-1/2 */
    int precond;                        /* 0 diag|H_f|, 1 |H_f|1, 2 Gauss-Newton */
} orc_problem;

typedef struct {
    int gn_iters;          /* Newton (Gauss-Newton-like) updates at most */
    int cg_iters;          /* PCG iterations per update at most */
    int newton_per_irls;   /* JTV weights refreshed every this many updates */
    int init;              /* 1: constant initial maps from the data means */
    double tol_gn;         /* stop when |F_prev - F| / |F_prev| < tol_gn (0: off) */
    double tol_cg;         /* stop PCG when |r_k| <= tol_cg |r_0| (0: off) */
    int mg_levels;         /* 0: the block preconditioner of Sec. 2.6; > 0: multigrid (orc_mg) */
    int mg_nu;
    double mg_omega;
    int mg_coarse_sweeps;
} orc_opts;

/* Multigrid V-cycle used as the CG preconditioner instead of the block
 * preconditioner (an option; not the paper's solver). */
typedef struct {
    int levels;          /* at most this many levels (>= 1) */
    int nu;              /* damped block-Jacobi sweeps before and after the coarse correction */
    double omega;        /* damping of the sweeps */
    int coarse_sweeps;   /* sweeps on the coarsest level */
} orc_mg;

/* Signal of one image in one voxel (Eq. 26 with the B1 footnote). */
double orc_signal(const double y[4], double alpha, double tr, double te,
                  int mt, double b1p, double b1m);

/* Signal, analytic gradient (Eqs. 27-30) and Hessian (Eqs. 31-34 on the
 * diagonal; off-diagonal terms derived the same way) w.r.t. the four
 * log-parameters.  d2s is row-major 4x4. */
void orc_signal_jet(const double y[4], double alpha, double tr, double te,
                    int mt, double b1p, double b1m,
                    double* s, double ds[4], double d2s[16]);

void orc_forward(const orc_problem* p, const double* y, const double* b1p,
                 const double* b1m, double* s);

/* Returns the negative log-likelihood (Eq. 25); writes g and h. */
double orc_grad_hess(const orc_problem* p, const double* x, const double* y,
                     const double* b1p, const double* b1m, double* g, double* h);

/* Spatial projection (Sec. 2.4).  Contrast c was acquired on its own grid of
 * dims[c] voxels (x fastest); affine[c] is the row-major 3 x 4 map from its
 * voxel coordinates (i, j, k, 1) to reconstruction voxel coordinates. */
typedef struct {
    int dims[ORC_MAX_CONTRASTS][3];
    double affine[ORC_MAX_CONTRASTS][12];
} orc_projection;

/* Psi u: trilinear interpolation of `channels` reconstruction-space images
 * u[ch][N] at A m for every acquisition voxel m; out[ch][M].  inside[m] (may
 * be NULL) is 1 when A m lies in the reconstruction grid, else 0 and out = 0. */
void orc_pull(const orc_problem* p, const int dims[3], const double A[12], int channels,
              const double* u, double* out, unsigned char* inside);

/* out[ch][N] += Psi' u (the adjoint of orc_pull; u is [ch][M]). */
void orc_push(const orc_problem* p, const int dims[3], const double A[12], int channels,
              const double* u, double* out);

/* NLL of the projected model (Sec. 2.4); g = sum_c Psi_c' g_c and
 * h = sum_c Psi_c' h_c (block-diagonal majoriser).  x[c] is [E_c][M_c];
 * b1p[c], b1m[c] are [M_c] (the arrays or their entries may be NULL). */
double orc_grad_hess_proj(const orc_problem* p, const orc_projection* q,
                          const double* const* x, const double* const* b1p,
                          const double* const* b1m, const double* y, double* g, double* h);

/* orc_init with each image's mean over its own acquisition grid. */
void orc_init_proj(const orc_problem* p, const orc_projection* q, const double* const* x,
                   double* y);

/* orc_fit with the projected likelihood. */
int orc_fit_proj(const orc_problem* p, const orc_projection* q, const orc_opts* o,
                 const double* const* x, const double* const* b1p, const double* const* b1m,
                 double* y, double* F, double* nll, double* jtv, double* cg_rel);

/* Returns JTV_eps(y) = sum_n sqrt(u_n + eps^2); writes w when w != NULL. */
double orc_jtv(const orc_problem* p, const double* y, double* w);

/* out = (G'WG (x) diag(lambda)) v   (Sec. 2.5). */
void orc_membrane(const orc_problem* p, const double* w, const double* v, double* out);

/* d = diag(G'WG)  ("cross" kernel applied to w, Sec. 2.5). */
void orc_membrane_diag(const orc_problem* p, const double* w, double* d);

/* PCG on (H + L) x = b with block preconditioner H + diag(G'WG) (x) diag(lambda)
 * (Sec. 2.6).  x starts at zero.  resid[k] = |r_k| (k = 0..returned count),
 * may be NULL.  Returns the number of iterations run. */
int orc_pcg(const orc_problem* p, const double* h, const double* w, const double* b,
            double* x, int max_iters, double tol, double* resid);

/* delta = (H + L)^-1 (g + L y) by orc_pcg (Eq. 42). */
int orc_solve(const orc_problem* p, const double* h, const double* w, const double* g,
              const double* y, double* delta, int max_iters, double tol, double* resid);

/* Number of multigrid levels for this grid (at most mg->levels; a level of
 * at most 512 voxels is the coarsest) and their dimensions (dims may be NULL). */
int orc_mg_levels(const orc_problem* p, const orc_mg* mg, int dims[][3]);

/* z = one V-cycle applied to r ([K][N]). */
void orc_mg_vcycle(const orc_problem* p, const double* h, const double* w, const orc_mg* mg,
                   const double* r, double* z);

/* e' A_l e for a vector e ([K][N_l]) of level `level` (the Galerkin coarse operator). */
double orc_mg_energy(const orc_problem* p, const double* h, const double* w, const orc_mg* mg,
                     int level, const double* e);

/* orc_pcg with the V-cycle as preconditioner. */
int orc_mg_pcg(const orc_problem* p, const double* h, const double* w, const double* b,
               double* x, int max_iters, double tol, const orc_mg* mg, double* resid);

/* delta = (H + L)^-1 (g + L y) by orc_mg_pcg. */
int orc_mg_solve(const orc_problem* p, const double* h, const double* w, const double* g,
                 const double* y, double* delta, int max_iters, double tol, const orc_mg* mg,
                 double* resid);

/* var[K][N]: diagonal of (H + diag(G'WG) (x) lambda)^-1 (Eq. 43); logdet[N]
 * (may be NULL): log-determinant of that covariance block; moments[4][N] (may be
 * NULL, needs y): E[r1], V[r1], E[t1], V[t1] (Eqs. 44-47).  Returns 0, or -1 if a
 * block is not positive definite. */
int orc_uncertainty(const orc_problem* p, const double* h, const double* w,
                    const double* y, double* var, double* logdet, double* moments);

/* Constant initial maps from the image means (Sec. 2.7, read as described in
 * the source). */
void orc_init(const orc_problem* p, const double* x, double* y);

/* The whole fit (Sec. 2.6-2.7).  F, nll, jtv: gn_iters+1 entries each (objective
 * before every update and after the last); cg_rel: gn_iters entries
 * (|r_end|/|r_0| of each solve).  Any may be NULL.  Returns the number of
 * updates made. */
int orc_fit(const orc_problem* p, const orc_opts* o, const double* x,
            const double* b1p, const double* b1m, double* y,
            double* F, double* nll, double* jtv, double* cg_rel);

/* Threads of the OpenMP build (the serial build ignores n and returns 1).
 * n > 0 sets the count; returns the count in use.  Results do not depend on
 * it: volume-wide sums are taken in fixed voxel chunks. */
int orc_threads(int n);

#endif
