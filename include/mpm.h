/*
 * mpm.h -- C ABI of the GB300 (sm_103a) implementation of the model-based
 * multi-parameter-mapping fit of Balbastre et al., "Model-Based
 * Multi-Parameter Mapping" (Medical Image Analysis, 2021).
 *
 * The fit recovers, in every voxel, the log-parameters
 *     y = (log A, log R1, log R2*, logit delta)            (Sec. 2.4)
 * from multi-echo spoiled-gradient-echo images acquired at several flip angles
 * with an optional MT pulse, by Newton updates with the paper's positive
 * definite approximate Hessian (Eq. 24) and a joint-total-variation prior
 * handled by reweighted least squares (Eqs. 38-40), each update solving
 * (H + L) delta = g + L y by preconditioned conjugate gradient (Eq. 42).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Grid: nx * ny * nz = N voxels, voxel n = x + nx*(y + ny*z) (x fastest).
 *  - Arrays are caller-owned DEVICE pointers (cudaMalloc / torch CUDA
 *    tensors), contiguous, aligned to their element size (a misaligned one is
 *    rejected with MPM_ERR_INVALID_ARG), planar.  With 16-byte alignment, as
 *    cudaMalloc and torch give, the solver streams float4 vectors and stages
 *    the stencil operands by TMA.  Otherwise it takes its scalar and
 *    shared-memory kernels.  Both paths meet the same parity bounds against
 *    the reference; their reductions group the sums differently, so the two
 *    agree to rounding, not bit for bit:
 *        y, g, delta, var      [K][N] float   K = n_maps
 *        h                     [T][N] float   T = K(K+1)/2, upper triangle row
 *                              by row: 00,01,02,03,11,12,13,22,23,33 (K=4) or
 *                              00,01,02,11,12,22 (K=3)
 *        x (images)            [I][N] float or bf16 (problem.echo_dtype),
 *                              I = sum of n_echoes, contrast-major
 *        b1p                   [N] float or NULL (= 1)
 *        b1m                   [C][N] float or NULL (= 1)
 *        w (JTV weights)       [N] float
 *    Host pointers are rejected with MPM_ERR_INVALID_ARG.
 *  - Device scalars (nll, jtv) are caller-owned device doubles, overwritten.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  The fits (mpm_fit, mpm_fit_batch, mpm_fit_proj), mpm_autotune
 *    and the server calls synchronise as their comments say; every other call
 *    only enqueues work on it and returns without synchronising.
 *  - Scratch memory: calls that need it take a caller-owned device workspace
 *    (ws, ws_bytes) of at least mpm_workspace_size() bytes.  The library
 *    allocates no device memory at run time (mpm_solve_static uses a fixed
 *    array compiled into the library instead).  Two calls that run
 *    concurrently must not share a workspace.
 *  - Errors: every call returns an mpm_status; argument errors are detected on
 *    the host before anything is enqueued.  Kernels never trap: numeric
 *    failures (a preconditioner block that is not positive definite, a NaN in
 *    a CG inner product) are recorded in the workspace and reported by
 *    mpm_fit, or read back with mpm_workspace_status().  mpm_last_error()
 *    gives a human-readable detail of the last failure on the calling thread.
 */
#ifndef MPM_H
#define MPM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MPM_MAX_CONTRASTS 8
#define MPM_MAX_IMAGES 64
#define MPM_MAX_REPORT 256
#define MPM_MAX_BATCH 64

typedef int mpm_status;

enum {
    MPM_OK = 0,
    MPM_WARN_NOT_CONVERGED = 1,       /* mpm_fit hit gn_iters with tol_gn > 0 */
    MPM_ERR_INVALID_ARG = -1,
    MPM_ERR_WORKSPACE_TOO_SMALL = -2,
    MPM_ERR_CUDA = -3,
    MPM_ERR_NUMERIC = -4,
    MPM_ERR_TIMEOUT = -5              /* reserved; a bounded copy wait that runs out
                                         inside a kernel is reported as
                                         MPM_ERR_NUMERIC (see mpm_workspace_status) */
};

/* Which call a workspace is sized for (mpm_workspace_size). */
enum {
    MPM_CALL_FIT = 0,
    MPM_CALL_SOLVE = 1,
    MPM_CALL_GRAD_HESS = 2,
    MPM_CALL_JTV = 3
};

/* Problem statement: the fixed parameters Theta of every image (Sec. 2.4:
 * flip angle, TR, TE, noise variance), the grid, and the prior (Sec. 2.5). */
typedef struct {
    int nx, ny, nz;
    double vx[3];                          /* voxel size along x, y, z (mm) */
    int n_contrasts;                       /* C, 1..MPM_MAX_CONTRASTS */
    int n_echoes[MPM_MAX_CONTRASTS];       /* echoes per contrast (>= 1) */
    double alpha[MPM_MAX_CONTRASTS];       /* nominal flip angle (rad), in (0, pi) */
    double tr[MPM_MAX_CONTRASTS];          /* repetition time (s), > 0 */
    int mt[MPM_MAX_CONTRASTS];             /* 1 if the contrast has an MT pulse */
    double sigma2[MPM_MAX_CONTRASTS];      /* noise variance of the contrast, > 0 */
    double te[MPM_MAX_IMAGES];             /* echo times (s), contrast-major */
    int n_maps;                            /* K: 4 if any mt[c], else 3 */
    double lambda[4];                      /* JTV factor per map (>= 0) */
    double eps;                            /* JTV smoothing: w = (u + eps^2)^-1/2, > 0 */
    int precond;                           /* loading of Eq. 24: 0 = |diag H_f| (the
                                              paper's choice), 1 = |H_f| 1 (row sums,
                                              "Proposed+"), 2 = none (Gauss-Newton) */
    int echo_dtype;                        /* 0 = float32 images, 1 = bfloat16 */
} mpm_problem;

/* Schedule (Sec. 2.7; the paper uses 10 IRLS x 5 Newton x 32 CG). */
typedef struct {
    int gn_iters;          /* Newton updates at most, 0..MPM_MAX_REPORT */
    int cg_iters;          /* PCG iterations per update at most, >= 1 */
    int newton_per_irls;   /* JTV weights refreshed every this many updates, >= 1 */
    int init;              /* 1: start from constant maps computed from the image
                              means; 0: y_inout holds the starting maps */
    double tol_gn;         /* stop when |F_prev - F| < tol_gn |F_prev| (0 = off) */
    double tol_cg;         /* stop PCG when |r_k| <= tol_cg |r_0| (0 = off) */
    int graph;             /* 1: with tol_gn = 0, run all updates as one captured CUDA
                              graph (instantiated on first use, cached per argument
                              set, replayed afterwards); 2: the same, phase-batched
                              across the subjects of mpm_fit_batch (see there);
                              0: direct launches */
    /* Preconditioner of the solve.  mg_levels = 0: the block preconditioner
     * H + diag(G'WG) (x) diag(lambda) of Sec. 2.6 (the paper's solver).
     * mg_levels >= 1 (an option the paper does not have): conjugate gradient
     * preconditioned by one aggregation multigrid V-cycle with at most
     * mg_levels levels (each merging 2 x 2 x 2 voxels; a level of at most 512
     * voxels is the coarsest), Galerkin coarse operators, damped block-Jacobi
     * smoothing.  The three fields below take their defaults when 0. */
    int mg_levels;         /* 0..16 */
    int mg_nu;             /* sweeps before and after each coarse correction (1) */
    double mg_omega;       /* damping of the sweeps, in (0, 2) (0.7) */
    int mg_coarse_sweeps;  /* sweeps on the coarsest level (20) */
} mpm_opts;

/* Per-update record filled by mpm_fit (host memory, caller-owned). */
typedef struct {
    int iters;                             /* updates made */
    double F[MPM_MAX_REPORT + 1];          /* NLL + JTV_eps before every update and
                                              after the last (entries 0..iters) */
    double nll[MPM_MAX_REPORT + 1];        /* negative log-likelihood, Eq. 25 */
    double jtv[MPM_MAX_REPORT + 1];        /* sum_n sqrt(u_n + eps^2), Eq. 38 */
    double cg_rel[MPM_MAX_REPORT];         /* |r_end| / |r_0| of each solve */
    int cg_done[MPM_MAX_REPORT];           /* PCG iterations run in each solve */
} mpm_report;

/* Text of a status code (static storage). */
const char* mpm_status_string(mpm_status s);

/* Detail of the last failing call on this thread ("" if none). */
const char* mpm_last_error(void);

/* Bytes of workspace that `call` (MPM_CALL_*) needs for this problem and
 * schedule (opts may be NULL except for MPM_CALL_FIT / MPM_CALL_SOLVE).  The
 * MPM_CALL_FIT size is enough for every call. */
mpm_status mpm_workspace_size(const mpm_problem* problem, const mpm_opts* opts, int call,
                              size_t* bytes);

/* Noise-free images s[I][N] (float32) from maps y (Eq. 26 with the B1
 * modulation of its footnote: flip angle alpha * b1p, signal times b1m). */
mpm_status mpm_forward(const mpm_problem* problem, const float* y, const float* b1p,
                       const float* b1m, float* s, void* stream);

/* The fused voxel pass (Eqs. 6, 24, 25, 27-34): in every voxel, over all
 * echoes of all contrasts, the signal, residual, gradient g[K][N] of the
 * negative log-likelihood and the approximate Hessian h[T][N]; *nll (device
 * double) receives the negative log-likelihood summed over the volume. */
mpm_status mpm_grad_hess(const mpm_problem* problem, const void* x, const float* y,
                         const float* b1p, const float* b1m, float* g, float* h,
                         double* nll, void* ws, size_t ws_bytes, void* stream);

/* JTV reweighting (Eqs. 38-40): u_n = sum_k lambda_k sum_{6 neighbours}
 * (y_k[m] - y_k[n])^2 / h_d^2 (neighbours outside the volume dropped),
 * w_n = (u_n + eps^2)^-1/2 written to w (skipped if w == NULL), and
 * *jtv = sum_n sqrt(u_n + eps^2). */
mpm_status mpm_jtv_weights(const mpm_problem* problem, const float* y, float* w,
                           double* jtv, void* ws, size_t ws_bytes, void* stream);

/* Newton system of Sec. 2.6 / Eq. 42: delta = (H + L)^-1 (g + L y) with
 * L = G'WG (x) diag(lambda), by PCG from delta = 0 with the block
 * preconditioner H + diag(G'WG) (x) diag(lambda), at most opts->cg_iters
 * iterations or until |r_k| <= opts->tol_cg |r_0|.  resid (device doubles,
 * cg_iters + 1 entries, or NULL) receives |r_k|; entries past the last
 * iteration run are left untouched. */
mpm_status mpm_solve(const mpm_problem* problem, const mpm_opts* opts, const float* h,
                     const float* w, const float* g, const float* y, float* delta,
                     double* resid, void* ws, size_t ws_bytes, void* stream);

/* mpm_solve without a caller workspace (the paper has no counterpart: this is
 * an interface for callers that cannot allocate device memory).  Some callers
 * cannot call cudaMalloc at all: code running inside another framework's
 * memory pool that owns the whole device, real-time pipelines that reserve
 * every byte up front, or paths that must not hit cudaMalloc's implicit device
 * synchronisation.  This entry point takes the same arguments as mpm_solve
 * minus (ws, ws_bytes), and keeps its scratch in a fixed 64 MiB device array
 * owned by the library.  Every GPU that loads the library holds that array
 * until the process exits.
 *  - Size limit: problems whose solve scratch exceeds 64 MiB (about 450 000
 *    voxels, e.g. 80 x 80 x 64) are refused with
 *    MPM_ERR_WORKSPACE_TOO_SMALL and a message giving the bytes needed; use
 *    mpm_solve with a workspace for those.
 *  - Allocates nothing: no cudaMalloc, no cudaFree, no allocating library
 *    routine.  The first call on each device looks up the array's device
 *    address (cudaGetSymbolAddress, with that device current); make that
 *    first call before any stream capture.
 *  - Shared state: all calls on a device share the one array, which keeps the
 *    last call's contents (the call clears what must start at zero).  Calls
 *    whose work overlaps on the GPU (other streams, other threads) race on it
 *    and must be serialised by the caller.
 * Numeric failures are not readable through mpm_workspace_status here; a NaN
 * or non positive definite block shows as non-finite entries of delta and
 * resid. */
mpm_status mpm_solve_static(const mpm_problem* problem, const mpm_opts* opts, const float* h,
                            const float* w, const float* g, const float* y, float* delta,
                            double* resid, void* stream);

/* Laplace uncertainty (Sec. 3.6, Eqs. 43-47): var[K][N] = diagonal of
 * (H_n + diag(G'WG)_n lambda)^-1, from float32 Cholesky factors of the
 * diagonally equilibrated blocks (float64 for a block whose smallest
 * equilibrated pivot is below 1e-2); logdet[N] (or NULL) = log-determinant of
 * that covariance block; moments[4][N] (or NULL; needs y) = E[r1], V[r1],
 * E[t1], V[t1] under the log-normal posterior.  A block that is not positive
 * definite gives non-finite entries (the call takes no workspace to report
 * it). */
mpm_status mpm_uncertainty(const mpm_problem* problem, const float* h, const float* w,
                           const float* y, float* var, float* logdet, float* moments,
                           void* stream);

/* The whole fit (Sec. 2.6-2.7): optional constant initial maps, then up to
 * gn_iters updates, each = JTV reweighting (every newton_per_irls updates),
 * fused voxel pass, PCG solve and y <- y - delta; the objective
 * F = NLL + JTV_eps is evaluated before every update and at the final maps.
 * If var_out != NULL the uncertainty at the final maps is written there
 * ([K][N]).  Synchronises `stream` before returning.  Returns MPM_OK,
 * MPM_WARN_NOT_CONVERGED (tol_gn > 0 and not reached) or an error. */
mpm_status mpm_fit(const mpm_problem* problem, const mpm_opts* opts, const void* x,
                   const float* b1p, const float* b1m, float* y_inout, float* var_out,
                   void* ws, size_t ws_bytes, mpm_report* report, void* stream);

/* Tile-shape autotuner for the PCG iteration kernel of the solve.  The
 * TMA-staged iteration can tile the (x, y) plane as 16 x 16, 32 x 8 or
 * 32 x 16 voxels; this
 * call times each applicable shape on this volume (zeroed operands in `ws`, a
 * MPM_CALL_SOLVE-sized workspace or larger), keeps the fastest for every later
 * solve of a volume of this size in the process, and writes its index to
 * *tile (-1 when the TMA kernel does not apply: nx not a multiple of 4, or the
 * volume smaller than a tile) and the mean time per launch of each shape to
 * ms[0..MPM_TILE_SHAPES-1] (-1 for shapes that do not apply; may be NULL).
 * If *tile >= 0 on entry, that shape is recorded without timing (ws may then
 * be NULL).  Without either, a default shape is used.  A shape that does not
 * fit a volume falls back to the plain iteration kernel.  Synchronises
 * `stream` when timing. */
#define MPM_TILE_SHAPES 3
mpm_status mpm_autotune(const mpm_problem* problem, const mpm_opts* opts, void* ws,
                        size_t ws_bytes, void* stream, int* tile, float* ms);

/* Several subjects fitted together (batched fits; the paper fits one subject
 * at a time).  Each subject i has its own problem (matrix size, contrasts and
 * echo counts may all differ), images x[i], optional b1p[i] / b1m[i] (the
 * arrays themselves may be NULL), maps y[i], optional var_out[i] and
 * workspace ws[i] of ws_bytes[i]; opts and the report array (n entries, may
 * be NULL) are shared.  With tol_gn = 0 and opts->graph = 1 the updates of all
 * subjects are captured into one CUDA graph (cached per argument set) as
 * lanes run side by side: subjects of about 2^21 voxels or more one after
 * another in one lane, the smaller ones dealt over as many lanes as keep the
 * load of the lanes running together within 1.5 (0.5 beside the large lane;
 * a subject's load is voxels / 2^21), so uneven volumes share the GPU in one
 * graph launch; each subject's result is its mpm_fit result bit for bit.
 * With opts->graph = 2 the graph is phase-batched instead: subjects that
 * share the map count, the preconditioner choice, the echo type and the tile
 * shape of the PCG iteration (each keeps its solo fit's) form a class; in
 * groups of at most 16, each phase of each update (JTV reweighting, voxel
 * pass, PCG start, every PCG iteration, PCG end, the posterior variance) is
 * ONE kernel launch for the whole group, each subject on its own share of the
 * blocks with its own scalars and reductions (the PCG iteration's wave of
 * resident blocks is divided so that the subject that finishes last does so
 * soonest, the other phases' blocks in proportion to the voxels); groups that
 * fill the GPU run one after another, smaller groups side by side.  Subjects that the TMA-staged iteration
 * cannot take (x size not a multiple of 4, a volume smaller than the tile's
 * box, an unaligned buffer), projected fits and multigrid solves run in lanes
 * as with graph = 1, beside the groups.  A batched subject's reductions sum
 * over fewer blocks than in its solo fit, so its result matches the solo
 * result to float32 rounding, not bit for bit.  Otherwise (graph = 0 or
 * tol_gn > 0) subjects run one after another, each exactly as its
 * mpm_fit.  Synchronises `stream`.  0 <= n <= MPM_MAX_BATCH; n = 0
 * returns MPM_OK at once, without touching any argument or the stream. */
mpm_status mpm_fit_batch(int n, const mpm_problem* const* problems, const mpm_opts* opts,
                         const void* const* x, const float* const* b1p, const float* const* b1m,
                         float* const* y, float* const* var_out, void* const* ws,
                         const size_t* ws_bytes, mpm_report* reports, void* stream);

/* Spatial projection (Sec. 2.4, "Spatial projection"): contrast c was
 * acquired on its own grid of dims[c] voxels (x fastest, M_c voxels) and
 * affine[c] is the row-major 3 x 4 map from its voxel coordinates (i, j, k, 1)
 * to reconstruction voxel coordinates (voxel centres at integer coordinates,
 * both 0-based; a world-space pair of voxel-to-world matrices gives
 * affine = inv(recon) * acq).  The paper's reslicing matrix Psi_c is
 * trilinear interpolation at affine[c] * m; an acquisition voxel whose point
 * lies outside [0, n_d - 1] on some axis of the reconstruction grid carries no
 * data term.  Singular or non-finite affines are refused, and so are
 * acquisition grids more than 4x finer than the reconstruction grid along an
 * axis (the row sums of the inverse affine's linear part must be <= 4). */
typedef struct {
    int dims[MPM_MAX_CONTRASTS][3];
    double affine[MPM_MAX_CONTRASTS][12];
} mpm_projection;

/* Workspace of the projected calls (call = MPM_CALL_FIT or
 * MPM_CALL_GRAD_HESS): the plain size plus the per-contrast gradient and
 * Hessian buffers on the acquisition grids. */
mpm_status mpm_workspace_size_proj(const mpm_problem* problem, const mpm_projection* proj,
                                   const mpm_opts* opts, int call, size_t* bytes);

/* out[ch][M_c] = Psi_c u for `channels` reconstruction-space images
 * u[ch][N] (the pull of Sec. 2.4). */
mpm_status mpm_pull(const mpm_problem* problem, const mpm_projection* proj, int contrast,
                    int channels, const float* u, float* out, void* stream);

/* out[ch][N] = Psi_c' u (+ out if accumulate) for u[ch][M_c]: the adjoint of
 * mpm_pull with the same weights (the push of Sec. 2.4).  Each output voxel
 * gathers its terms in a fixed order, so results repeat bit for bit. */
mpm_status mpm_push(const mpm_problem* problem, const mpm_projection* proj, int contrast,
                    int channels, const float* u, float* out, int accumulate, void* stream);

/* The projected voxel pass (Sec. 2.4 with Eqs. 6, 24-34): per contrast, the
 * maps y[K][N] are pulled to its grid, the NLL, gradient g_c and loaded
 * Hessian H_c of its echoes are formed per acquisition voxel, and
 * g = sum_c Psi_c' g_c, h = sum_c Psi_c' H_c (the block-diagonal majoriser of
 * Psi' H Psi, Ashburner et al. 2018 as cited there).  x[c] points to contrast
 * c's echoes [E_c][M_c] (float32, or bfloat16 with echo_dtype = 1); b1p[c],
 * b1m[c] to its B1 fields [M_c] (the arrays or their entries may be NULL: 1).
 * x, b1p, b1m are host arrays of device pointers.  *nll (device) = the
 * summed NLL.  ws: mpm_workspace_size_proj(..., MPM_CALL_GRAD_HESS) bytes. */
mpm_status mpm_grad_hess_proj(const mpm_problem* problem, const mpm_projection* proj,
                              const void* const* x, const float* const* b1p,
                              const float* const* b1m, const float* y, float* g, float* h,
                              double* nll, void* ws, size_t ws_bytes, void* stream);

/* mpm_fit with the projected likelihood (the JTV prior and the solve stay on
 * the reconstruction grid).  Constant initial maps use each image's mean over
 * its own acquisition grid.  ws: mpm_workspace_size_proj(..., MPM_CALL_FIT). */
mpm_status mpm_fit_proj(const mpm_problem* problem, const mpm_projection* proj,
                        const mpm_opts* opts, const void* const* x, const float* const* b1p,
                        const float* const* b1m, float* y_inout, float* var_out, void* ws,
                        size_t ws_bytes, mpm_report* report, void* stream);

/* Continuous batching of fit requests (a serving loop; the paper fits one
 * subject at a time).  The server owns no device memory: every admitted
 * request's fit workspace is carved from `arena` (caller-owned device memory,
 * 256-byte aligned), so admission follows the free HBM the caller hands over.
 * Requests are admitted while one of `max_slots` slots is free, their
 * workspace fits and the GPU load allows: a request's load is
 * min(1, voxels / 2^21) (about 2^21 voxels keep every kernel of a fit at a full
 * wave) and the active requests' loads may sum to at most 1.5, so one large
 * fit runs with small ones beside it but never two large fits at once.  Among
 * those, the smallest volume goes first (ties by arrival; when the smallest
 * does not fit the arena, the first in arrival order that does); a request
 * overtaken by 2 x max_slots later ones goes before all others, so none
 * starves.  An active request keeps its maps, weights, gradient, Hessian and
 * PCG state resident in the arena until it is done.  The server creates CUDA streams
 * of its own (per slot, one for each stream priority level of the device) and
 * pinned host staging per slot;
 * `stream` is the caller's stream on which the request inputs are produced
 * (each request waits for the state of that stream at its submission).
 *  - mpm_server_submit: queue one fit (same arguments as mpm_fit minus the
 *    workspace and report; x, b1p, b1m, y_inout, var_out stay caller-owned
 *    and must stay valid until the request is done).  Returns a ticket.
 *    Refuses requests larger than the whole arena.
 *  - mpm_server_step: one non-blocking pass -- every active request whose
 *    last enqueued work has completed moves on (initial maps; the stopping
 *    rule of mpm_fit on its objective; then either its PCG solve, update and
 *    next evaluation, or its uncertainty and report; finished requests
 *    release their workspace), then queued requests are admitted into free
 *    slots while the arena has room.  Requests run on their own streams and
 *    advance independently, so their kernels overlap on the GPU; smaller
 *    volumes get higher stream priorities (below 2^19 voxels the highest,
 *    one level lower per doubling).  Call it in a loop; reports the active,
 *    queued and just-finished counts (any pointer may be NULL).
 *  - mpm_server_poll: state of a ticket (MPM_REQ_*), its final status and,
 *    once done, its report.  The server keeps a finished request's state and
 *    report (about 10 KB of host memory) until mpm_server_release.
 *  - mpm_server_release: forgets a finished ticket (MPM_REQ_DONE or
 *    MPM_REQ_FAILED), after which polling it is an error.  A ticket that is
 *    still queued or active is refused with MPM_ERR_INVALID_ARG.
 *  - mpm_server_destroy: waits for the work already enqueued on the server's
 *    streams, then frees its streams, events and staging; requests not yet
 *    done are dropped (their outputs are undefined).  NULL is a no-op that
 *    returns MPM_OK.
 * A request's result equals mpm_fit's with the same arguments.  The server is
 * guarded by a mutex; calls from several threads are serialised. */
enum { MPM_REQ_QUEUED = 0, MPM_REQ_ACTIVE = 1, MPM_REQ_DONE = 2, MPM_REQ_FAILED = 3 };
typedef struct mpm_server mpm_server;
mpm_status mpm_server_create(void* arena, size_t arena_bytes, int max_slots, void* stream,
                             mpm_server** out);
mpm_status mpm_server_submit(mpm_server* server, const mpm_problem* problem, const mpm_opts* opts,
                             const void* x, const float* b1p, const float* b1m, float* y_inout,
                             float* var_out, int* ticket);
mpm_status mpm_server_step(mpm_server* server, int* n_active, int* n_queued, int* n_finished);
mpm_status mpm_server_poll(mpm_server* server, int ticket, int* state, mpm_status* status,
                           mpm_report* report);
mpm_status mpm_server_release(mpm_server* server, int ticket);
mpm_status mpm_server_destroy(mpm_server* server);

/* Synchronises `stream` and returns MPM_ERR_NUMERIC if a kernel that used this
 * workspace recorded a failure since the workspace was last cleared (every
 * mpm_solve / mpm_fit clears it): a preconditioner block that is not positive
 * definite, a NaN in a reduction, or a bounded copy wait of the PCG iteration
 * or of the voxel pass that ran out (mpm_last_error() names which).  Every
 * mpm_grad_hess call clears it too.  Otherwise MPM_OK. */
mpm_status mpm_workspace_status(const void* ws, size_t ws_bytes, void* stream);

/* Test hook for the bounded waits of the staged kernels, the TMA-staged PCG
 * iteration and the staged voxel pass (the paper has no counterpart; tests
 * use it to drive the timeout path without a fault).  withhold != 0: from the
 * next launch on, their producers issue no copies, so every copy wait of
 * their compute warps runs out.
 * wait_us > 0 sets the bound of every such wait (converted to clock cycles
 * at the current device's clock rate); 0 restores the default of about 2 s.
 * A launch whose wait ran out skips its work, drains its own copies, records
 * the failure in the workspace status (mpm_workspace_status reports
 * MPM_ERR_NUMERIC, "copy wait timed out") and returns; the solve then stops
 * without a step, and the voxel pass leaves g and h undefined.  Process-wide.  Returns MPM_ERR_INVALID_ARG for
 * wait_us < 0. */
mpm_status mpm_test_copy_timeout(int withhold, double wait_us);

/* Diagnostic: number of kernels this library has launched in this process. */
unsigned long long mpm_kernel_launches(void);

/* Kernel kinds reported by mpm_profile_read. */
enum {
    MPM_KERNEL_GRAD_HESS = 0,    /* fused voxel pass */
    MPM_KERNEL_JTV = 1,          /* JTV weights */
    MPM_KERNEL_PCG_INIT = 2,     /* r0 = g + L y, z0 = M^-1 r0 */
    MPM_KERNEL_PCG_STEP = 3,     /* one PCG iteration: z, p, q = (H + L) p, v = M^-1 q, x */
    MPM_KERNEL_PCG_FINAL = 4,    /* delta or y update */
    MPM_KERNEL_UNCERTAINTY = 5,
    MPM_KERNEL_FORWARD = 6,
    MPM_KERNEL_INIT = 7,         /* image means and constant maps */
    MPM_KERNEL_GRAD_HESS_PROJ = 8, /* projected voxel pass, one contrast */
    MPM_KERNEL_RESLICE = 9,      /* pull / push of the spatial projection */
    MPM_KERNEL_MG = 10,          /* multigrid hierarchy and V-cycle (mg_levels > 0) */
    MPM_KERNEL_KINDS = 11
};

/* Diagnostic timing.  While enabled (on != 0, process-wide), every kernel
 * launch is bracketed by two CUDA events recorded on its stream.
 * mpm_profile_read waits for those events, writes per kind the summed
 * milliseconds (ms[k]) and launch counts (launches[k]) for k < n, and clears
 * the records.  Either output may be NULL. */
mpm_status mpm_profile_enable(int on);
mpm_status mpm_profile_read(double* ms, unsigned long long* launches, int n);

#ifdef __cplusplus
}
#endif

#endif /* MPM_H */
