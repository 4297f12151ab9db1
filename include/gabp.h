/*
 * gabp.h — C ABI of the GB300 Gaussian belief propagation library (libgabp.so).
 *
 * The library solves the spatial data-assimilation posterior of "Scalable Data
 * Assimilation with Message Passing" (Key, Takao, Giles, Deisenroth): a 2-D grid field f
 * with the SPDE/GMRF prior of Sec. 3.1 (L f = w, L = kappa^2 I - Delta_h, prior precision
 * gamma L^T L) and linear Gaussian observations y = H f + noise (Sec. 2.1), by synchronous
 * ("flooding") Gaussian belief propagation in information form (Sec. 2.3, Alg. 1; App. A;
 * Alg. 2 "Iterate MP Until Convergence").
 *
 * Factor graph.  One rank-1 factor exp(-(gamma/2) (l_i . f)^2) per grid cell i, with l_i
 * the i-th row of L (the cell itself and its existing 4-neighbours; zero-Neumann
 * boundary, i.e. kappa^2 + deg(i) on the diagonal and -1 per neighbour), and one 4-node
 * factor exp(-(1/(2 sigma_k^2)) (h_k . f - y_k)^2) per observation, with h_k the bilinear
 * interpolation weights of the observation's location.  Messages are (eta, Lambda) pairs
 * per factor-variable edge; the beliefs are their sums (App. A, state update) and the
 * marginals are mu = eta / Lambda, sigma^2 = 1 / Lambda (App. A, marginal extraction with
 * c = 1).  The converged mean equals the exact posterior mean A^-1 b with
 * A = gamma L^T L + H^T R^-1 H and b = H^T R^-1 y.
 *
 * Conventions.
 *   - Grid: nx columns (x), ny rows (y), unit spacing, node (i, j) at x = j, y = i, stored
 *     row-major (index i * nx + j).  Every array of per-node values has nx * ny entries in
 *     that order.
 *   - Observation k sits at (obs_xy[2k], obs_xy[2k+1]) = (x, y) in grid units, inside
 *     [0, nx-1] x [0, ny-1].  Its base cell is j0 = min(floor(x), nx-2),
 *     i0 = min(floor(y), ny-2) (so x = nx-1 falls in the last cell with weight 1 on the far
 *     node); weights on (i0,j0), (i0,j0+1), (i0+1,j0), (i0+1,j0+1) are (1-fu)(1-fv),
 *     fu(1-fv), (1-fu)fv, fu fv with fu = x - j0, fv = y - i0.
 *   - Damping beta is the weight on the OLD message: m_t = beta m_{t-1} + (1 - beta) m_new
 *     (Sec. 3.2 "Update Damping" writes the weight on the new message, eta = 1 - beta).
 *   - Pointers named "host or device" may point to host memory (pageable or pinned) or to
 *     device memory of the context's device; the library detects which.
 *   - All calls are synchronous with respect to the host unless stated otherwise; they run
 *     on the context's stream (gabp_options.stream, or a stream the context creates).
 *   - The library never exits, traps or prints.  Every call returns a status code; the text
 *     of the last error is available from gabp_last_error().  After GABP_ERR_CUDA the
 *     context should be destroyed.
 */
#ifndef GABP_H
#define GABP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define GABP_OK 0
#define GABP_ERR_ARG 1       /* an argument is out of range, NULL or inconsistent */
#define GABP_ERR_OOM 2       /* device or host allocation failed */
#define GABP_ERR_CUDA 3      /* a CUDA runtime call or kernel launch failed */
#define GABP_ERR_DIVERGED 4  /* the residual became NaN/Inf or grew by more than 1e6 */
#define GABP_ERR_TIMEOUT 5   /* gabp_iterate(n < 0) reached max_iters above the tolerance, or a
                                bounded wait inside a kernel gave up (the kernel returned early;
                                the messages of that call are incomplete) */
#define GABP_ERR_STATE 6     /* call not valid in the context's current state */

/* message precision */
#define GABP_FP32 0          /* FP32 messages, compensated (two-term) belief sums */
#define GABP_FP64 1          /* FP64 messages and sums */

/* message initialisation (gabp_options.init) */
#define GABP_INIT_COLD 0     /* Lambda = s a_v^2 (the factor's own diagonal term), eta = 0 */
#define GABP_INIT_PAPER 1    /* Lambda = 1e-8, eta = 0 (Alg. 1 / Alg. 2 initialisation) */

/* iteration kernel (gabp_options.kernel) */
#define GABP_KERNEL_AUTO 0   /* FP32: GABP_KERNEL_TMA if nx is a multiple of 4, else
                                GABP_KERNEL_SWEEP; FP64: GABP_KERNEL_FUSED.  The alpha = 4
                                prior: GABP_KERNEL_FUSED (FP32), GABP_KERNEL_SPLIT (FP64) */
#define GABP_KERNEL_FUSED 1  /* one fused kernel per iteration (beliefs + all factors) */
#define GABP_KERNEL_SPLIT 2  /* three kernels per iteration: beliefs, prior factors, obs factors */
#define GABP_KERNEL_TMA 3    /* the fused kernel as persistent blocks fed by TMA tensor loads;
                                FP32 and nx a multiple of 4 only */
#define GABP_KERNEL_SWEEP 4  /* one fused kernel per iteration as warp-synchronous column sweeps
                                (30-column strips, beliefs in registers); FP32 only */

typedef struct gabp_ctx gabp_ctx;   /* opaque; owns every device buffer it allocates */

typedef struct {
    int nx;        /* columns, >= 1 (>= 2 when there are observations) */
    int ny;        /* rows,    >= 1 (>= 2 when there are observations) */
    double h;      /* grid spacing of the prior's Laplacian, > 0 (1.0 = unit spacing): L = kappa^2 I -
                      Delta_h with the 5-point Delta_h at spacing h (App. C), which is h^-2 times
                      the unit-spacing operator at kappa h; observation locations stay in grid
                      units */
} gabp_grid;

typedef struct {
    double gamma;  /* prior precision scale gamma of P = gamma L^T L (Sec. 3.1); > 0 */
    int boundary;  /* 0 = zero-Neumann (the only boundary implemented) */
    int alpha;     /* SPDE exponent (Sec. 3.1, (kappa^2 - Delta)^(alpha/2) f = W): 0 or 2 = the
                      operator L (one 5-slot factor per cell, a = row of L); 4 = L^2 (App. C,
                      powers of the operator: one 13-slot factor per cell, a = row of L^2,
                      P = gamma (L^2)^T L^2).  alpha = 4 contexts run, with FP32 messages, one
                      fused tile kernel per iteration (kernel AUTO or FUSED; tiles 28x8, the
                      default, or 28x4) or the split kernels (kernel SPLIT; the only form for
                      FP64), with bit-identical messages; their prior messages are 13 planes;
                      warm starts, multigrid and the pairwise form need alpha = 2
                      (GABP_ERR_STATE).  Other values: GABP_ERR_ARG. */
} gabp_prior;

typedef struct {
    int precision;    /* GABP_FP32 (default) or GABP_FP64 */
    int init;         /* GABP_INIT_COLD (default) or GABP_INIT_PAPER */
    int kernel;       /* GABP_KERNEL_AUTO (default), _FUSED, _SPLIT, _TMA or _SWEEP */
    int tile_x;       /* fused-kernel tile width in cells; 0 = the default / autotuned shape */
    int tile_y;       /* fused-kernel tile height in cells; 0 = the default / autotuned shape.
                         GABP_KERNEL_FUSED: 32x8, 32x16, 32x32, 64x8, 64x16, 128x8;
                         GABP_KERNEL_TMA: 30x14, 30x22, 30x30;
                         GABP_KERNEL_SWEEP: 30x16, 30x32, 30x64, 30x128;
                         GABP_KERNEL_FUSED with alpha = 4: 28x4, 28x8 */
    double tol;       /* relative-residual target of gabp_iterate(n < 0); default 1e-5 */
    int check_every;  /* iterations between residual checks when n < 0; default 50 */
    int max_iters;    /* iteration cap when n < 0; default 200000 */
    int device;       /* CUDA device ordinal; -1 (default) = the calling thread's device */
    void *stream;     /* cudaStream_t to run on; NULL (default) = a stream the context owns */
    int debug_flags;  /* 0 (default).  Bit 0 is a test hook for failure detection: every launch of
                         the TMA kernel first waits on an mbarrier that nothing completes, so its
                         bounded wait runs out (after ~2 ms) and gabp_iterate returns
                         GABP_ERR_TIMEOUT without having changed the messages; for a batch
                         the batched TMA kernel does the same and gabp_batch_iterate
                         returns GABP_ERR_TIMEOUT (its messages are then unspecified). */
    int tile_run;     /* GABP_KERNEL_TMA: tiles per run of its schedule, 1..8 (the tile rows are cut
                         into bands of tile_run rows and a block walks one band's tile column top
                         to bottom, reusing two belief rows from tile to tile); 0 (default) = the
                         length in 1..4 that balances the blocks best.  The fused alpha = 4
                         kernel: the same, reusing four belief rows; 0 = the length among 1, 2,
                         4, 8 and 16 that balances the blocks best.  Results do not depend on
                         it.  Other kernels ignore it; values outside 0..8: GABP_ERR_ARG. */
} gabp_options;

typedef struct {
    int64_t iterations;     /* iterations run since create / the last re-initialisation */
    double last_residual;   /* last relative residual computed (NaN if none yet) */
    int64_t n;              /* nodes */
    int64_t m;              /* observations */
    int64_t edges;          /* factor-variable edges: sum of prior factor sizes + 4 m */
    int precision;          /* GABP_FP32 / GABP_FP64 */
    int kernel;             /* the iteration kernel in use (GABP_KERNEL_FUSED/_SPLIT/_TMA/_SWEEP) */
    int tile_x, tile_y;     /* tile shape in use by the fused kernel */
    double bytes_per_iter;  /* algorithmic HBM bytes of one iteration (messages read and
                               written once, plus the static observation data) */
    int tile_run;           /* tiles per run of the TMA or fused alpha = 4 kernel's schedule (0 for
                               other kernels) */
} gabp_stats;

/* Fill *opt with the defaults listed above. */
void gabp_default_options(gabp_options *opt);

/*
 * Build the factor graph (Sec. 3.1 "Derivation of the Factor Graph"; Sec. 3.2
 * "Including Observations", here with bilinear observation rows) and initialise messages.
 *
 *   out        receives the new context (set to NULL on failure).
 *   grid       grid size and the spacing h of the prior's Laplacian (> 0).
 *   kappa      SPDE parameter kappa of (kappa^2 - Delta) (Eq. for the Matern SPDE); > 0.
 *   prior      prior options; NULL = { gamma = 1, zero-Neumann }.
 *   m          number of observations, >= 0.
 *   obs_xy     2m doubles (x0, y0, x1, y1, ...), HOST memory.
 *   y          m observed values, HOST memory.
 *   noise_var  m observation noise variances sigma_k^2 > 0, HOST memory.
 *   opt        options; NULL = defaults.
 *
 * The host arrays are read during the call only (the caller keeps ownership).  Observation
 * locations are validated (finite, inside the grid) and sorted by base cell on the host;
 * the interpolation weights and 1/sigma^2 are then computed on the GPU in FP64 and stored
 * in the message precision.  Errors: GABP_ERR_ARG for invalid sizes, NaN/Inf values,
 * non-positive kappa/gamma/variances or locations outside the grid; GABP_ERR_OOM;
 * GABP_ERR_CUDA.
 */
int gabp_create(gabp_ctx **out, gabp_grid grid, double kappa, const gabp_prior *prior,
                int64_t m, const double *obs_xy, const double *y, const double *noise_var,
                const gabp_options *opt);

/*
 * Run synchronous damped GaBP iterations (Alg. 2, "Iterate MP Until Convergence", with the
 * damping of Sec. 3.2): every new message uses only the previous iteration's messages.
 *
 *   n_iters >= 0: run exactly n_iters iterations.
 *   n_iters <  0: iterate until the relative residual ||b - A mu|| / ||b|| (FP64) is at most
 *                 opt.tol, checking every opt.check_every iterations; returns
 *                 GABP_ERR_TIMEOUT after opt.max_iters iterations and GABP_ERR_DIVERGED if
 *                 the residual becomes non-finite or grows by 1e6 over its best value.
 *   damping       beta in [0, 1): weight on the old message.
 *
 * Runs as CUDA-graph replays on the context's stream and synchronises before returning.
 */
int gabp_iterate(gabp_ctx *ctx, int n_iters, double damping);

/*
 * Marginals from the current messages (App. A, marginal extraction, c = 1):
 * mean = eta / Lambda and var = 1 / Lambda per node, written as FP64.  FP32 contexts form
 * the mean from the compensated (hi + lo) beliefs as a double-float quotient (about 46
 * significant bits, the value the residual uses); FP64 contexts divide in FP64.
 *   mean  nx*ny doubles, host or device; must not be NULL.
 *   var   nx*ny doubles, host or device; may be NULL.
 */
int gabp_marginals(gabp_ctx *ctx, double *mean, double *var);

/*
 * Relative residual ||b - A mu||_2 / ||b||_2 of the current mean, computed in FP64 on the
 * GPU (A applied as gamma L (L mu) + H^T R^-1 (H mu), deterministic reductions).  This is the
 * convergence measure used in place of the paper's message-change early stop (App. B).
 *   rel_residual  one double, host memory.  If ||b|| = 0 (no observations) the absolute
 *                 norm ||A mu|| is returned instead.
 */
int gabp_residual(gabp_ctx *ctx, double *rel_residual);

/*
 * Re-initialise the messages from predicted beliefs (a warm start; the closest paper
 * counterpart is the multigrid "Upscale Messages" of App. B, which also seeds messages
 * from a previous estimate): every edge into node v gets Lambda = lam0[v] / deg(v) and
 * eta = mu0[v] * Lambda, deg(v) being the number of factors touching v, so that the
 * initial beliefs equal (mu0, lam0).
 *   mu0, lam0   nx*ny doubles each, host or device; lam0 > 0.
 */
int gabp_warm_start(gabp_ctx *ctx, const double *mu0, const double *lam0);

/* Re-initialise the messages with the context's initialisation mode (opt.init). */
int gabp_reset(gabp_ctx *ctx);

/*
 * Prior mean (Sec. 2.2: the Gaussian prior N(f_b, Sigma) has a mean f_b; Sec. 4.2 uses a
 * climatology as f_b).  With the SPDE prior of Sec. 3.1 the prior factor of cell c becomes
 * exp(-(gamma / 2) (l_c . f - l_c . f_b)^2): its target is r_c = (L f_b)_c instead of 0, and
 * the posterior mean solves A mu = gamma L^T L f_b + H^T R^-1 y.  f_b: nx*ny doubles, host
 * or device, copied; NULL restores the zero mean.  The targets are formed in FP64 and stored
 * in the message precision; ||b|| is recomputed.  Messages are kept (iterating moves them to
 * the new fixed point).  GABP_ERR_STATE for the alpha = 4 prior; a context with a prior mean
 * refuses gabp_mg_create and gabp_pw_create (GABP_ERR_STATE).
 */
int gabp_set_prior_mean(gabp_ctx *ctx, const double *f_b);


/*
 * Copy the current messages out / in (checkpoint and resume).  The buffer is opaque:
 * gabp_message_bytes() bytes (prior planes, 5 or 13 for alpha = 4, then the observation
 * messages), host or device, valid only for a context with the same problem and precision.
 */
int64_t gabp_message_bytes(const gabp_ctx *ctx);
int gabp_get_messages(gabp_ctx *ctx, void *buf);
int gabp_set_messages(gabp_ctx *ctx, const void *buf);

/* Statistics of the context (host struct). */
int gabp_get_stats(const gabp_ctx *ctx, gabp_stats *stats);

/* Text of the last error on this context ("" if none); valid until the next call. */
const char *gabp_last_error(const gabp_ctx *ctx);

/* Text of the last error of a gabp_create call that failed on this thread. */
const char *gabp_create_error(void);

/*
 * Mean over the 2 E message components (eta and Lambda of every factor-variable edge) of
 * |m_t - m_{t-1}|: the change made by the last iteration, the quantity of the paper's
 * early-stopping rule (App. B).  GABP_ERR_STATE if no iteration ran since the last
 * initialisation.
 */
int gabp_message_change(gabp_ctx *ctx, double *mean_abs_change);

/*
 * Iterate with the paper's early-stopping rule (App. B): stop after iteration t once
 * mean|m_t - m_{t-1}| < tau * mean|m_2 - m_1|, where m_i is the message set after i iterations
 * of this call (the paper uses tau = 1e-3).  The rule is checked after iteration 2 + j *
 * check_every (check_every = 1: after every iteration, as in the paper).  *stopped_at (may be
 * NULL) receives t.  GABP_ERR_TIMEOUT after max_iters (>= 3) iterations, GABP_ERR_DIVERGED if a
 * change is not finite.
 */
int gabp_iterate_early_stop(gabp_ctx *ctx, int max_iters, double damping, double tau, int check_every,
                            int64_t *stopped_at);

/* Release the context and all its device memory.  NULL is ignored. */
void gabp_destroy(gabp_ctx *ctx);

/* ---------------------------------------------------------------------------------------
 * Batches: many independent problems (ensemble members, successive analysis windows) of
 * uneven sizes iterated together.  Every iteration of the whole batch is ONE persistent
 * kernel launch over the work items of all active problems (FP32 messages), replayed from a
 * CUDA graph; the per-problem residual checks are a second graph.  Two kernels serve batches:
 * the TMA kernel over 30 x 14, 30 x 22 or 30 x 30 tiles (tensor copies of every problem's tiles:
 * the message planes of a problem of odd width are stored with rows padded to an even pitch,
 * its observation index in a copy with rows padded to a multiple of 4) and the column-sweep
 * kernel over strips of 16, 32, 64 or 128 rows.  The autotuner times every candidate on this batch at create time
 * and keeps the fastest (cached per device and batch shape in the file named by
 * GABP_AUTOTUNE_CACHE, if set).  Messages are bit-identical to single-problem contexts
 * whichever kernel runs.
 * --------------------------------------------------------------------------------------- */
typedef struct gabp_batch gabp_batch;   /* opaque; owns the device memory of all its problems */

typedef struct {
    gabp_grid grid;             /* as for gabp_create */
    double kappa;               /* > 0 */
    double gamma;               /* > 0 (prior scale); 0 means 1 */
    int64_t m;                  /* observations, >= 0 */
    const double *obs_xy;       /* 2m doubles, HOST */
    const double *y;            /* m doubles, HOST */
    const double *noise_var;    /* m doubles, HOST */
} gabp_problem;

/*
 * Create a batch of `count` problems (each built as in gabp_create: Sec. 3.1 and Sec. 3.2).
 * opt: NULL = defaults; precision must be GABP_FP32; opt->kernel GABP_KERNEL_AUTO (the
 * autotuner's choice among both kernels), GABP_KERNEL_TMA or GABP_KERNEL_SWEEP (the
 * autotuner's choice among that kernel's shapes; others: GABP_ERR_ARG); opt->tile_y, if
 * non-zero, fixes the configuration instead of the autotuner: 14, 22 or 30 = the TMA kernel's tile
 * height, 16, 32, 64 or 128 = the sweep kernel's strip height; tol, check_every (rounded up
 * to even), max_iters, device and stream apply
 * to the whole batch.  Host arrays are read during the call only.  Errors as for gabp_create;
 * the failing problem's index is in the message.
 */
int gabp_batch_create(gabp_batch **out, int count, const gabp_problem *problems, const gabp_options *opt);

/*
 * Iterate every problem of the batch in lockstep (Alg. 2 with damping, as gabp_iterate).
 *   n_iters >= 0: exactly n_iters iterations of every problem.
 *   n_iters <  0: iterate until every problem's relative residual is <= opt.tol; a problem that
 *                 reaches it stops being updated at the next check (every check_every
 *                 iterations).  GABP_ERR_TIMEOUT after max_iters, GABP_ERR_DIVERGED if a
 *                 residual becomes non-finite.
 * GABP_ERR_TIMEOUT also if a bounded wait inside the TMA kernel gave up (reported at the end
 * of the call or at the next residual check; the messages are then unspecified).
 */
int gabp_batch_iterate(gabp_batch *b, int n_iters, double damping);

/* Relative residuals of every problem (count doubles, HOST), computed now in FP64. */
int gabp_batch_residuals(gabp_batch *b, double *rel);

/* Marginals of problem `index` (as gabp_marginals). */
int gabp_batch_marginals(gabp_batch *b, int index, double *mean, double *var);

/* Statistics of problem `index` (iterations it has been updated, last residual, sizes; kernel
 * is GABP_KERNEL_TMA or GABP_KERNEL_SWEEP, tile_x x tile_y its tile or strip shape). */
int gabp_batch_get_stats(const gabp_batch *b, int index, gabp_stats *stats);

/* Tile or strip height in use (chosen by the autotuner or opt.tile_y): 14, 22 or 30 for the TMA
 * kernel, 16, 32, 64 or 128 for the sweep kernel. */
int gabp_batch_strip_height(const gabp_batch *b);

const char *gabp_batch_last_error(const gabp_batch *b);
void gabp_batch_destroy(gabp_batch *b);

/* ---------------------------------------------------------------------------------------
 * Multigrid warm start (Sec. 3.2 "Multigrid"; Alg. 2 "Multigrid MP" and "Upscale Messages").
 * Level k = 1 .. levels-1 is the context's problem on a grid of spacing 2^k target cells:
 * ceil(nx / 2^k) x ceil(ny / 2^k) nodes, kappa_k = 2^k kappa and gamma_k = gamma / 4^k (the
 * same SPDE discretised at that spacing), every observation at (x / 2^k, y / 2^k) clamped to
 * the level's last node, with its own value and noise variance.  From the coarsest level
 * (cold start) up, each level runs GaBP; every node of the next finer level then takes the
 * marginal (mean, precision) of its parent node (floor(i/2), floor(j/2)) and its messages are
 * set as by gabp_warm_start.  Finally the target context is warm-started from level 1.  A level
 * whose final relative residual is not finite or not below 1 is re-run from the same start
 * with damping (1 + damping) / 2, up to three times; a level that still fails passes its own
 * start on (or a cold start).
 * --------------------------------------------------------------------------------------- */
#define GABP_MG_MAX_LEVELS 16
typedef struct gabp_mg gabp_mg;   /* opaque; owns the coarse levels' contexts */

typedef struct {
    int levels;                                  /* as created */
    int64_t iterations[GABP_MG_MAX_LEVELS];      /* level k at [k] ([0] unused): GaBP iterations, all attempts */
    double damping[GABP_MG_MAX_LEVELS];          /* damping of the level's last attempt */
    double residual[GABP_MG_MAX_LEVELS];         /* the level's final relative residual */
    int converged[GABP_MG_MAX_LEVELS];           /* 1 if the level's state was passed on */
} gabp_mg_stats;

/* Build the coarse levels of ctx's problem, 2 <= levels <= GABP_MG_MAX_LEVELS; every coarse level
 * needs at least 2 nodes per axis (GABP_ERR_ARG otherwise).  The coarse contexts use ctx's
 * precision, device and stream.  ctx must outlive the multigrid object.  Errors of this call are
 * reported by gabp_last_error(ctx). */
int gabp_mg_create(gabp_mg **out, gabp_ctx *ctx, int levels);

/* Run the coarse levels and warm-start the target context (its iteration count restarts at 0).
 * tol > 0: each level iterates until its relative residual is <= tol (checked every
 * check_every iterations of ctx's options) or max_iters iterations; tol <= 0: exactly max_iters
 * iterations per level.  damping in [0, 1), max_iters >= 1; stats may be NULL. */
int gabp_mg_warm_start(gabp_mg *mg, double damping, double tol, int max_iters, gabp_mg_stats *stats);
const char *gabp_mg_last_error(const gabp_mg *mg);
void gabp_mg_destroy(gabp_mg *mg);

/* ---------------------------------------------------------------------------------------
 * The paper's own pairwise re-weighted message passing (App. A, "Gaussian Setting" and
 * "Re-weighted message updates"), a second iteration family over the same posterior: one node
 * factor exp(-P_ii f_i^2 / 2 + h_i f_i) per node and one pair factor exp(-P_ij f_i f_j) per
 * nonzero P_ij of P = gamma L^T L + H^T R^-1 H (the 13-point pattern), fractional messages with
 * weight c, damping with the paper's learning rate eta (m <- (1 - eta) m_old + eta m_new; the
 * paper uses c = 10, eta = 0.6).  The factor message follows the integral that defines it.
 * Messages start at zero; the marginal is mean (h_i + c sum b) / (P_ii + c sum a), precision
 * P_ii + c sum a (with the c of the last gabp_pw_iterate call).
 * --------------------------------------------------------------------------------------- */
typedef struct gabp_pw gabp_pw;   /* opaque; owns its coefficient and message buffers */

/* The pairwise form of ctx's problem (ctx's precision, device and stream; ctx must outlive it).
 * Errors are reported by gabp_last_error(ctx). */
int gabp_pw_create(gabp_pw **out, gabp_ctx *ctx);
/* n_iters synchronous iterations with weight c (finite, nonzero) and learning_rate in (0, 1]. */
int gabp_pw_iterate(gabp_pw *pw, int n_iters, double c, double learning_rate);
/* Marginal means and variances (n doubles each, host or device; var may be NULL). */
int gabp_pw_marginals(gabp_pw *pw, double *mean, double *var);
/* Relative residual ||b - A mu|| / ||b|| of the current means (as gabp_residual). */
int gabp_pw_residual(gabp_pw *pw, double *rel_residual);
int gabp_pw_reset(gabp_pw *pw);
int64_t gabp_pw_iterations(const gabp_pw *pw);
/* Alg. 2 around the pairwise form (Sec. 3.2 "Multigrid", App. B "Early Stop"):
 * gabp_pw_message_change: mean |m_t - m_{t-1}| over both components (a, b) of every directed
 *   pair-factor message (pairs within the 13-point pattern); GABP_ERR_STATE before the first
 *   iteration after a reset.
 * gabp_pw_iterate_early_stop: iterate under the early-stopping rule: after iterations 1 and 2 of
 *   the call the change is the reference; stop after the first t >= 3 whose change is below
 *   tau times it (*stopped_at = t).  GABP_ERR_TIMEOUT after max_iters (>= 3), GABP_ERR_DIVERGED
 *   if a change is not finite.
 * gabp_pw_iterate_early_stop_ref: the same rule with the reference given: reference > 0 is
 *   compared against instead of this call's own change between its iterations 1 and 2 (App. B
 *   names m_1 and m_2 without a level; a multigrid driver can pass every level the coarsest
 *   level's change); reference <= 0 is gabp_pw_iterate_early_stop.  *reference_used (may be
 *   NULL) receives the reference the rule compared against.
 * gabp_pw_upscale: "Upscale Messages": fine's messages = coarse's current messages on the same
 *   directions, node (i, j) of fine taking those of (floor(i/2), floor(j/2)) of coarse (clamped
 *   to its grid), (0, 0) where either level lacks the pair; same precision and device;
 *   resets fine's iteration count. */
int gabp_pw_message_change(gabp_pw *pw, double *mean_abs_change);
int gabp_pw_iterate_early_stop(gabp_pw *pw, int max_iters, double c, double learning_rate, double tau,
                               int64_t *stopped_at);
int gabp_pw_iterate_early_stop_ref(gabp_pw *pw, int max_iters, double c, double learning_rate, double tau,
                                   double reference, int64_t *stopped_at, double *reference_used);
int gabp_pw_upscale(gabp_pw *fine, const gabp_pw *coarse);
const char *gabp_pw_last_error(const gabp_pw *pw);
void gabp_pw_destroy(gabp_pw *pw);

/* ---------------------------------------------------------------------------------------
 * Learned warm start.  A small convolutional encoder-decoder (4 levels, 32 -> 256 channels,
 * BF16 weights and activations, FP32 accumulation) maps the gridded observations to initial
 * beliefs (mean, log precision); gabp_wsnet_warm_start() seeds a context's messages with them
 * (as gabp_warm_start).  The paper has no learned component; its own accelerator of
 * convergence is the multigrid warm start (Sec. 3.2 "Multigrid", App. B "Upscale Messages").
 * Network input per node (grid padded to multiples of 8): the mean of y / scale over the
 * observations whose nearest node it is, that mask, log(kappa) + 3 (13 zero channels follow);
 * scale = standard deviation of the problem's observed values.  Output: mean / scale, log
 * precision.
 * --------------------------------------------------------------------------------------- */
typedef struct gabp_wsnet gabp_wsnet;

/* Create a network with seeded He-normal weights on `device` (-1 = current). */
int gabp_wsnet_create(gabp_wsnet **out, uint64_t seed, int device);
int64_t gabp_wsnet_param_count(const gabp_wsnet *net);
/* FP32 parameter vector (host or device, gabp_wsnet_param_count floats). */
int gabp_wsnet_get_params(gabp_wsnet *net, float *params);
int gabp_wsnet_set_params(gabp_wsnet *net, const float *params);
/* Kernel family of the forward pass: GABP_WSNET_TCGEN05 (default) runs every convolution on the
 * tcgen05 tensor cores (TMA-fed implicit GEMM, accumulators in tensor memory) with pooling,
 * upsampling additions and the head fused into the convolutions; GABP_WSNET_MMA_SYNC runs the
 * mma.sync kernels that the backward pass uses.  Both compute the same network in BF16 with FP32
 * accumulation (results differ by rounding order only).  GABP_ERR_ARG for another value. */
#define GABP_WSNET_TCGEN05 0
#define GABP_WSNET_MMA_SYNC 1
int gabp_wsnet_set_kernels(gabp_wsnet *net, int kernels);
/* Forward pass: x [B][H][W][16] BF16, out [B][H][W][2] FP32 (host or device); H, W multiples of 8. */
int gabp_wsnet_forward(gabp_wsnet *net, const void *x, int B, int H, int W, float *out);
/* Loss (mean over pixels of the squared errors of both outputs) and its gradient w.r.t. every
 * parameter (FP32, host or device; NULL = do not copy) for B samples given as device pointers
 * to [H][W][16] BF16 inputs and [H][W][2] FP32 targets. */
int gabp_wsnet_gradients(gabp_wsnet *net, const void *const *xs, const float *const *ts, int B, int H, int W,
                         float *grads, float *loss);
/* One Adam step (beta 0.9 / 0.999) on B samples; loss before the step into *loss. */
int gabp_wsnet_train_step(gabp_wsnet *net, const void *const *xs, const float *const *ts, int B, int H, int W,
                          float lr, float *loss);
const char *gabp_wsnet_last_error(const gabp_wsnet *net);
const char *gabp_wsnet_create_error(void);
void gabp_wsnet_destroy(gabp_wsnet *net);

/* Padded network grid of a context (H, W multiples of 8) and its input scale. */
int gabp_wsnet_input_shape(const gabp_ctx *ctx, int *H, int *W, double *scale);
/* A training sample of a context: network input (DEVICE, [H][W][16] BF16, may be NULL) and target
 * from its current beliefs (DEVICE, [H][W][2] FP32: mean / scale, log precision; may be NULL). */
int gabp_wsnet_sample(gabp_ctx *ctx, void *x_out, float *t_out);
int gabp_batch_input_shape(const gabp_batch *b, int index, int *H, int *W, double *scale);
int gabp_batch_wsnet_sample(gabp_batch *b, int index, void *x_out, float *t_out);
/* Scatter the observations, run the network and seed the messages from its prediction
 * (all on the GPU, on the context's stream). */
int gabp_wsnet_warm_start(gabp_ctx *ctx, gabp_wsnet *net);

/*
 * Allocation-free residual.  The paper has no counterpart: this entry point exists for callers
 * that cannot allocate device memory through this library, e.g. a process whose device memory
 * is held by another allocator (a framework's caching allocator keeps freed blocks, so a plain
 * cudaMalloc can fail while that allocator still has room), or a loop with a fixed memory
 * budget.  It computes the same FP64 relative residual ||b - A mu|| / ||b|| as
 * gabp_residual(), for a mean the caller supplies, using only memory the caller passes in plus
 * a static scratch array inside the library.  It calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *
 *   grid, kappa, gamma  as for gabp_create (gamma > 0; zero-Neumann boundary).
 *   m                   number of observations, >= 0.
 *   obs_xy, y, noise_var  DEVICE arrays (2m, m, m doubles) of the current device, with the
 *                       observations SORTED by base cell (i0 * nx + j0 non-decreasing, base
 *                       cell as defined for gabp_create); GABP_ERR_ARG if they are not, or if an
 *                       observation lies outside the grid or has a variance <= 0 (that reason
 *                       is reported when both occur).
 *   mean                DEVICE array of nx*ny doubles (the field mu).
 *   Pointers that are not device (or managed) memory of the current device are GABP_ERR_ARG
 *   (checked with cudaPointerGetAttributes, which allocates nothing).  The sizes cannot be
 *   checked through a pointer: arrays shorter than stated make the kernels read past them.
 *   rel_residual        HOST pointer to one double, written on success.  If ||b|| = 0 the
 *                       absolute norm ||A mu|| is returned instead.
 *   stream              cudaStream_t to run on (NULL = the legacy default stream); the call
 *                       synchronises that stream before returning.
 *
 * Scratch: a file-scope device array of GABP_NOALLOC_MAX_DOUBLES doubles (24 MiB) that every
 * GPU loading the library holds until the process exits; nx*ny + m must not exceed
 * GABP_NOALLOC_MAX_DOUBLES - 2052 (GABP_ERR_ARG otherwise, before any GPU work).  Every call
 * shares the array and it keeps the last call's contents (the call clears what must start at
 * zero), so calls that overlap on the GPU (from two streams or two host threads) race and
 * must be serialised by the caller.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress, with that device current); make that first call before any
 * stream capture.  The text of the last error on the calling thread is returned by
 * gabp_residual_noalloc_error().
 */
#define GABP_NOALLOC_MAX_DOUBLES (3 * 1024 * 1024)
int gabp_residual_noalloc(gabp_grid grid, double kappa, double gamma, int64_t m, const double *obs_xy,
                          const double *y, const double *noise_var, const double *mean,
                          double *rel_residual, void *stream);
const char *gabp_residual_noalloc_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GABP_H */
