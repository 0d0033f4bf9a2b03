/*
 * f3r.h -- C ABI of libf3r.so, a GB300 (sm_103a) implementation of the F3R
 * nested Krylov solver for sparse A x = b from "A Nested Krylov Method Using
 * Half-Precision Arithmetic" (arXiv 2505.20719).
 *
 * F3R = (F_{m1}, F_{m2}, F_{m3}, R_{m4}, M): an fp64 flexible GMRES whose
 * preconditioner is an fp32 FGMRES, preconditioned by an FGMRES with fp16 A
 * and fp32 vectors, preconditioned by an fp16 Richardson iteration with
 * adaptive weights, preconditioned by the primary preconditioner M
 * (Sec. 3 tuple notation; Sec. 4.2; Table 1; Algorithm 1; Eqs. 4-5).
 *
 * Conventions for every entry point:
 *  - Pointers may be host memory (pageable or pinned) or device memory of
 *    the current device; the library tells them apart with
 *    cudaPointerGetAttributes and copies host data itself.  The caller owns
 *    every pointer it passes; setup copies what it keeps.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  All device work of a call is ordered on that stream.
 *  - Indices are 0-based int32 (Sec. 5: 32-bit column indices and row
 *    pointers); rowptr has n+1 monotone entries, 0 <= colidx < n.
 *  - Errors are returned as f3r_status; nothing aborts the process and no
 *    kernel traps.  After F3R_ERR_CUDA the context should be destroyed.
 *  - One context is used by one host thread at a time.  There is no CPU
 *    fallback: without a usable GPU every call returns F3R_ERR_CUDA.
 *
 * Precision codes (Table 1): 0 = fp64, 1 = fp32, 2 = fp16 (binary16),
 * 3 = bf16 (bfloat16, with power-of-two per-row scaling of A).
 */
#ifndef F3R_H
#define F3R_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct f3r_ctx f3r_ctx;

typedef enum {
    F3R_OK = 0,
    F3R_ERR_ARG = 1,          /* invalid argument or matrix (bad rowptr/colidx, n <= 0, ...) */
    F3R_ERR_CUDA = 2,         /* a CUDA call failed or no device is usable */
    F3R_ERR_NOMEM = 3,        /* device or pinned host allocation failed */
    F3R_NOT_CONVERGED = 4,    /* max_outer reached; x holds the last iterate */
    F3R_ERR_BREAKDOWN = 5,    /* reserved */
    F3R_ERR_NONFINITE = 6,    /* a non-finite value reached the outer fp64 level */
    F3R_ERR_TIMEOUT = 7,      /* a bounded device-side wait gave up */
    F3R_ERR_UNSUPPORTED = 8   /* parameter combination not built */
} f3r_status;

enum { F3R_F64 = 0, F3R_F32 = 1, F3R_F16 = 2, F3R_BF16 = 3 };
enum { F3R_PC_IDENTITY = 0, F3R_PC_JACOBI = 1, F3R_PC_LEARNED = 2, F3R_PC_AINV = 3 };

/* Solver configuration.  f3r_default_params gives F3R with the paper's
 * defaults: (m1, m2, m3, m4) = (100, 8, 4, 2), c = 64, Table 1 precisions,
 * Jacobi M, CGS2, tolerance 1e-9, 300 outer iterations at most. */
typedef struct {
    int nlevels;        /* FGMRES levels 1..4; level 0 is the outer fp64 FGMRES on the original A */
    int m[4];           /* iterations per FGMRES level; m[0] is the restart length m1 (<= 128),
                           inner levels <= 15 */
    int a_prec[4];      /* precision of A used by each level; a_prec[0] must be F3R_F64 */
    int v_prec[4];      /* vector precision per level: F3R_F64 or F3R_F32 (v_prec[0] = F3R_F64);
                           F3R_F16 / F3R_BF16 at the innermost FGMRES level when it applies M
                           (rich_m = 0; Table 4's fp16 levels): fp32 arithmetic and fp32 arrays
                           whose stored V and Z values are rounded to that format, so the
                           level's f3r_apply / f3r_get_basis vectors are float */
    int rich_m;         /* Richardson iterations m4 (0 = the innermost FGMRES applies M), <= 8 */
    int rich_a_prec;    /* precision of A inside Richardson */
    int rich_v_prec;    /* precision of Richardson vectors: F16, BF16, F32 or F64 */
    int m_prec;         /* storage precision of M */
    int precond;        /* F3R_PC_JACOBI (M = diag(A^)^-1), F3R_PC_IDENTITY, F3R_PC_LEARNED
                           (the learned net as M inside an fp16 Richardson level; Jacobi
                           until f3r_learned_load is called), or F3R_PC_AINV: the
                           two-SpMV approximate inverse
                             M = (I - Dt^-1 U) Dt^-1 (I - L Dt^-1),  Dt = ainv_alpha diag(A^),
                           L / U the strict triangles of A^, factors stored in fp16
                           (fp16 Richardson level, no row scaling) */
    int c;              /* weight-update period of Algorithm 1 (>= 1) */
    double omega_fixed; /* > 0: fixed Richardson weight, no adaptive update */
    int diag_scale;     /* 1: inner nest works on A^ = D^-1/2 A D^-1/2, D = |diag A| (Sec. 5) */
    int row_scale;      /* 1: power-of-two row scaling of 16-bit copies of A */
    int scale_cast;     /* 1: power-of-two scaling of vectors cast into 16-bit storage */
    int cgs_passes;     /* 1 = classical Gram-Schmidt (Sec. 4.2), 2 = CGS2 */
    double tol;         /* target ||b - A x||_2 / ||b||_2 */
    int max_outer;      /* total outer iterations before F3R_NOT_CONVERGED (Sec. 5: 300) */
    int use_graphs;     /* 1: replay each outer iteration as one CUDA graph */
    int keep_omega;     /* 1: keep the Richardson weights and counter of the previous solve */
    int fuse_cgs;       /* 1: second CGS pass, norm, Givens step and normalisation of an inner
                           iteration in one cooperative launch (when a block's rows fit in
                           shared memory); 0: three launches.  Same arithmetic per row; only
                           the summation order of the dot products differs. */
    float inner_rtol;   /* > 0: the innermost FGMRES level (F_m3 in F3R) stops once its
                           residual estimate |g_{j+1}| <= inner_rtol * beta (adaptive m3,
                           Sec. 6 / Sec. 7; the Richardson weight counter still counts the
                           scheduled calls); 0: always m iterations */
    float ainv_alpha;   /* diagonal boost of the approximate inverse (> 0; default 1) */
    int fuse_step;      /* 1 (with fuse_cgs): a plain iteration of the innermost FGMRES level
                           (Richardson call, SpMV + dots, CGS2, normalisation) in one
                           cooperative launch when the default precision schedule, Jacobi M
                           and m4 = 2 apply; 0 (default): separate launches, which measured
                           as fast inside CUDA graphs with more blocks per SM */
    int batch_split;    /* f3r_setup_batched only: systems of at least this many rows are large
                           (see batch_wide); 0 (default): 2048 rows per SM of the device; < 0: no
                           system is large */
    int batch_wide;     /* f3r_setup_batched only: the large systems' instances run in the same
                           persistent launch, each on a wide team of this many thread-block
                           clusters (0, default: an eighth of the launch's clusters, at least 2);
                           < 0: they are solved one after another by the single-system path
                           (the whole GPU each) before the launch */
    int reserved;
} f3r_params;

typedef struct {
    int status;            /* f3r_status of the solve */
    int outer_iters;       /* outer (F_{m1}) iterations over all restarts */
    int restarts;          /* number of restarts of the whole nest */
    double rel_res_true;   /* final fp64 ||b - A x|| / ||b|| */
    int64_t m_applies;     /* applications of M (Sec. 4.2: 64 per outer iteration) */
    int64_t r_calls;       /* Richardson calls */
    int64_t r_update_calls;/* Richardson calls that computed w' (every c-th) */
    double omega[8];       /* Richardson weights at exit */
    double *hist;          /* caller-owned host array: |g_{j+1}|/||b|| per outer iteration */
    int hist_cap;
    int hist_len;
    double *true_hist;     /* caller-owned host array: true residual at each cycle start and exit */
    int true_cap;
    int true_len;
    double t_solve_ms;     /* device time of the solve (CUDA events) */
    int64_t kernel_launches; /* kernels launched by the solve (graph nodes included) */
    int64_t graph_launches;
} f3r_stats;

/* Fill *p with the paper's F3R defaults (Sec. 4.2, Sec. 5, Table 1). */
f3r_status f3r_default_params(f3r_params *p);

/* Build a solver for the n x n CSR matrix (rowptr, colidx, val; host or
 * device pointers, fp64 values): validates the matrix, applies the diagonal
 * scaling of Sec. 5, converts A to sliced ELLPACK with slices of 32 rows
 * (Sec. 5.2) and stores the fp64 / fp32 / fp16 / bf16 copies the levels use
 * (Table 1), allocates all workspace.  *ctx is written on success.
 * Errors: F3R_ERR_ARG (bad matrix or parameters), F3R_ERR_NOMEM, F3R_ERR_CUDA. */
f3r_status f3r_setup(f3r_ctx **ctx, int32_t n, int64_t nnz, const int32_t *rowptr,
                     const int32_t *colidx, const double *val, const f3r_params *params,
                     void *stream);

/* Solve A x = b (b, x: n fp64 values, host or device).  x holds the initial
 * guess on entry (Sec. 5 uses x0 = 0) and the solution on exit.  Returns
 * F3R_OK when ||b - A x|| / ||b|| < tol, F3R_NOT_CONVERGED after max_outer
 * outer iterations (x = last iterate), F3R_ERR_NONFINITE if a non-finite
 * value reaches the outer level.  `stats` may be NULL.  Synchronises the
 * stream once per outer iteration to read the convergence estimate. */
f3r_status f3r_solve(f3r_ctx *ctx, const double *b, double *x, f3r_stats *stats, void *stream);

/* y = A_p x with A_p the precision-p copy of the scaled matrix (p = 0
 * returns the original fp64 A).  x and y are device pointers of vector
 * precision vp: fp64 for p = 0, else vp = F3R_F32 (y fp32, row sums in
 * fp32) or vp = F3R_F16 / F3R_BF16 (x 16-bit, y fp32).  Row sums use
 * fused multiply-add in CSR order.  Errors: F3R_ERR_ARG if the context
 * holds no copy in precision p. */
f3r_status f3r_spmv(f3r_ctx *ctx, int p, int vp, const void *x, void *y, void *stream);

/* One preconditioner application at nesting depth `level` with the current
 * Richardson state (test and instrumentation entry):
 *   1 <= level < nlevels : one call of inner FGMRES level `level`, x and z in
 *                          that level's vector precision;
 *   level == nlevels     : one Richardson call (Algorithm 1), or M if
 *                          rich_m = 0; x and z in the vector precision of
 *                          level nlevels-1.
 * x and z are device pointers of n elements. */
f3r_status f3r_apply(f3r_ctx *ctx, int level, const void *x, void *z, void *stream);

/* Copy basis vector V[k] (0 <= k <= m of that level; an inner level, which
 * ends at its m-th Givens step, never forms V[m]) of FGMRES level `level`
 * as the context's last call left it -- for level 0 the last restart cycle of
 * the last f3r_solve: the normalised residual (k = 0) and the Arnoldi vectors
 * of the outer fp64 FGMRES (Sec. 4.2) -- into `out` (n elements in the
 * level's vector precision; host or device memory).  Used to build training
 * pairs for the learned preconditioner from the solver's own vectors. */
f3r_status f3r_get_basis(f3r_ctx *ctx, int level, int k, void *out, void *stream);

/* Read / write the Richardson state (omega[0..m4-1], call counter c_ntr). */
f3r_status f3r_get_rich_state(f3r_ctx *ctx, double *omega8, int64_t *c_ntr);
f3r_status f3r_set_rich_state(f3r_ctx *ctx, const double *omega8, int64_t c_ntr);

/* Copy a set-up array back to host memory `out` in CSR order (test entry):
 * 0 d = D^-1/2 (double, n); 1 A^ fp64 (nnz); 2 A^ fp32 (float, nnz);
 * 3 A^/s fp16 (uint16 bits, nnz); 4 A^/s bf16 (uint16 bits, nnz);
 * 5 row scales (float, n); 6 M in m_prec (n elements of that precision);
 * approximate inverse (F3R_PC_AINV), fp16 bits: 7 L Dt^-1 (nnz, zero off the
 * strict lower triangle), 8 Dt^-1 U (nnz, zero off the strict upper
 * triangle), 9 Dt^-1 (n); 10 (windowed matrices, see f3r_matrix_info) the
 * column each entry's 16-bit window index stands for (int32, nnz: equal to
 * colidx when the set-up is right).
 * Returns F3R_ERR_ARG if the array does not exist. */
f3r_status f3r_export(f3r_ctx *ctx, int which, void *out);

/* Round n fp32 values x to prec (F3R_F16 or F3R_BF16) with the conversion
 * every kernel of this library applies when it stores a 16-bit value (round
 * to nearest, ties to even, subnormals kept, overflow to infinity; Table 1's
 * fp16 storage, and bf16 in its place), writing the 16-bit patterns to out
 * (test entry: it lets a test compare the device conversion with an
 * independent definition over every fp32 bit pattern).  x and out are device
 * pointers, asynchronous on stream.  Errors: F3R_ERR_ARG (prec, n < 0, null
 * pointers), F3R_ERR_CUDA. */
f3r_status f3r_round16(int prec, const float *x, uint16_t *out, int64_t n, void *stream);

/* Storage of the set-up matrix (instrumentation), out[8]:
 *   [0] 1 if the matrix is windowed (below), [1] largest window of a tile
 *   (entries), [2] stored SELL entries (padding included), [3] widest slice,
 *   [4] slices of 32 rows, [5] bytes per stored column index (2 windowed,
 *   4 otherwise), [6] window chunk (entries), [7] 1 if every entry of M is 1.
 * Windowed: the columns of every 256-row tile lie in at most 14 runs of x
 * (4096 entries in all) that the kernels bulk-copy into shared memory with
 * the tile's SELL slices (Sec. 5.2), and each entry stores a 16-bit index
 * into that window instead of an int32 column.  Set up for every matrix
 * whose tiles fit (banded and stencil matrices); otherwise the kernels
 * gather x by int32 column from global memory.  Same results either way. */
f3r_status f3r_matrix_info(f3r_ctx *ctx, int64_t *out);

/* Kernel event profiler (instrumentation).  With enable = 1 the totals are
 * reset, every kernel the context launches is bracketed by two CUDA events
 * on its launching stream, and solves run without graph replay.  Slot s
 * aggregates one kernel kind at one nesting level: kind = s / 4, level =
 * s % 4; f3r_profile_slot_name(s) names the kind.  f3r_profile_get returns
 * the number of timed launches and their summed device time (ms). */
f3r_status f3r_profile_enable(f3r_ctx *ctx, int enable);
f3r_status f3r_profile_get(f3r_ctx *ctx, int slot, int64_t *launches, double *total_ms);
int f3r_profile_slots(void);
const char *f3r_profile_slot_name(int slot);

/* ------------------------------------------------------------ learned M
 * Learned preconditioner M_theta (project addition; the paper's M is an
 * algebraic preconditioner, Sec. 3): a 3-layer message-passing network of
 * width 32 over the graph of A^ (fp16 copy), bf16 weights, activations and
 * messages, fp32 accumulation (mma.sync bf16 tensor-core products), with the
 * s-normalisation that makes it homogeneous for powers of two:
 *   h0 = relu(e r~ + b0), g = offdiag(A^) h, h = relu([h|g][Ws|Wm]^T + b) (x3),
 *   z = s (omega_j r~ + wo . h),  r~ = r / s,  s = 2^ceil(log2 max|r|).
 * Parameters are a flat fp32 vector of F3R_LEARNED_NPARAMS values in the order
 * e[32], b0[32], Ws[3][32][32], Wm[3][32][32], b[3][32], wo[32], omega_j.
 * Training needs a symmetric A^ and a context holding the fp16 copy of A^. */
#define F3R_LEARNED_NPARAMS 6337

/* Load parameters (host or device, fp32) into the context; `train` = 1 also
 * allocates the training buffers (activations of all layers).  With
 * precond = F3R_PC_LEARNED the solver then uses the net as M. */
f3r_status f3r_learned_load(f3r_ctx *ctx, const float *params, int train);
/* Copy the current fp32 parameters to host memory `out` (NPARAMS floats). */
f3r_status f3r_learned_get(f3r_ctx *ctx, float *out);
/* z = M_theta(r), r and z device fp32 vectors of n values. */
f3r_status f3r_learned_apply(f3r_ctx *ctx, const float *r, float *z, void *stream);
/* Training loss: kind 0 (default) ||M_theta(r) - e||^2 / ||e||^2 with
 * e = A^-1 r given; kind 1 ||A16 M_theta(r) - r||^2 / ||r||^2 with A16 the
 * fp16 copy of A^ (no e needed: pass E = NULL).  Needs a loaded net;
 * F3R_ERR_ARG for another kind. */
f3r_status f3r_learned_set_loss(f3r_ctx *ctx, int kind);
/* Mean loss over P samples (kind of f3r_learned_set_loss) and its gradient
 * (R, E device fp32, P x n row-major; E may be NULL for kind 1); loss and
 * grad (NPARAMS) are host outputs, either may be NULL. */
f3r_status f3r_learned_loss_grad(f3r_ctx *ctx, const float *R, const float *E, int P, float *loss, float *grad,
                                 void *stream);
/* Adam training: `steps` steps, each on a mini-batch of `batch` consecutive
 * samples (cycling through the P pairs), learning rate lr; loss_hist (host,
 * optional, `steps` floats) receives each step's mini-batch loss. */
f3r_status f3r_learned_train(f3r_ctx *ctx, const float *R, const float *E, int P, int steps, int batch, float lr,
                             float *loss_hist, void *stream);

/* ------------------------------------------------------ Krylov comparators
 * The paper's comparators (Sec. 5): preconditioned CG (symmetric A) and
 * BiCGStab (any A), fp64 throughout, on the context's original matrix with
 * the preconditioner the F3R nest wraps, P = D^-1/2 M D^-1/2 (M the stored
 * Jacobi preconditioner in m_prec, D = |diag A| with diag_scale, else I).
 * Stops when the recurrence residual falls below params.tol * ||b|| and the
 * true fp64 residual confirms it (else the recurrence restarts from x, at
 * most 3 times), or after max_iters iterations.  b, x: host or device fp64
 * (x = x0 on entry).  stats: outer_iters = iterations, restarts, hist = the
 * recurrence's ||r|| / ||b|| per iteration of the last start, rel_res_true;
 * status F3R_ERR_BREAKDOWN when the method broke down (a zero inner product)
 * before convergence. */
#define F3R_KRYLOV_CG 1
#define F3R_KRYLOV_BICGSTAB 2
f3r_status f3r_solve_krylov(f3r_ctx *ctx, int method, const double *b, double *x, int max_iters,
                            f3r_stats *stats, void *stream);

/* ---------------------------------------------------------------- batched
 * Many systems, each with one or more right-hand sides, solved by F3R
 * (project addition; the paper solves one system at a time).  Each
 * (system, right-hand side) instance of a small system is solved entirely on
 * the device by one thread-block cluster of a single persistent kernel
 * launch with the default F3R precision schedule (Table 1): fp64
 * FGMRES(m1) with its convergence test and restarts, fp32 FGMRES(m2),
 * FGMRES(m3) with fp16 A, fp16 Richardson R_2 with adaptive weights
 * (Algorithm 1), Jacobi M.  Clusters take instances largest-first from an
 * atomic work queue.  An instance of a large system (params.batch_split rows
 * or more) is solved in the same launch by a wide team of several clusters
 * that meet at bounded barriers in global memory (on one cluster it would
 * keep the launch waiting long after the other clusters finished); the wide
 * teams take the large instances first, then their clusters join the queue
 * of the others.  With params.batch_wide < 0 the large systems are set up as
 * single-system contexts instead and solved one after another (the whole GPU
 * each) before the launch.  Every cluster of the launch is resident at once
 * (the grid is the device's cluster occupancy); a wide barrier that waits
 * longer than ~4 s gives up, and the wide instances then report
 * F3R_ERR_TIMEOUT. */
typedef struct f3r_batch f3r_batch;

typedef struct {
    int32_t n;               /* rows */
    int64_t nnz;
    const int32_t *rowptr;   /* CSR, host or device pointers (copied at setup) */
    const int32_t *colidx;
    const double *val;
    int32_t nrhs;            /* right-hand sides of this system (>= 1) */
} f3r_system_desc;

typedef struct {
    int status;              /* f3r_status of this instance */
    int outer_iters;
    int restarts;
    double rel_res_true;     /* final ||b - A x|| / ||b|| */
    int64_t m_applies;
    int64_t r_calls;
    double t_solve_ms;       /* device time of the whole persistent launch, or of the
                                instance's own solve (systems of >= batch_split rows) */
    int system, rhs;         /* which instance */
    int path;                /* 0: the persistent launch, one cluster; 1: the single-system
                                path; 2: the persistent launch, a wide team of clusters */
} f3r_batch_result;

/* Set up all systems (setup of each matrix as in f3r_setup) and the
 * per-instance workspace.  params must keep the default precision schedule
 * (nlevels 3, m4 = 2, fp16 A at level 2 and in R, no row scaling); m1, m2,
 * m3, c, tol, max_outer, cgs_passes, omega_fixed and scale_cast are honoured.
 * Errors: F3R_ERR_ARG, F3R_ERR_UNSUPPORTED, F3R_ERR_NOMEM, F3R_ERR_CUDA. */
f3r_status f3r_setup_batched(f3r_batch **batch, int nsys, const f3r_system_desc *systems,
                             const f3r_params *params, void *stream);

/* Solve every instance: B[q] and X[q] are device pointers (n of system q's
 * system fp64 values) for instance q, instances numbered system by system
 * and right-hand side by right-hand side; X[q] holds x0 on entry.  With
 * batch_wide < 0 the instances of large systems first (f3r_solve each); one
 * persistent kernel launch for all the others, replayed as a CUDA graph (the instances' b and x
 * pointers reach it through a pinned host table that the graph copies to the
 * device; one graph per cluster and block size, captured on first use, so the
 * first call should come before any stream capture of the caller's); res
 * (optional, one entry per instance) receives each instance's result.
 * Returns F3R_OK if every instance converged, else the status of the first
 * instance that did not. */
f3r_status f3r_solve_batched(f3r_batch *batch, const double *const *B, double *const *X, f3r_batch_result *res,
                             void *stream);

/* Thread-block cluster size of the batched launch (1, 2, 4 or 8; default 8). */
f3r_status f3r_batched_set_cluster(f3r_batch *batch, int cluster_size);
/* Team shape of the batched launch: blocks per instance (the cluster size: 1,
 * 2, 4 or 8) and threads per block (256 or 512; default 512). */
f3r_status f3r_batched_set_shape(f3r_batch *batch, int cluster_size, int threads);
/* Autotuner: times one outer iteration of the persistent launch's instances
 * (from x0 = 0) for every team shape (cluster sizes 1, 2, 4, 8 times 256 or
 * 512 threads per block; with large systems and batch_wide = 0 also 2, 4 or
 * 8 clusters per wide team) and keeps the fastest (its cluster size written
 * to *chosen if not NULL; f3r_batched_info and f3r_batched_wide_info give
 * the rest).  B and X as in f3r_solve_batched; X is zero on return. */
f3r_status f3r_batched_autotune(f3r_batch *batch, const double *const *B, double *const *X, int *chosen,
                                void *stream);
int f3r_batched_instances(const f3r_batch *batch);
/* How the batch runs, out[8]: [0] cluster size, [1] threads per block, [2]
 * instances in the persistent launch, [3] instances solved one after another
 * by the single-system path (systems of >= batch_split rows), [4] / [5] their
 * rows in all, [6] blocks of the persistent launch, [7] graph launches so far. */
f3r_status f3r_batched_info(const f3r_batch *batch, int64_t *out);
/* The wide teams of the last persistent launch, out[4]: [0] clusters per wide
 * team, [1] wide teams, [2] instances of large systems in the launch, [3]
 * their rows in all. */
f3r_status f3r_batched_wide_info(const f3r_batch *batch, int64_t *out);
int64_t f3r_batched_device_bytes(const f3r_batch *batch);
void f3r_destroy_batched(f3r_batch *batch);

/* Residual without device allocation (no counterpart in the paper).
 *
 * r = b - A x (fp64 row sums in CSR order with fused multiply-add) and
 * norms[0] = ||r||_2, norms[1] = ||b||_2, for an n x n fp64 CSR matrix.  For
 * callers that may not call cudaMalloc -- code whose device memory belongs
 * to another allocator (a framework's caching pool, a fixed budget set up
 * front) and so cannot let a library allocate -- this entry point needs no
 * context and allocates nothing: every buffer is the caller's (rowptr,
 * colidx, val, b, x, r and norms[2] are device pointers of the current
 * device; r and norms are written).  Its only scratch is a 65,792-byte
 * static device array inside libf3r (per-block partial sums and a ticket),
 * which every GPU that loads the library holds until the process exits.
 *   - n must be 1 .. 4,194,304 (the scratch holds 4096 blocks of 1024
 *     rows); larger n, n <= 0 or a NULL pointer return F3R_ERR_ARG.
 *   - The first call on a device looks up that device's address of the
 *     scratch array (with the device current); make that first call before
 *     any stream capture.  The address is kept per device and CUDA context:
 *     after a cudaDeviceReset the next call looks it up again in the new
 *     context (again before any capture).
 *   - All calls share the one scratch array, which keeps the last call's
 *     contents (each call clears the part that must start at zero), so calls
 *     that overlap on the GPU -- on different streams or host threads -- race
 *     and must be serialised by the caller.
 *   - Work is ordered on `stream`; the call returns after the launch. */
f3r_status f3r_residual_noalloc(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val,
                                const double *b, const double *x, double *r, double *norms, void *stream);

/* Device memory held by the context, in bytes. */
int64_t f3r_device_bytes(const f3r_ctx *ctx);

/* Releases the context (its buffers return to the library's per-device memory
 * pool, which keeps them for later contexts of this process). */
void f3r_destroy(f3r_ctx *ctx);

/* Returns the device memory that the library's pools keep but no context uses
 * to the CUDA driver.  Contexts' own buffers are not touched. */
f3r_status f3r_trim_memory(void);
const char *f3r_status_str(f3r_status s);

#ifdef __cplusplus
}
#endif
#endif /* F3R_H */
