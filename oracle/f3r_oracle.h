/*
 * F3R oracle -- C interface.
 *
 * TEST INFRASTRUCTURE ONLY: a plain, slow CPU restatement of the nested
 * Krylov solver (F_{m1}, F_{m2}, F_{m3}, R_{m4}, M) of "A Nested Krylov Method
 * Using Half-Precision Arithmetic" (Sec. 4.2, Table 1, Algorithm 1, Eqs. 4-5).
 * Only the test suite, the package smoke check and the benchmark's CPU
 * baseline may load it.  It shares no code, header or table with the CUDA
 * library, and the CUDA library never calls it.
 *
 * Every vector crossing this interface is float64; values that a level keeps
 * in a lower precision are passed as float64 copies of those values.
 */
#ifndef F3R_ORACLE_H
#define F3R_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* storage / arithmetic precisions */
enum { ORC_F64 = 0, ORC_F32 = 1, ORC_F16 = 2, ORC_BF16 = 3 };
enum { ORC_PC_IDENTITY = 0, ORC_PC_JACOBI = 1, ORC_PC_AINV = 3 };
enum { ORC_OK = 0, ORC_NOT_CONVERGED = 4, ORC_BREAKDOWN = 5, ORC_NONFINITE = 6, ORC_ERR_ARG = 1 };

typedef struct {
    int nlevels;        /* number of FGMRES levels, 1..4; level 0 is the outer fp64 solver */
    int m[4];           /* iterations of each FGMRES level (m[0] = restart length m1) */
    int a_prec[4];      /* precision of A used by each level (level 0: ORC_F64, original A) */
    int v_prec[4];      /* vector precision of each level: ORC_F64 or ORC_F32; ORC_F16 / ORC_BF16
                           (fp32 arithmetic, stored vectors rounded) at the innermost
                           FGMRES level when it applies M (rich_m = 0) */
    int rich_m;         /* Richardson iterations m4; 0 = no Richardson level */
    int rich_a_prec;    /* precision of A inside Richardson */
    int rich_v_prec;    /* precision of Richardson vectors (F16, BF16, F32, F64) */
    int m_prec;         /* storage precision of the primary preconditioner M */
    int precond;        /* ORC_PC_IDENTITY, ORC_PC_JACOBI or ORC_PC_AINV (needs orc_problem_set_ainv) */
    int c;              /* weight-update period (Algorithm 1) */
    double omega_fixed; /* > 0: fixed Richardson weights, no adaptive update */
    int diag_scale;     /* symmetric diagonal scaling of the inner nest */
    int row_scale;      /* power-of-two per-row scaling of the 16-bit copies of A */
    int scale_cast;     /* power-of-two scaling of vectors cast into 16-bit storage */
    int cgs_passes;     /* 1 = classical Gram-Schmidt, 2 = CGS2 */
    double tol;         /* relative residual target of the outer solver */
    int max_outer;      /* total outer iterations before giving up */
    double inner_rtol;  /* > 0: the innermost FGMRES level stops once its residual estimate
                           |g_{j+1}| <= inner_rtol * beta (adaptive m, Sec. 6 / Sec. 7);
                           0: always m iterations */
} orc_params;

typedef struct {
    double omega[8];    /* Richardson weights omega_1..omega_m4 */
    int64_t c_ntr;      /* Algorithm 1 call counter (1 before the first call) */
} orc_rich_state;

typedef struct {
    int status;
    int outer_iters;
    int restarts;
    double rel_res_true;
    int64_t m_applies;
    int64_t r_calls;
    int64_t r_update_calls;
    double omega[8];
    double *hist;        /* caller-owned: estimated relative residual per outer iteration */
    int hist_cap;
    int hist_len;
    double *true_hist;   /* caller-owned: true relative residual at each cycle start and at exit */
    int true_cap;
    int true_len;
} orc_stats;

/* rounding to binary16 / bfloat16 (round to nearest, ties to even) */
void orc_round(int prec, const double *x, double *y, int64_t n);

/* problem: copies the CSR matrix and derives the scaled / rounded copies */
void *orc_problem_create(int32_t n, const int32_t *rowptr, const int32_t *colidx,
                         const double *val, int diag_scale, int row_scale, int precond);
void orc_problem_destroy(void *p);
/* approximate inverse M = (I - Dt^-1 U) Dt^-1 (I - L Dt^-1) of the scaled
 * matrix A^ = L + D + U, Dt = alpha D: factors L Dt^-1 and Dt^-1 U per CSR
 * entry (zero off their strict triangles) and Dt^-1, exact in fp64; rounded
 * to m_prec when applied.  orc_problem_get which 11, 12, 13 returns them. */
void orc_problem_set_ainv(void *p, double alpha);
/* which: 0 d = D^{-1/2}, 1 scaled A (f64), 2 A f32, 3 A f16 (divided by row scale),
 *        4 A bf16 (divided by row scale), 5 row scale f16, 6 row scale bf16,
 *        7 M f64, 8 M f32, 9 M f16, 10 M bf16 */
int64_t orc_problem_get(void *p, int which, double *out);

void orc_default_params(orc_params *prm);

/* y = A_prec x, x and y in vector precision vprec (row sums in CSR order with fma) */
void orc_spmv(void *p, int a_prec, int v_prec, const double *x, double *y);
/* y = original A x in f64 */
void orc_spmv_orig(void *p, const double *x, double *y);

/* One application of the preconditioner at nesting depth `level`:
 *   level = nlevels: one Richardson call (Algorithm 1) on input v (the parent's
 *                    vector type), or M if rich_m = 0;
 *   1 <= level < nlevels: one call of inner FGMRES level `level`.
 * The Richardson state is read and updated in place. */
void orc_apply(void *p, const orc_params *prm, orc_rich_state *st, int level,
               const double *v, double *z);

/* Full solve; x holds x0 on entry. */
int orc_solve(void *p, const orc_params *prm, const double *b, double *x, orc_stats *stats);

/* Plain FGMRES(m) level-0 instrumentation: runs one outer cycle of `steps`
 * iterations from x0 = 0 and returns V (n x (steps+1)), Z (n x steps) and the
 * Hessenberg matrix H ((steps+1) x steps, before rotation), column-major. */
int orc_outer_arnoldi(void *p, const orc_params *prm, const double *b, int steps,
                      double *V, double *Z, double *H);

/* One call of inner FGMRES level `level` (1 <= level < nlevels) on input v
 * (the parent's vector type), recording that call's basis V (n x (m+1)),
 * preconditioned vectors Z (n x m), Hessenberg matrix H before rotation
 * ((m+1) x m, column-major) and rotated right-hand side g (m+1), all as
 * float64 copies of the level's values; z receives the level's output.
 * Returns the number of columns kept (k <= m), or -1 if nothing ran. */
int orc_inner_arnoldi(void *p, const orc_params *prm, orc_rich_state *st, int level,
                      const double *v, double *z, double *V, double *Z, double *H, double *g);

int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
