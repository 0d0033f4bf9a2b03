/*
 * F3R oracle: a plain, slow CPU restatement of the nested Krylov solver of
 * "A Nested Krylov Method Using Half-Precision Arithmetic".
 *
 * TEST INFRASTRUCTURE ONLY -- used by the test suite, the package smoke check
 * and the benchmark's CPU-baseline leg, never by the CUDA library.  It shares
 * no code with the CUDA path.
 *
 * What it follows:
 *   Sec. 3          tuple notation: each level preconditions its parent.
 *   Sec. 4.2        F3R = (F_{m1}, F_{m2}, F_{m3}, R_{m4}, M), defaults
 *                   (100, 8, 4, 2); convergence checked only in the outermost
 *                   level; the whole nest is re-run ("restarted") when m1
 *                   outer iterations are not enough.
 *   Table 1         precisions: F_{m1} fp64 A and vectors; F_{m2} fp32 A and
 *                   vectors; F_{m3} fp16 A with fp32 vectors (SpMV computed in
 *                   fp32, the higher of the two input precisions); R_{m4} fp16
 *                   A, vectors and M.
 *   Sec. 4.2        classical Gram-Schmidt Arnoldi and Givens-rotation QR in
 *                   the level's vector precision (CGS2 = two CGS passes).
 *   Algorithm 1,    Richardson z_k = z_{k-1} + w_k M (v - A z_{k-1}), z_0 = 0,
 *   Eqs. 4-5        with the locally optimal weight (r, AMr)/(AMr, AMr) used on
 *                   every c-th call and folded into the cumulative average
 *                   w_k := (l w_k + w'_k)/(l+1), l = c_ntr / c; w'_k computed
 *                   in fp32.
 *   Sec. 5          x0 = 0, stop at ||b - Ax||/||b|| < tol, give up after 300
 *                   outer iterations; diagonal scaling of the matrix.
 *
 * Rounding model (the readings are listed with the design notes): every
 * stored low-precision value is rounded to nearest-even when stored; fp32
 * arithmetic is C float arithmetic (one rounding per operation); row sums of
 * SpMV and dot products accumulate sequentially in index order with fused
 * multiply-add, in the level's arithmetic precision.
 *
 * Build: g++ -std=c++17 -O2 -ffp-contract=off -fopenmp -shared -fPIC.
 * -ffp-contract=off keeps the compiler from fusing multiplies and adds that
 * the code writes separately; every fused multiply-add here is an explicit
 * std::fma / std::fmaf.
 */
#include "f3r_oracle.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

/* ------------------------------------------------------------------ rounding
 * Round x to a binary format with p significand bits (implicit bit included),
 * smallest normal exponent emin and largest finite value maxv, with
 * round-to-nearest ties-to-even (IEEE 754 roundTiesToEven).  In the binade
 * [2^e, 2^(e+1)) the spacing of representable numbers is 2^(e-p+1); below
 * 2^emin it stays 2^(emin-p+1) (gradual underflow).  x / spacing is exact in
 * double, nearbyint() rounds it to an integer in the default (ties-to-even)
 * mode, and a result above maxv overflows to infinity. */
double round_format(double x, int p, int emin, double maxv) {
    if (std::isnan(x) || std::isinf(x) || x == 0.0) return x;
    double a = std::fabs(x);
    int e;
    std::frexp(a, &e);  // a = f * 2^e with f in [0.5, 1): binade exponent is e-1
    int eb = std::max(e - 1, emin);
    double spacing = std::ldexp(1.0, eb - (p - 1));
    double q = std::nearbyint(a / spacing);
    double r = q * spacing;
    if (r > maxv) r = INFINITY;
    return std::copysign(r, x);
}
const double kMaxF16 = 65504.0;
const double kMaxBF16 = 3.3895313892515355e38;  // (2 - 2^-7) * 2^127
inline double rnd16(double x) { return round_format(x, 11, -14, kMaxF16); }
inline double rndbf16(double x) { return round_format(x, 8, -126, kMaxBF16); }
inline double rnd_prec(int prec, double x) {
    switch (prec) {
        case ORC_F64: return x;
        case ORC_F32: return (double)(float)x;  // C conversion rounds to nearest even
        case ORC_F16: return rnd16(x);
        default: return rndbf16(x);
    }
}

inline float fma_t(float a, float b, float c) { return std::fmaf(a, b, c); }
inline double fma_t(double a, double b, double c) { return std::fma(a, b, c); }

#define OMP_FOR _Pragma("omp parallel for schedule(static) if (n > 32768)")

/* --------------------------------------------------------------- the problem */
struct Problem {
    int n = 0;
    std::vector<int32_t> rp, ci;
    std::vector<double> a;         // original A (fp64), used by the outer level
    std::vector<double> d;         // D^{-1/2}, D = |diag A| (ones without scaling)
    std::vector<double> ah;        // scaled A^ = D^{-1/2} A D^{-1/2} in fp64
    std::vector<double> a32;       // A^ rounded to fp32
    std::vector<double> a16, abf;  // A^_ij / s_i rounded to fp16 / bf16
    std::vector<double> rs16, rsbf;// s_i (powers of two; ones without row scaling)
    std::vector<double> m64, m32, m16, mbf;  // M = diag(A^)^{-1} in each precision
    std::vector<double> ainv_l, ainv_u, ainv_dinv;  // approximate-inverse factors (fp64)
    int diag_scale = 1, row_scale = 0, precond = ORC_PC_JACOBI;
};

const std::vector<double> &vals_for(const Problem &P, int prec) {
    switch (prec) {
        case ORC_F64: return P.ah;
        case ORC_F32: return P.a32;
        case ORC_F16: return P.a16;
        default: return P.abf;
    }
}
const std::vector<double> *rowscale_for(const Problem &P, int prec) {
    if (prec == ORC_F16) return &P.rs16;
    if (prec == ORC_BF16) return &P.rsbf;
    return nullptr;
}
const std::vector<double> &m_for(const Problem &P, int prec) {
    switch (prec) {
        case ORC_F64: return P.m64;
        case ORC_F32: return P.m32;
        case ORC_F16: return P.m16;
        default: return P.mbf;
    }
}

/* s_i = 2^ceil(log2 max_j |A^_ij|) (1 for an empty or all-zero row) */
double row_scale_of(const Problem &P, int i) {
    double mx = 0.0;
    for (int k = P.rp[i]; k < P.rp[i + 1]; ++k) mx = std::max(mx, std::fabs(P.ah[k]));
    if (!(mx > 0.0) || std::isinf(mx)) return 1.0;
    int e;
    double f = std::frexp(mx, &e);  // mx = f 2^e, f in [0.5, 1)
    int c = (f == 0.5) ? e - 1 : e;  // ceil(log2 mx)
    return std::ldexp(1.0, c);
}

Problem *make_problem(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val,
                      int diag_scale, int row_scale, int precond) {
    Problem *P = new Problem;
    P->n = n;
    P->diag_scale = diag_scale;
    P->row_scale = row_scale;
    P->precond = precond;
    int64_t nnz = rowptr[n];
    P->rp.assign(rowptr, rowptr + n + 1);
    P->ci.assign(colidx, colidx + nnz);
    P->a.assign(val, val + nnz);
    // D = |diag A|; Sec. 5 scales every matrix by its diagonal.
    std::vector<double> diag(n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int k = rowptr[i]; k < rowptr[i + 1]; ++k)
            if (colidx[k] == i) diag[i] = val[k];
    P->d.assign(n, 1.0);
    if (diag_scale)
        for (int i = 0; i < n; ++i)
            P->d[i] = (diag[i] != 0.0) ? 1.0 / std::sqrt(std::fabs(diag[i])) : 1.0;
    P->ah.resize(nnz);
    for (int i = 0; i < n; ++i)
        for (int k = rowptr[i]; k < rowptr[i + 1]; ++k)
            P->ah[k] = (val[k] * P->d[i]) * P->d[colidx[k]];
    P->a32.resize(nnz);
    P->a16.resize(nnz);
    P->abf.resize(nnz);
    P->rs16.assign(n, 1.0);
    P->rsbf.assign(n, 1.0);
    for (int i = 0; i < n; ++i) {
        double s = row_scale ? row_scale_of(*P, i) : 1.0;
        P->rs16[i] = s;
        P->rsbf[i] = s;
        for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            P->a32[k] = rnd_prec(ORC_F32, P->ah[k]);
            P->a16[k] = rnd16(P->ah[k] / s);
            P->abf[k] = rndbf16(P->ah[k] / s);
        }
    }
    // primary preconditioner M: Jacobi on the scaled matrix, or the identity
    P->m64.assign(n, 1.0);
    if (precond == ORC_PC_JACOBI)
        for (int i = 0; i < n; ++i) {
            double di = 0.0;
            for (int k = rowptr[i]; k < rowptr[i + 1]; ++k)
                if (colidx[k] == i) di = P->ah[k];
            P->m64[i] = (di != 0.0) ? 1.0 / di : 1.0;
        }
    P->m32.resize(n);
    P->m16.resize(n);
    P->mbf.resize(n);
    for (int i = 0; i < n; ++i) {
        P->m32[i] = rnd_prec(ORC_F32, P->m64[i]);
        P->m16[i] = rnd16(P->m64[i]);
        P->mbf[i] = rndbf16(P->m64[i]);
    }
    return P;
}

/* ----------------------------------------------------------- basic kernels */
/* y = A_prec x: row sums in CSR order, fused multiply-add in type T, then
 * times the row scale of a 16-bit copy (exact: a power of two). */
template <class T>
void spmv_t(const Problem &P, int a_prec, const T *x, T *y) {
    const std::vector<double> &v = vals_for(P, a_prec);
    const std::vector<double> *rs = rowscale_for(P, a_prec);
    const int n = P.n;
    OMP_FOR
    for (int i = 0; i < n; ++i) {
        T acc = 0;
        for (int k = P.rp[i]; k < P.rp[i + 1]; ++k) acc = fma_t((T)v[k], x[P.ci[k]], acc);
        if (rs) acc = acc * (T)(*rs)[i];
        y[i] = acc;
    }
}

void spmv_orig(const Problem &P, const double *x, double *y) {
    const int n = P.n;
    OMP_FOR
    for (int i = 0; i < n; ++i) {
        double acc = 0;
        for (int k = P.rp[i]; k < P.rp[i + 1]; ++k) acc = std::fma(P.a[k], x[P.ci[k]], acc);
        y[i] = acc;
    }
}

/* (x, y) accumulated sequentially with fused multiply-add in type T */
template <class T>
T dot_t(const T *x, const T *y, int n) {
    T s = 0;
    for (int i = 0; i < n; ++i) s = fma_t(x[i], y[i], s);
    return s;
}

template <class T>
bool all_finite(const T *x, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(x[i])) return false;
    return true;
}

/* Gram-Schmidt of w against V[0..j] (classical: all projections of a pass
 * are computed before w is updated); `passes` = 2 is CGS2.  hcol[l] is the
 * sum of the passes' coefficients. */
template <class T>
void cgs(std::vector<std::vector<T>> &V, int j, std::vector<T> &w, int passes, std::vector<T> &hcol) {
    const int n = (int)w.size();
    std::vector<T> h(j + 1);
    for (int p = 0; p < passes; ++p) {
        for (int l = 0; l <= j; ++l) h[l] = dot_t(V[l].data(), w.data(), n);
        OMP_FOR
        for (int i = 0; i < n; ++i) {
            T wi = w[i];
            for (int l = 0; l <= j; ++l) wi = fma_t(-h[l], V[l][i], wi);
            w[i] = wi;
        }
        for (int l = 0; l <= j; ++l) hcol[l] = (p == 0) ? h[l] : hcol[l] + h[l];
    }
}

/* Least-squares state of one FGMRES cycle: Hessenberg columns reduced to
 * upper-triangular form by Givens rotations, and the rotated right-hand side
 * g = beta e_1 (Saad, Iterative Methods for Sparse Linear Systems, 6.5.3). */
template <class T>
struct Givens {
    int m;
    std::vector<T> H;  // (m+1) x m, column-major: H[i + (m+1) j]
    std::vector<T> cs, sn, g;
    explicit Givens(int m_) : m(m_), H((m_ + 1) * m_, T(0)), cs(m_), sn(m_), g(m_ + 1, T(0)) {}
    T &h(int i, int j) { return H[i + (m + 1) * j]; }
    /* Store column j (hcol[0..j], h_{j+1,j} = hn), apply the previous
     * rotations, form rotation j.  Returns false if the column is degenerate. */
    bool add_column(int j, const std::vector<T> &hcol, T hn) {
        for (int i = 0; i <= j; ++i) h(i, j) = hcol[i];
        h(j + 1, j) = hn;
        for (int i = 0; i < j; ++i) {
            T t = cs[i] * h(i, j) + sn[i] * h(i + 1, j);
            h(i + 1, j) = -sn[i] * h(i, j) + cs[i] * h(i + 1, j);
            h(i, j) = t;
        }
        T a = h(j, j), b = h(j + 1, j);
        T rho = std::sqrt(a * a + b * b);
        if (!(rho > 0) || !std::isfinite(rho)) return false;
        cs[j] = a / rho;
        sn[j] = b / rho;
        h(j, j) = rho;
        h(j + 1, j) = 0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        return true;
    }
    /* back substitution R y = g[0..k-1] */
    std::vector<T> solve(int k) {
        std::vector<T> y(k);
        for (int r = k - 1; r >= 0; --r) {
            T s = g[r];
            for (int l = r + 1; l < k; ++l) s = fma_t(-h(r, l), y[l], s);
            y[r] = s / h(r, r);
        }
        return y;
    }
};

/* z_i = sum_k y_k Z[k]_i accumulated in k order with fused multiply-add */
template <class T>
void combine(const std::vector<std::vector<T>> &Z, const std::vector<T> &y, int k, T *z, int n) {
    OMP_FOR
    for (int i = 0; i < n; ++i) {
        T s = 0;
        for (int l = 0; l < k; ++l) s = fma_t(y[l], Z[l][i], s);
        z[i] = s;
    }
}

/* ------------------------------------------------------------------ the nest */
/* What one call of an inner FGMRES level leaves behind, for the Arnoldi and
 * Givens pins: basis V (m+1 vectors), preconditioned vectors Z (m), the
 * Hessenberg matrix before rotation ((m+1) x m, column-major), the rotated
 * right-hand side g (m+1) and the number of columns kept. */
struct InnerRecord {
    int level = -1;
    bool done = false;
    double *V = nullptr, *Z = nullptr, *H = nullptr, *g = nullptr;
    int kdim = 0;
};

struct Nest {
    const Problem &P;
    orc_params prm;
    orc_rich_state *st;
    int64_t m_applies = 0, r_calls = 0, r_update_calls = 0;
    InnerRecord *rec = nullptr;

    Nest(const Problem &P_, const orc_params &prm_, orc_rich_state *st_) : P(P_), prm(prm_), st(st_) {}

    /* M v in the caller's arithmetic type (Table 1: M stored in m_prec) */
    template <class T>
    void apply_M(const T *v, T *z) {
        if (prm.precond == ORC_PC_AINV) {
            ainv_apply<T>(v, z);
            m_applies += 1;
            return;
        }
        const std::vector<double> &m = m_for(P, prm.m_prec);
        const int n = P.n;
        OMP_FOR
        for (int i = 0; i < n; ++i) z[i] = (T)m[i] * v[i];
        m_applies += 1;
    }

    /* u = M r with the approximate inverse M = (I - Dt^-1 U) Dt^-1 (I - L Dt^-1),
     * factors rounded to m_prec, arithmetic in T, row sums in CSR order:
     * t = Dt^-1 (r - (L Dt^-1) r),  u = t - (Dt^-1 U) t. */
    template <class T>
    void ainv_apply(const T *r, T *u) {
        const int n = P.n;
        const int mp = prm.m_prec;
        std::vector<T> t(n);
        for (int i = 0; i < n; ++i) {
            T acc = 0;
            for (int k = P.rp[i]; k < P.rp[i + 1]; ++k)
                acc = fma_t((T)rnd_prec(mp, P.ainv_l[k]), r[P.ci[k]], acc);
            t[i] = (T)rnd_prec(mp, P.ainv_dinv[i]) * (r[i] - acc);
        }
        for (int i = 0; i < n; ++i) {
            T acc = 0;
            for (int k = P.rp[i]; k < P.rp[i + 1]; ++k)
                acc = fma_t((T)rnd_prec(mp, P.ainv_u[k]), t[P.ci[k]], acc);
            u[i] = t[i] - acc;
        }
    }

    /* One call of Algorithm 1 (Richardson with adaptive weights).
     * TP: the parent's vector type; TR: Richardson arithmetic type (fp32 for
     * 16-bit and fp32 storage, fp64 for fp64 storage). */
    template <class TP, class TR>
    void richardson(const TP *v, TP *zout) {
        const int n = P.n;
        const int prec = prm.rich_v_prec;
        const int m4 = prm.rich_m;
        const bool fixed = prm.omega_fixed > 0.0;
        if (st->c_ntr == 1 || fixed)
            for (int k = 0; k < m4; ++k) st->omega[k] = fixed ? (double)(TR)prm.omega_fixed : 1.0;
        const bool update = !fixed && (st->c_ntr % prm.c == 0);
        // power-of-two scaling sigma = 2^-floor(log2 max|v|) before a cast into 16-bit storage
        TP sigma = 1;
        if (prm.scale_cast && (prec == ORC_F16 || prec == ORC_BF16)) {
            TP amax = 0;
            for (int i = 0; i < n; ++i) amax = std::max(amax, (TP)std::fabs(v[i]));
            if (amax > 0 && std::isfinite(amax)) {
                int e;
                std::frexp((double)amax, &e);  // floor(log2 amax) = e - 1
                sigma = (TP)std::ldexp(1.0, 1 - e);
            }
        }
        const std::vector<double> &mv = m_for(P, prm.m_prec);
        std::vector<TR> vr(n), z(n, TR(0)), r(n), u(n), s(n), w(n);
        for (int i = 0; i < n; ++i) vr[i] = (TR)rnd_prec(prec, (double)(sigma * v[i]));
        for (int k = 0; k < m4; ++k) {
            if (k == 0) {
                r = vr;  // r_0 = v without an SpMV (z_0 = 0)
            } else {
                spmv_t<TR>(P, prm.rich_a_prec, z.data(), s.data());
                for (int i = 0; i < n; ++i) r[i] = (TR)rnd_prec(prec, (double)(vr[i] - s[i]));
            }
            if (prm.precond == ORC_PC_AINV)
                ainv_apply<TR>(r.data(), u.data());
            else
                for (int i = 0; i < n; ++i) u[i] = (TR)mv[i] * r[i];
            m_applies += 1;
            if (update) {
                spmv_t<TR>(P, prm.rich_a_prec, u.data(), w.data());
                TR num = dot_t(r.data(), w.data(), n);
                TR den = dot_t(w.data(), w.data(), n);
                TR wk = (TR)st->omega[k];
                TR wp = wk;
                bool ok = den > 0 && std::isfinite(num / den);
                if (ok) wp = num / den;
                for (int i = 0; i < n; ++i) z[i] = (TR)rnd_prec(prec, (double)fma_t(wp, u[i], z[i]));
                if (ok) {
                    TR l = (TR)(st->c_ntr / prm.c);
                    st->omega[k] = (double)((l * wk + wp) / (l + (TR)1));
                }
            } else {
                TR wk = (TR)st->omega[k];
                for (int i = 0; i < n; ++i) z[i] = (TR)rnd_prec(prec, (double)fma_t(wk, u[i], z[i]));
            }
        }
        st->c_ntr += 1;
        r_calls += 1;
        if (update) r_update_calls += 1;
        TP inv_sigma = (TP)1 / sigma;
        for (int i = 0; i < n; ++i) zout[i] = (TP)z[i] * inv_sigma;
    }

    template <class TP>
    void richardson_dispatch(const TP *v, TP *z) {
        if (prm.rich_v_prec == ORC_F64)
            richardson<TP, double>(v, z);
        else
            richardson<TP, float>(v, z);
    }

    /* The preconditioner of FGMRES level d: the next FGMRES level, else
     * Richardson, else M.  Leaving level 0 enters the scaled system:
     * P(v) = D^{-1/2} inner(D^{-1/2} v). */
    template <class T>
    void apply_below(int d, const T *v, T *z) {
        const int n = P.n;
        std::vector<T> u(v, v + n);
        const bool scale = (d == 0) && P.diag_scale;
        if (scale)
            for (int i = 0; i < n; ++i) u[i] = (T)(P.d[i] * (double)v[i]);
        const int child = d + 1;
        if (child < prm.nlevels) {
            if (prm.v_prec[child] == ORC_F64) {
                std::vector<double> uc(n), zc(n);
                for (int i = 0; i < n; ++i) uc[i] = (double)u[i];
                fgmres_inner<double>(child, uc.data(), zc.data());
                for (int i = 0; i < n; ++i) z[i] = (T)zc[i];
            } else {
                std::vector<float> uc(n), zc(n);
                for (int i = 0; i < n; ++i) uc[i] = (float)u[i];
                fgmres_inner<float>(child, uc.data(), zc.data());
                for (int i = 0; i < n; ++i) z[i] = (T)zc[i];
            }
        } else if (prm.rich_m > 0) {
            richardson_dispatch<T>(u.data(), z);
        } else {
            apply_M<T>(u.data(), z);
        }
        if (scale)
            for (int i = 0; i < n; ++i) z[i] = (T)(P.d[i] * (double)z[i]);
    }

    /* Richardson calls that one child call of level d schedules. */
    int64_t calls_below(int d) const {
        if (d + 1 >= prm.nlevels) return prm.rich_m > 0 ? 1 : 0;
        return (int64_t)prm.m[d + 1] * calls_below(d + 1);
    }

    /* One call of an inner FGMRES level (x0 = 0, a fixed m iterations, no
     * convergence check -- Sec. 4.2), or, with inner_rtol > 0 at the innermost
     * FGMRES level, until its residual estimate falls below inner_rtol * beta.
     * The weight counter c_ntr counts the scheduled Richardson calls: those of
     * iterations a level does not run are added when it ends.
     * A level with 16-bit vectors (v_prec F16 / BF16, the fp16 levels of
     * Table 4) computes in fp32 and rounds what it stores -- V[0], each
     * normalised V[j+1] and each Z[j] = M V[j] -- to that format; w and the
     * small Hessenberg problem stay in fp32. */
    template <class T>
    void fgmres_inner(int d, const T *v, T *z) {
        const int n = P.n, m = prm.m[d];
        const int vs = prm.v_prec[d];
        const bool v16 = vs == ORC_F16 || vs == ORC_BF16;
        auto store = [&](T x) { return v16 ? (T)rnd_prec(vs, (double)x) : x; };
        T beta = std::sqrt(dot_t(v, v, n));
        if (!std::isfinite(beta)) {
            for (int i = 0; i < n; ++i) z[i] = (T)NAN;
            st->c_ntr += (int64_t)m * calls_below(d);
            return;
        }
        if (!(beta > 0)) {
            for (int i = 0; i < n; ++i) z[i] = 0;
            st->c_ntr += (int64_t)m * calls_below(d);
            return;
        }
        const bool adaptive = prm.inner_rtol > 0.0 && d == prm.nlevels - 1;
        const T rtol = (T)prm.inner_rtol;
        int ran = 0;
        std::vector<std::vector<T>> V(m + 1, std::vector<T>(n)), Z(m, std::vector<T>(n));
        std::vector<T> w(n), hcol(m + 1), Hraw((size_t)(m + 1) * m, T(0));
        Givens<T> G(m);
        T inv = (T)1 / beta;
        for (int i = 0; i < n; ++i) V[0][i] = store(v[i] * inv);
        G.g[0] = beta;
        int kdim = 0;
        for (int j = 0; j < m; ++j) {
            apply_below<T>(d, V[j].data(), Z[j].data());
            if (v16)
                for (int i = 0; i < n; ++i) Z[j][i] = store(Z[j][i]);
            ran = j + 1;
            spmv_t<T>(P, prm.a_prec[d], Z[j].data(), w.data());
            cgs<T>(V, j, w, prm.cgs_passes, hcol);
            T hn = std::sqrt(dot_t(w.data(), w.data(), n));
            for (int i = 0; i <= j; ++i) Hraw[i + (size_t)(m + 1) * j] = hcol[i];
            Hraw[j + 1 + (size_t)(m + 1) * j] = hn;
            if (!std::isfinite(hn) || !all_finite(hcol.data(), j + 1)) break;  // drop column j
            if (!G.add_column(j, hcol, hn)) break;
            kdim = j + 1;
            if (!(hn > 0)) break;  // exact breakdown: the subspace holds the solution
            if (adaptive && std::abs(G.g[j + 1]) <= rtol * beta) break;  // level residual small enough
            T invh = (T)1 / hn;
            for (int i = 0; i < n; ++i) V[j + 1][i] = store(w[i] * invh);
        }
        st->c_ntr += (int64_t)(m - ran) * calls_below(d);
        std::vector<T> y = G.solve(kdim);
        combine(Z, y, kdim, z, n);
        if (rec && rec->level == d && !rec->done) record_inner(V, Z, Hraw, G, kdim, m);
    }

    /* copy one inner call's basis, Hessenberg matrix and rotated g out */
    template <class T>
    void record_inner(const std::vector<std::vector<T>> &V, const std::vector<std::vector<T>> &Z,
                      const std::vector<T> &Hraw, const Givens<T> &G, int kdim, int m) {
        const int n = P.n;
        rec->done = true;
        rec->kdim = kdim;
        for (int k = 0; k <= m; ++k)
            for (int i = 0; i < n; ++i) rec->V[(size_t)k * n + i] = (double)V[k][i];
        for (int k = 0; k < m; ++k)
            for (int i = 0; i < n; ++i) rec->Z[(size_t)k * n + i] = (double)Z[k][i];
        for (int k = 0; k < (m + 1) * m; ++k) rec->H[k] = (double)Hraw[k];
        for (int k = 0; k <= m; ++k) rec->g[k] = (double)G.g[k];
    }

    /* The outermost fp64 FGMRES(m1) with restarts (Sec. 4.2, Sec. 5). */
    int solve(const double *b, double *x, orc_stats *S, double *recV, double *recZ, double *recH,
              int rec_steps) {
        const int n = P.n, m = prm.m[0];
        auto push = [](double *arr, int cap, int &len, double v) {
            if (arr && len < cap) arr[len] = v;
            ++len;
        };
        int hist_len = 0, true_len = 0;
        double nb = std::sqrt(dot_t(b, b, n));
        st->c_ntr = 1;
        int status = ORC_NOT_CONVERGED;
        int total = 0, cycles = 0;
        double rel = 0.0;
        std::vector<double> r(n), w(n), hcol(m + 1), zy(n);
        if (!(nb > 0)) {
            for (int i = 0; i < n; ++i) x[i] = 0.0;
            status = std::isfinite(nb) ? ORC_OK : ORC_NONFINITE;
        }
        while (nb > 0) {
            spmv_orig(P, x, r.data());
            for (int i = 0; i < n; ++i) r[i] = b[i] - r[i];
            double beta = std::sqrt(dot_t(r.data(), r.data(), n));
            rel = beta / nb;
            push(S ? S->true_hist : nullptr, S ? S->true_cap : 0, true_len, rel);
            if (!std::isfinite(beta)) { status = ORC_NONFINITE; break; }
            if (rel < prm.tol) { status = ORC_OK; break; }
            if (total >= prm.max_outer || (rec_steps > 0 && cycles > 0)) { status = ORC_NOT_CONVERGED; break; }
            ++cycles;
            std::vector<std::vector<double>> V(m + 1, std::vector<double>(n)), Z(m, std::vector<double>(n));
            Givens<double> G(m);
            double inv = 1.0 / beta;
            for (int i = 0; i < n; ++i) V[0][i] = r[i] * inv;
            G.g[0] = beta;
            int kdim = 0;
            bool nonfinite = false;
            for (int j = 0; j < m; ++j) {
                apply_below<double>(0, V[j].data(), Z[j].data());
                spmv_orig(P, Z[j].data(), w.data());
                cgs<double>(V, j, w, prm.cgs_passes, hcol);
                double hn = std::sqrt(dot_t(w.data(), w.data(), n));
                ++total;
                if (recH && j < rec_steps) {
                    for (int i = 0; i <= j; ++i) recH[i + (rec_steps + 1) * j] = hcol[i];
                    recH[j + 1 + (rec_steps + 1) * j] = hn;
                }
                if (!std::isfinite(hn) || !all_finite(hcol.data(), j + 1)) { nonfinite = true; break; }
                if (!G.add_column(j, hcol, hn)) break;
                kdim = j + 1;
                double est = std::fabs(G.g[j + 1]) / nb;
                push(S ? S->hist : nullptr, S ? S->hist_cap : 0, hist_len, est);
                if (!(hn > 0)) break;
                for (int i = 0; i < n; ++i) V[j + 1][i] = w[i] * (1.0 / hn);
                if (rec_steps > 0 && j + 1 >= rec_steps) break;
                if (est < prm.tol || total >= prm.max_outer) break;
            }
            if (recV) {
                for (int k = 0; k <= std::min(kdim, rec_steps); ++k)
                    std::memcpy(recV + (size_t)k * n, V[k].data(), sizeof(double) * n);
                for (int k = 0; k < std::min(kdim, rec_steps); ++k)
                    std::memcpy(recZ + (size_t)k * n, Z[k].data(), sizeof(double) * n);
            }
            std::vector<double> y = G.solve(kdim);
            combine(Z, y, kdim, zy.data(), n);
            for (int i = 0; i < n; ++i) x[i] = x[i] + zy[i];
            if (nonfinite) {
                status = ORC_NONFINITE;
                break;
            }
        }
        if (S) {
            S->status = status;
            S->outer_iters = total;
            S->restarts = cycles > 0 ? cycles - 1 : 0;
            S->rel_res_true = rel;
            S->m_applies = m_applies;
            S->r_calls = r_calls;
            S->r_update_calls = r_update_calls;
            for (int k = 0; k < 8; ++k) S->omega[k] = st->omega[k];
            S->hist_len = hist_len;
            S->true_len = true_len;
        }
        return status;
    }
};

}  // namespace

/* ------------------------------------------------------------------ C API */
extern "C" {

void orc_round(int prec, const double *x, double *y, int64_t n) {
    for (int64_t i = 0; i < n; ++i) y[i] = rnd_prec(prec, x[i]);
}

void *orc_problem_create(int32_t n, const int32_t *rowptr, const int32_t *colidx, const double *val,
                         int diag_scale, int row_scale, int precond) {
    return make_problem(n, rowptr, colidx, val, diag_scale, row_scale, precond);
}

void orc_problem_destroy(void *p) { delete (Problem *)p; }

void orc_problem_set_ainv(void *p, double alpha) {
    Problem &P = *(Problem *)p;
    const int n = P.n;
    std::vector<double> dt(n);
    for (int i = 0; i < n; ++i) {
        double dii = 0.0;
        for (int k = P.rp[i]; k < P.rp[i + 1]; ++k)
            if (P.ci[k] == i) dii = P.ah[k];
        dt[i] = (dii != 0.0) ? alpha * dii : alpha;
    }
    const size_t nnz = P.ci.size();
    P.ainv_l.assign(nnz, 0.0);
    P.ainv_u.assign(nnz, 0.0);
    P.ainv_dinv.resize(n);
    for (int i = 0; i < n; ++i) {
        P.ainv_dinv[i] = 1.0 / dt[i];
        for (int k = P.rp[i]; k < P.rp[i + 1]; ++k) {
            const int c = P.ci[k];
            if (c < i) P.ainv_l[k] = P.ah[k] / dt[c];
            else if (c > i) P.ainv_u[k] = P.ah[k] / dt[i];
        }
    }
}

int64_t orc_problem_get(void *p, int which, double *out) {
    const Problem &P = *(const Problem *)p;
    const std::vector<double> *src = nullptr;
    switch (which) {
        case 0: src = &P.d; break;
        case 1: src = &P.ah; break;
        case 2: src = &P.a32; break;
        case 3: src = &P.a16; break;
        case 4: src = &P.abf; break;
        case 5: src = &P.rs16; break;
        case 6: src = &P.rsbf; break;
        case 7: src = &P.m64; break;
        case 8: src = &P.m32; break;
        case 9: src = &P.m16; break;
        case 10: src = &P.mbf; break;
        case 11: src = &P.ainv_l; break;
        case 12: src = &P.ainv_u; break;
        case 13: src = &P.ainv_dinv; break;
        default: return -1;
    }
    if (out) std::memcpy(out, src->data(), sizeof(double) * src->size());
    return (int64_t)src->size();
}

void orc_default_params(orc_params *prm) {
    std::memset(prm, 0, sizeof(*prm));
    prm->nlevels = 3;
    prm->m[0] = 100; prm->m[1] = 8; prm->m[2] = 4; prm->m[3] = 0;
    prm->a_prec[0] = ORC_F64; prm->a_prec[1] = ORC_F32; prm->a_prec[2] = ORC_F16; prm->a_prec[3] = ORC_F16;
    prm->v_prec[0] = ORC_F64; prm->v_prec[1] = ORC_F32; prm->v_prec[2] = ORC_F32; prm->v_prec[3] = ORC_F32;
    prm->rich_m = 2;
    prm->rich_a_prec = ORC_F16;
    prm->rich_v_prec = ORC_F16;
    prm->m_prec = ORC_F16;
    prm->precond = ORC_PC_JACOBI;
    prm->c = 64;
    prm->omega_fixed = 0.0;
    prm->diag_scale = 1;
    prm->row_scale = 0;
    prm->scale_cast = 1;
    prm->cgs_passes = 2;
    prm->tol = 1e-9;
    prm->max_outer = 300;
    prm->inner_rtol = 0.0;
}

void orc_spmv(void *p, int a_prec, int v_prec, const double *x, double *y) {
    const Problem &P = *(const Problem *)p;
    const int n = P.n;
    if (v_prec == ORC_F64) {
        spmv_t<double>(P, a_prec, x, y);
    } else {
        std::vector<float> xf(n), yf(n);
        for (int i = 0; i < n; ++i) xf[i] = (float)x[i];
        spmv_t<float>(P, a_prec, xf.data(), yf.data());
        for (int i = 0; i < n; ++i) y[i] = yf[i];
    }
}

void orc_spmv_orig(void *p, const double *x, double *y) { spmv_orig(*(const Problem *)p, x, y); }

void orc_apply(void *p, const orc_params *prm, orc_rich_state *st, int level, const double *v, double *z) {
    const Problem &P = *(const Problem *)p;
    Nest N(P, *prm, st);
    const int n = P.n;
    // the input arrives in the vector type of the parent level
    const int parent_prec = prm->v_prec[level - 1 < 0 ? 0 : level - 1];
    if (level < prm->nlevels) {
        if (prm->v_prec[level] == ORC_F64) {
            N.fgmres_inner<double>(level, v, z);
        } else {
            std::vector<float> vf(n), zf(n);
            for (int i = 0; i < n; ++i) vf[i] = (float)v[i];
            N.fgmres_inner<float>(level, vf.data(), zf.data());
            for (int i = 0; i < n; ++i) z[i] = zf[i];
        }
    } else if (prm->rich_m > 0) {
        if (parent_prec == ORC_F64) {
            N.richardson_dispatch<double>(v, z);
        } else {
            std::vector<float> vf(n), zf(n);
            for (int i = 0; i < n; ++i) vf[i] = (float)v[i];
            N.richardson_dispatch<float>(vf.data(), zf.data());
            for (int i = 0; i < n; ++i) z[i] = zf[i];
        }
    } else {
        if (parent_prec == ORC_F64) {
            N.apply_M<double>(v, z);
        } else {
            std::vector<float> vf(n), zf(n);
            for (int i = 0; i < n; ++i) vf[i] = (float)v[i];
            N.apply_M<float>(vf.data(), zf.data());
            for (int i = 0; i < n; ++i) z[i] = zf[i];
        }
    }
}

int orc_solve(void *p, const orc_params *prm, const double *b, double *x, orc_stats *stats) {
    const Problem &P = *(const Problem *)p;
    orc_rich_state st;
    std::memset(&st, 0, sizeof(st));
    st.c_ntr = 1;
    Nest N(P, *prm, &st);
    return N.solve(b, x, stats, nullptr, nullptr, nullptr, 0);
}

int orc_outer_arnoldi(void *p, const orc_params *prm, const double *b, int steps, double *V, double *Z,
                      double *H) {
    const Problem &P = *(const Problem *)p;
    orc_rich_state st;
    std::memset(&st, 0, sizeof(st));
    st.c_ntr = 1;
    orc_params q = *prm;
    q.m[0] = steps;
    q.tol = 0.0;
    std::vector<double> x(P.n, 0.0);
    Nest N(P, q, &st);
    return N.solve(b, x.data(), nullptr, V, Z, H, steps);
}

int orc_inner_arnoldi(void *p, const orc_params *prm, orc_rich_state *st, int level, const double *v,
                      double *z, double *V, double *Z, double *H, double *g) {
    const Problem &P = *(const Problem *)p;
    if (level < 1 || level >= prm->nlevels) return -1;
    Nest N(P, *prm, st);
    InnerRecord R;
    R.level = level;
    R.V = V;
    R.Z = Z;
    R.H = H;
    R.g = g;
    N.rec = &R;
    const int n = P.n;
    if (prm->v_prec[level] == ORC_F64) {
        N.fgmres_inner<double>(level, v, z);
    } else {
        std::vector<float> vf(n), zf(n);
        for (int i = 0; i < n; ++i) vf[i] = (float)v[i];
        N.fgmres_inner<float>(level, vf.data(), zf.data());
        for (int i = 0; i < n; ++i) z[i] = zf[i];
    }
    return R.done ? R.kdim : -1;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

}  // extern "C"
