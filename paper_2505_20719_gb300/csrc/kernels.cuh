// Device kernels of the F3R nest: SpMV with fused Gram-Schmidt dot products,
// CGS2 passes, normalisation with the precision cast into the next level,
// the Givens / least-squares step, the solution combination, the primary
// preconditioner and the fp64 outer level.
//
// One FGMRES level (Sec. 4.2, Table 1) runs, per iteration j,
//   child call -> Z[j]
//   k_spmv_dots   : w = A_l Z[j], hA = V[0..j]^T w           (pass-1 dots fused)
//   k_cgs_pass    : w -= V hA, hB = V[0..j]^T w              (second CGS pass)
//   k_cgs_final   : w -= V hB, ||w||^2, max|w| -> Givens     (norm fused)
//   k_normalize   : V[j+1] = w / ||w|| and the child's input (cast, scaling)
// and finally k_combine: z = sum_k y_k Z[k] into the parent's slot.
#pragma once
#include <utility>

#include "common.cuh"

namespace f3r {

enum { CHILD_F = 0, CHILD_R = 1, CHILD_M = 2 };

// misc scalars of a level (after H, cs, sn, g, y, hA, hB)
enum { MS_BETA = 0, MS_INV = 1, MS_SIGMA = 2, MS_INV_SIGMA = 3, MS_NB = 4, MS_EST = 5, MS_REL = 6,
       MS_AMAX = 7, MS_COUNT = 16 };
// per-level int flags (4 per level)
enum { IF_KDIM = 0, IF_STOP = 1, IF_NONFINITE = 2, IF_J = 3 };

__host__ __device__ inline int scal_H(int m) { return 0; }
__host__ __device__ inline int scal_cs(int m) { return (m + 1) * m; }
__host__ __device__ inline int scal_sn(int m) { return (m + 1) * m + m; }
__host__ __device__ inline int scal_g(int m) { return (m + 1) * m + 2 * m; }
__host__ __device__ inline int scal_y(int m) { return (m + 1) * m + 3 * m + 1; }
__host__ __device__ inline int scal_hA(int m) { return (m + 1) * m + 4 * m + 1; }
__host__ __device__ inline int scal_hB(int m) { return (m + 1) * m + 5 * m + 2; }
__host__ __device__ inline int scal_misc(int m) { return (m + 1) * m + 6 * m + 3; }
__host__ __device__ inline int scal_size(int m) { return scal_misc(m) + MS_COUNT; }

// Device view of one FGMRES level with vector type T.
template <class T> struct LevelDev {
    int n, ld, m, depth;
    float rtol;        // > 0: stop once |g_{j+1}| <= rtol * beta (adaptive inner level)
    T *V, *Z, *w;
    T *scal;
    int *flags;        // base of all levels' flags; this level's at flags[4*depth]
    const int *jptr;   // outer level: iteration index read on the device (graph replay)
    int vround = 0;    // the level's stored vectors V, Z rounded to 1: fp16, 2: bf16 (Table 4's fp16 levels)
    __device__ T *H() const { return scal + scal_H(m); }
    __device__ T *cs() const { return scal + scal_cs(m); }
    __device__ T *sn() const { return scal + scal_sn(m); }
    __device__ T *g() const { return scal + scal_g(m); }
    __device__ T *y() const { return scal + scal_y(m); }
    __device__ T *hA() const { return scal + scal_hA(m); }
    __device__ T *hB() const { return scal + scal_hB(m); }
    __device__ T *misc() const { return scal + scal_misc(m); }
    __device__ int *fl() const { return flags + 4 * depth; }
};

// a value of a level's stored vector V or Z: rounded to 16 bits at the levels
// that store their vectors in fp16 / bf16 (kept in fp32 arrays)
template <class T> __device__ __forceinline__ T vstore(int vround, T v) {
    if (vround == 1) return rnd<h16>(v);
    if (vround == 2) return rnd<b16>(v);
    return v;
}

// true when level `upto` or one of its inner ancestors (levels >= 1) stopped
__device__ __forceinline__ bool stopped(const int *flags, int upto) {
    for (int l = 1; l <= upto; ++l)
        if (((volatile const int *)flags)[4 * l + IF_STOP]) return true;
    return false;
}

// ---------------------------------------------------------------- Givens step
// Thread-serial update of the least-squares state with column j
// (Saad, Iterative Methods for Sparse Linear Systems, 6.5.3); solves for y
// when the level ends at this column.
template <class T>
__device__ void givens_column(const LevelDev<T> &L, int j, const T *hcol, T hn, bool last_iter) {
    T *H = L.H(), *cs = L.cs(), *sn = L.sn(), *g = L.g();
    const int ldh = L.m + 1;
    int *fl = L.fl();
    bool finite = isfinite(hn);
    for (int i = 0; i <= j; ++i) finite = finite && isfinite(hcol[i]);
    bool ok = finite;
    if (ok) {
        for (int i = 0; i <= j; ++i) H[i + ldh * j] = hcol[i];
        H[j + 1 + ldh * j] = hn;
        for (int i = 0; i < j; ++i) {
            T t = add_rn(mul_rn(cs[i], H[i + ldh * j]), mul_rn(sn[i], H[i + 1 + ldh * j]));
            H[i + 1 + ldh * j] = add_rn(mul_rn(-sn[i], H[i + ldh * j]), mul_rn(cs[i], H[i + 1 + ldh * j]));
            H[i + ldh * j] = t;
        }
        T a = H[j + ldh * j], b = H[j + 1 + ldh * j];
        T rho = sqrt_rn(add_rn(mul_rn(a, a), mul_rn(b, b)));
        ok = (rho > (T)0) && isfinite(rho);
        if (ok) {
            cs[j] = div_rn(a, rho);
            sn[j] = div_rn(b, rho);
            H[j + ldh * j] = rho;
            H[j + 1 + ldh * j] = (T)0;
            g[j + 1] = mul_rn(-sn[j], g[j]);
            g[j] = mul_rn(cs[j], g[j]);
        }
    }
    if (!finite) fl[IF_NONFINITE] = 1;
    bool stop = !ok;
    if (ok) {
        fl[IF_KDIM] = j + 1;
        if (!(hn > (T)0)) stop = true;  // exact breakdown
        else L.misc()[MS_INV] = div_rn((T)1, hn);
        if (L.rtol > 0.0f && fabs(g[j + 1]) <= mul_rn((T)L.rtol, L.misc()[MS_BETA])) stop = true;
    }
    if (stop) fl[IF_STOP] = 1;
    if (stop || last_iter) {
        // back substitution R y = g over the kept columns
        const int k = fl[IF_KDIM];
        T *y = L.y();
        for (int r = k - 1; r >= 0; --r) {
            T s = g[r];
            for (int l = r + 1; l < k; ++l) s = fma_rn(-H[r + ldh * l], y[l], s);
            y[r] = div_rn(s, H[r + ldh * r]);
        }
    }
}

// ---------------------------------------------------------- inner-level kernels
// w = A Z[j] (times the row scale of a 16-bit copy), hA = V[0..j]^T w
template <class TA, class T>
__global__ void __launch_bounds__(kBlock) k_spmv_dots(Sell S, const TA *__restrict__ val,
                                                      const float *__restrict__ rs, LevelDev<T> L, int j,
                                                      GridRed<T> gr) {
    pdl_enter();
    if (stopped(L.flags, L.depth)) return;
    const T *__restrict__ x = L.Z + (size_t)j * L.ld;
    T acc[kMaxDots];
#pragma unroll
    for (int l = 0; l < kMaxDots; ++l) acc[l] = (T)0;
    const int lane = threadIdx.x & 31;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int s = wid; s < S.nslices; s += nw) {
        T y = sell_row<T>(S, val, s, lane, [&](int c) { return __ldg(x + c); });
        const int i = s * kSlice + lane;
        if (rs) y = mul_rn(y, (T)__ldg(rs + i));
        if (i < L.n) {
            L.w[i] = y;
#pragma unroll
            for (int l = 0; l < kMaxDots; ++l)
                if (l <= j) acc[l] = fma_rn(L.V[(size_t)l * L.ld + i], y, acc[l]);
        }
    }
    grid_reduce<T, kMaxDots>(acc, j + 1, false, gr, [&](T *res) {
        T *hA = L.hA();
        for (int l = 0; l <= j; ++l) hA[l] = res[l];
    });
}

constexpr int kVecBlock = 512;  // threads per block of the streaming vector kernels
constexpr int kUnroll = 1;       // 16-byte packs in flight per thread and vector

// Grid-stride walk over 16-byte packs, kUnroll packs per thread per step:
// f(q, valid) is called for packs q = base + tid + u * nth (coalesced per u).
template <class F> __device__ __forceinline__ void for_packs(int npacks, F f) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    for (int base = 0; base < npacks; base += nth * kUnroll) f(base + tid, nth);
}

// w -= V[0..j] h (fma in l order), then hB = V[0..j]^T w.  Streams 16-byte
// packs; MAXD bounds j + 1 so the register footprint follows the level size.
template <class T, int MAXD>
__global__ void __launch_bounds__(kVecBlock) k_cgs_pass(LevelDev<T> L, int j, GridRed<T> gr) {
    pdl_enter();
    if (stopped(L.flags, L.depth)) return;
    constexpr int N = PackN<T>::N;
    __shared__ T hs[MAXD];
    if (threadIdx.x <= j) hs[threadIdx.x] = L.hA()[threadIdx.x];
    __syncthreads();
    T acc[MAXD];
#pragma unroll
    for (int l = 0; l < MAXD; ++l) acc[l] = (T)0;
    const int nq = L.n / N;
    T *__restrict__ w = L.w;
    const T *__restrict__ V = L.V;
    for_packs(nq, [&](int q0, int nth) {
        Pack<T, N> wv[kUnroll];
        Pack<T, N> v[kUnroll][MAXD];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int q = q0 + u * nth;
            if (q < nq) {
                wv[u] = ldp<T, N>(w + (size_t)q * N);
#pragma unroll
                for (int l = 0; l < MAXD; ++l)
                    if (l <= j) v[u][l] = ldp<T, N>(V + (size_t)l * L.ld + (size_t)q * N);
            }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int q = q0 + u * nth;
            if (q < nq) {
#pragma unroll
                for (int l = 0; l < MAXD; ++l)
                    if (l <= j) {
#pragma unroll
                        for (int e = 0; e < N; ++e) wv[u].v[e] = fma_rn(-hs[l], v[u][l].v[e], wv[u].v[e]);
                    }
                stp<T, N>(w + (size_t)q * N, wv[u]);
#pragma unroll
                for (int l = 0; l < MAXD; ++l)
                    if (l <= j) {
#pragma unroll
                        for (int e = 0; e < N; ++e) acc[l] = fma_rn(v[u][l].v[e], wv[u].v[e], acc[l]);
                    }
            }
        }
    });
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    for (int i = nq * N + tid; i < L.n; i += nth) {
        T wi = w[i];
        T v[MAXD];
#pragma unroll
        for (int l = 0; l < MAXD; ++l)
            if (l <= j) {
                v[l] = V[(size_t)l * L.ld + i];
                wi = fma_rn(-hs[l], v[l], wi);
            }
        w[i] = wi;
#pragma unroll
        for (int l = 0; l < MAXD; ++l)
            if (l <= j) acc[l] = fma_rn(v[l], wi, acc[l]);
    }
    grid_reduce<T, MAXD>(acc, j + 1, false, gr, [&](T *res) {
        T *hB = L.hB();
        for (int l = 0; l <= j; ++l) hB[l] = res[l];
    });
}

// w -= V[0..j] h_last; ||w||^2 and max|w|; Givens step with column hA (+ hB);
// the scale of the child's 16-bit cast of V[j+1] from max|w| / ||w||.
template <class T, int MAXD>
__global__ void __launch_bounds__(kVecBlock) k_cgs_final(LevelDev<T> L, int j, int passes, int last_iter,
                                                         int want_sigma, GridRed<T> gr) {
    pdl_enter();
    if (stopped(L.flags, L.depth)) return;
    constexpr int N = PackN<T>::N;
    __shared__ T hs[MAXD];
    const T *hl = (passes == 2) ? L.hB() : L.hA();
    if (threadIdx.x <= j) hs[threadIdx.x] = hl[threadIdx.x];
    __syncthreads();
    T acc[2] = {(T)0, (T)0};
    const int nq = L.n / N;
    T *__restrict__ w = L.w;
    const T *__restrict__ V = L.V;
    for_packs(nq, [&](int q0, int nth) {
        Pack<T, N> wv[kUnroll];
        Pack<T, N> v[kUnroll][MAXD];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int q = q0 + u * nth;
            if (q < nq) {
                wv[u] = ldp<T, N>(w + (size_t)q * N);
#pragma unroll
                for (int l = 0; l < MAXD; ++l)
                    if (l <= j) v[u][l] = ldp<T, N>(V + (size_t)l * L.ld + (size_t)q * N);
            }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int q = q0 + u * nth;
            if (q < nq) {
#pragma unroll
                for (int l = 0; l < MAXD; ++l)
                    if (l <= j) {
#pragma unroll
                        for (int e = 0; e < N; ++e) wv[u].v[e] = fma_rn(-hs[l], v[u][l].v[e], wv[u].v[e]);
                    }
                stp<T, N>(w + (size_t)q * N, wv[u]);
#pragma unroll
                for (int e = 0; e < N; ++e) {
                    acc[0] = fma_rn(wv[u].v[e], wv[u].v[e], acc[0]);
                    acc[1] = fmax(acc[1], fabs(wv[u].v[e]));
                }
            }
        }
    });
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    for (int i = nq * N + tid; i < L.n; i += nth) {
        T wi = w[i];
#pragma unroll
        for (int l = 0; l < MAXD; ++l)
            if (l <= j) wi = fma_rn(-hs[l], V[(size_t)l * L.ld + i], wi);
        w[i] = wi;
        acc[0] = fma_rn(wi, wi, acc[0]);
        acc[1] = fmax(acc[1], fabs(wi));
    }
    grid_reduce<T, 2>(acc, 1, true, gr, [&](T *res) {
        T hcol[MAXD];
        const T *hA = L.hA(), *hB = L.hB();
        for (int l = 0; l <= j; ++l) hcol[l] = (passes == 2) ? add_rn(hA[l], hB[l]) : hA[l];
        T hn = sqrt_rn(res[0]);
        givens_column(L, j, hcol, hn, last_iter != 0);
        T *ms = L.misc();
        if (want_sigma && hn > (T)0) {
            T sig = pow2_scale_for(mul_rn(res[1], ms[MS_INV]));
            ms[MS_SIGMA] = sig;
            ms[MS_INV_SIGMA] = div_rn((T)1, sig);
        } else {
            ms[MS_SIGMA] = (T)1;
            ms[MS_INV_SIGMA] = (T)1;
        }
    });
}

// Child of a normalisation: where V[j+1] goes next.
//   CHILD_F: the next FGMRES level's V[0] (type TC), optionally times D^-1/2
//            (leaving level 0), with its norm and max -> the child's beta.
//   CHILD_R: the 16-bit Richardson input sigma * V[j+1] (type TC = storage).
//   CHILD_M: nothing.
template <class TC> struct ChildOut {
    TC *x;              // CHILD_F: child V[0]; CHILD_R: Richardson input vector
    const double *dsc;  // D^-1/2 when leaving level 0 with scaling, else null
    // CHILD_F only: the child level's scalar block and flags
    void *cscal;
    int cm;             // child m
    int cdepth;
    int want_sigma;     // grandchild is a 16-bit Richardson level
};

// V[dst] = src * inv (inv = 1/||src|| of this level); child input from it.
// src == V[0] (in place) at a level start, w otherwise.
template <class T, class TC, int CHILD>
__global__ void __launch_bounds__(kVecBlock) k_normalize(LevelDev<T> L, const T *src, int dst, int check_depth,
                                                      ChildOut<TC> co, GridRed<T> gr) {
    pdl_enter();
    if (stopped(L.flags, check_depth)) return;
    constexpr int N = PackN<T>::N;
    const int jd = L.jptr ? (*L.jptr + dst) : dst;
    T *out = L.V + (size_t)jd * L.ld;
    const T inv = L.misc()[MS_INV];
    const T sig = L.misc()[MS_SIGMA];
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    const int nq = L.n / N;
    if constexpr (CHILD == CHILD_F) {
        TC acc[2] = {(TC)0, (TC)0};
        auto one = [&](int i, T sv) {
            const T v = vstore(L.vround, mul_rn(sv, inv));
            const TC c = co.dsc ? Store<TC>::from(mul_rn(co.dsc[i], (double)v)) : Store<TC>::from(v);
            acc[0] = fma_rn(c, c, acc[0]);
            acc[1] = fmax(acc[1], fabs(c));
            return std::pair<T, TC>(v, c);
        };
        for_packs(nq, [&](int q0, int nthr) {
            Pack<T, N> sp[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
                if (q0 + u * nthr < nq) sp[u] = ldp<T, N>(src + (size_t)(q0 + u * nthr) * N);
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const int q = q0 + u * nthr;
                if (q < nq) {
                    Pack<T, N> op;
                    Pack<TC, N> cp;
#pragma unroll
                    for (int e = 0; e < N; ++e) {
                        auto vc = one(q * N + e, sp[u].v[e]);
                        op.v[e] = vc.first;
                        cp.v[e] = vc.second;
                    }
                    stp<T, N>(out + (size_t)q * N, op);
                    stp<TC, N>(co.x + (size_t)q * N, cp);
                }
            }
        });
        for (int i = nq * N + tid; i < L.n; i += nth) {
            auto vc = one(i, src[i]);
            out[i] = vc.first;
            co.x[i] = vc.second;
        }
        GridRed<TC> grc{(TC *)gr.partials, gr.ticket, gr.stride};
        grid_reduce<TC, 2>(acc, 1, true, grc, [&](TC *res) {
            LevelDev<TC> C;
            C.m = co.cm;
            C.scal = (TC *)co.cscal;
            C.depth = co.cdepth;
            C.flags = L.flags;
            TC *ms = C.misc();
            int *cf = C.fl();
            const TC beta = sqrt_rn(res[0]);
            cf[IF_KDIM] = 0;
            cf[IF_NONFINITE] = isfinite(beta) ? 0 : 1;
            const bool run = (beta > (TC)0) && isfinite(beta);
            cf[IF_STOP] = run ? 0 : 1;
            ms[MS_BETA] = beta;
            if (run) {
                ms[MS_INV] = div_rn((TC)1, beta);
                C.g()[0] = beta;
                const TC sg = co.want_sigma ? pow2_scale_for(mul_rn(res[1], ms[MS_INV])) : (TC)1;
                ms[MS_SIGMA] = sg;
                ms[MS_INV_SIGMA] = div_rn((TC)1, sg);
            }
            if (L.jptr && dst == 1) atomicAdd(const_cast<int *>(L.jptr), 1);  // closes outer iteration j
        });
    } else {
        for_packs(nq, [&](int q0, int nthr) {
            Pack<T, N> sp[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
                if (q0 + u * nthr < nq) sp[u] = ldp<T, N>(src + (size_t)(q0 + u * nthr) * N);
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const int q = q0 + u * nthr;
                if (q < nq) {
                    Pack<T, N> op;
#pragma unroll
                    for (int e = 0; e < N; ++e) op.v[e] = vstore(L.vround, mul_rn(sp[u].v[e], inv));
                    stp<T, N>(out + (size_t)q * N, op);
                    if constexpr (CHILD == CHILD_R) {
                        Pack<TC, N> cp;
#pragma unroll
                        for (int e = 0; e < N; ++e) cp.v[e] = Store<TC>::from(mul_rn(sig, op.v[e]));
                        stp<TC, N>(co.x + (size_t)q * N, cp);
                    }
                }
            }
        });
        for (int i = nq * N + tid; i < L.n; i += nth) {
            const T v = vstore(L.vround, mul_rn(src[i], inv));
            out[i] = v;
            if constexpr (CHILD == CHILD_R) co.x[i] = Store<TC>::from(mul_rn(sig, v));
        }
        if (L.jptr && dst == 1) {
            // outer level without an FGMRES child: advance j after every block read it
            __shared__ bool last;
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) last = (atomicAdd(gr.ticket, 1u) == gridDim.x - 1);
            __syncthreads();
            if (last && threadIdx.x == 0) {
                atomicAdd(const_cast<int *>(L.jptr), 1);
                *gr.ticket = 0u;
            }
        }
    }
}

// z = sum_{k < kdim} y_k Z[k] (fma in k order) into the parent's slot, times
// D^-1/2 when returning to level 0.  A level whose input was non-finite
// returns NaN so that the outer level notices.  A thread loads its pack of
// every Z[k] (k < kdim <= MAXD) before the first fma, so the kdim loads are
// in flight together.
template <class T, class TP, int MAXD>
__global__ void __launch_bounds__(kVecBlock) k_combine(LevelDev<T> L, TP *out_base, const int *out_j, int out_ld,
                                                       const double *dsc) {
    pdl_enter();
    if (stopped(L.flags, L.depth - 1)) return;
    constexpr int N = PackN<T>::N;
    const int *fl = L.fl();
    const int k = fl[IF_KDIM];
    const bool nonfinite = fl[IF_NONFINITE] != 0 && k == 0;
    __shared__ T ys[kMaxDots];
    if (threadIdx.x < k) ys[threadIdx.x] = L.y()[threadIdx.x];
    __syncthreads();
    TP *out = out_base + (out_j ? (size_t)(*out_j) * out_ld : 0);
    auto one = [&](int i, T s) { out[i] = dsc ? (TP)mul_rn(dsc[i], (double)s) : (TP)s; };
    const bool vec = ((reinterpret_cast<uintptr_t>(out) & 15) == 0) && ((sizeof(TP) * N) % 16 == 0 || sizeof(TP) >= sizeof(T));
    const int nq = vec ? L.n / N : 0;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    for (int q = tid; q < nq; q += nth) {
        Pack<T, N> zl[MAXD];
#pragma unroll
        for (int l = 0; l < MAXD; ++l)
            if (l < k) zl[l] = ldp<T, N>(L.Z + (size_t)l * L.ld + (size_t)q * N);
        Pack<T, N> sum;
#pragma unroll
        for (int e = 0; e < N; ++e) sum.v[e] = (T)0;
#pragma unroll
        for (int l = 0; l < MAXD; ++l)
            if (l < k)
#pragma unroll
                for (int e = 0; e < N; ++e) sum.v[e] = fma_rn(ys[l], zl[l].v[e], sum.v[e]);
#pragma unroll
        for (int e = 0; e < N; ++e) one(q * N + e, nonfinite ? (T)NAN : sum.v[e]);
    }
    for (int i = nq * N + tid; i < L.n; i += nth) {
        T s = (T)0;
        for (int l = 0; l < k; ++l) s = fma_rn(ys[l], L.Z[(size_t)l * L.ld + i], s);
        one(i, nonfinite ? (T)NAN : s);
    }
}

// z = M v (primary preconditioner applied by the innermost FGMRES level)
// (v is addressed through the outer iteration index when in_j is given)
template <class T, class MS>
__global__ void __launch_bounds__(kBlock) k_apply_M(const MS *__restrict__ mv, const T *__restrict__ v_base,
                                                    const int *in_j, int ld, T *z, int n, const int *flags,
                                                    int check_depth, long long *m_count, int vround) {
    pdl_enter();
    if (stopped(flags, check_depth)) return;
    const T *__restrict__ v = v_base + (in_j ? (size_t)(*in_j) * ld : 0);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        z[i] = vstore(vround, mul_rn(to_c<T>(mv[i]), v[i]));
    if (blockIdx.x == 0 && threadIdx.x == 0 && m_count) atomicAdd((unsigned long long *)m_count, 1ull);
}

// ------------------------------------------------------------ outer (fp64) level
// Reductions with up to kMaxOuterM + 1 sums use partials laid out [d][block]
// and one warp per sum in the finishing block.
template <class T, class Fin>
__device__ __forceinline__ void grid_reduce_many(T *blocksum /*smem, nd*/, int nd, T *partials,
                                                 unsigned *ticket, Fin fin) {
    __shared__ bool am_last;
    for (int d = threadIdx.x; d < nd; d += blockDim.x) partials[(size_t)d * gridDim.x + blockIdx.x] = blocksum[d];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) am_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int d = warp; d < nd; d += nwarp) {
        T s = (T)0;
        for (int b = lane; b < (int)gridDim.x; b += 32) s = add_rn(s, __ldcg(partials + (size_t)d * gridDim.x + b));
        s = warp_sum(s);
        if (lane == 0) blocksum[d] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        fin(blocksum);
        *ticket = 0u;
    }
}

// block-level sum of `v` into smem slot `dst` (all threads participate)
template <class T> __device__ __forceinline__ void block_sum_into(T v, T *dst, T *scratch /*kWarps*/) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        T s = scratch[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) s = add_rn(s, scratch[w]);
        *dst = s;
    }
    __syncthreads();
}

// r = b - A x (original fp64 A), ||r||^2; with x == null, r = b.
// Finish: beta, rel = beta / ||b||; the level's g[0], inv.
static __global__ void __launch_bounds__(kBlock) k_outer_residual(Sell S, const double *__restrict__ a, const double *b,
                                                           const double *x, LevelDev<double> L, GridRed<double> gr,
                                                           int compute_nb) {
    pdl_enter();
    double acc[2] = {0.0, 0.0};
    const int lane = threadIdx.x & 31;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    double *r = L.w;
    for (int s = wid; s < S.nslices; s += nw) {
        const int i = s * kSlice + lane;
        double ax = x ? sell_row<double>(S, a, s, lane, [&](int c) { return __ldg(x + c); }) : 0.0;
        if (i < L.n) {
            const double bi = b[i];
            const double ri = sub_rn(bi, ax);
            r[i] = ri;
            acc[0] = fma_rn(ri, ri, acc[0]);
            acc[1] = fma_rn(bi, bi, acc[1]);
        }
    }
    grid_reduce<double, 2>(acc, 2, false, gr, [&](double *res) {
        double *ms = L.misc();
        int *fl = L.fl();
        if (compute_nb) ms[MS_NB] = sqrt_rn(res[1]);
        const double beta = sqrt_rn(res[0]);
        const double nb = ms[MS_NB];
        ms[MS_BETA] = beta;
        ms[MS_REL] = div_rn(beta, nb);
        fl[IF_KDIM] = 0;
        fl[IF_STOP] = 0;
        fl[IF_NONFINITE] = isfinite(beta) ? 0 : 1;
        *const_cast<int *>(L.jptr) = 0;
        if (beta > 0.0 && isfinite(beta)) {
            ms[MS_INV] = div_rn(1.0, beta);
            L.g()[0] = beta;
        }
    });
}

// w = A Z[j] with the original fp64 A (j read on the device)
static __global__ void __launch_bounds__(kBlock) k_outer_spmv(Sell S, const double *__restrict__ a, LevelDev<double> L) {
    pdl_enter();
    const int j = *L.jptr;
    const double *__restrict__ x = L.Z + (size_t)j * L.ld;
    const int lane = threadIdx.x & 31;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int s = wid; s < S.nslices; s += nw) {
        const double y = sell_row<double>(S, a, s, lane, [&](int c) { return __ldg(x + c); });
        const int i = s * kSlice + lane;
        if (i < L.n) L.w[i] = y;
    }
}

// MODE 0: hA = V^T w.  MODE 1: w -= V hA, then hB = V^T w.
// MODE 2: w -= V hB (hA when passes = 1), ||w||^2 -> Givens, estimate.
template <int MODE>
__global__ void __launch_bounds__(512) k_outer_cgs(LevelDev<double> L, int passes, double *partials,
                                                   unsigned *ticket) {
    pdl_enter();
    __shared__ double bs[kMaxOuterM + 2];
    __shared__ double scratch[16];
    __shared__ double hs[kMaxOuterM + 1];
    const int j = *L.jptr;
    const int nv = j + 1;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    if (MODE >= 1) {
        const double *h = (MODE == 1 || passes == 1) ? L.hA() : L.hB();
        for (int l = threadIdx.x; l < nv; l += blockDim.x) hs[l] = h[l];
        __syncthreads();
        for (int i = tid; i < L.n; i += nth) {
            double wi = L.w[i];
            for (int l = 0; l < nv; ++l) wi = fma_rn(-hs[l], L.V[(size_t)l * L.ld + i], wi);
            L.w[i] = wi;
        }
    }
    if (MODE <= 1) {
        // dot products in chunks of 8 vectors
        for (int l0 = 0; l0 < nv; l0 += 8) {
            double acc[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[q] = 0.0;
            for (int i = tid; i < L.n; i += nth) {
                const double wi = L.w[i];
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (l0 + q < nv) acc[q] = fma_rn(L.V[(size_t)(l0 + q) * L.ld + i], wi, acc[q]);
            }
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (l0 + q < nv) block_sum_into(acc[q], &bs[l0 + q], scratch);
        }
        grid_reduce_many(bs, nv, partials, ticket, [&](double *res) {
            double *h = (MODE == 0) ? L.hA() : L.hB();
            for (int l = 0; l < nv; ++l) h[l] = res[l];
        });
    } else {
        double acc = 0.0;
        for (int i = tid; i < L.n; i += nth) acc = fma_rn(L.w[i], L.w[i], acc);
        block_sum_into(acc, &bs[0], scratch);
        grid_reduce_many(bs, 1, partials, ticket, [&](double *res) {
            double hcol[kMaxOuterM + 1];
            const double *hA = L.hA(), *hB = L.hB();
            for (int l = 0; l < nv; ++l) hcol[l] = (passes == 2) ? add_rn(hA[l], hB[l]) : hA[l];
            const double hn = sqrt_rn(res[0]);
            givens_column(L, j, hcol, hn, false);
            double *ms = L.misc();
            ms[MS_EST] = div_rn(fabs(L.g()[L.fl()[IF_KDIM]]), ms[MS_NB]);
        });
    }
}

// y = R^-1 g over the kept columns (outer level, on exit of a cycle)
static __global__ void k_outer_solve_y(LevelDev<double> L) {
    pdl_enter();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int k = L.fl()[IF_KDIM];
    const int ldh = L.m + 1;
    const double *H = L.H(), *g = L.g();
    double *y = L.y();
    for (int r = k - 1; r >= 0; --r) {
        double s = g[r];
        for (int l = r + 1; l < k; ++l) s = fma_rn(-H[r + ldh * l], y[l], s);
        y[r] = div_rn(s, H[r + ldh * r]);
    }
}

// ------------------------------------------------ long inner levels (m > kMaxInnerM)
// An inner FGMRES level with more iterations than the fused dot registers
// hold (Table 4's F2: an inner FGMRES(64)) runs its CGS2 over the basis in
// groups of kLongGroup vectors per sweep of 16-byte packs: MODE 0: hA = V^T w;
// MODE 1: w -= V hA (fma in l order), then hB = V^T w; MODE 2: w -= V h (hB,
// or hA with one pass), ||w||^2 and max|w| -> Givens step and the child's
// 16-bit cast scale.  w = A Z[j] comes from the stand-alone SpMV.
constexpr int kLongGroup = 16;
constexpr int kLongBlock = 512;

template <class T, int MODE>
__global__ void __launch_bounds__(kLongBlock) k_long_cgs(LevelDev<T> L, int j, int passes, int last_iter,
                                                         int want_sigma, T *partials, unsigned *ticket, GridRed<T> gr) {
    pdl_enter();
    if (stopped(L.flags, L.depth)) return;
    constexpr int N = PackN<T>::N;
    __shared__ T bs[kMaxOuterM + 2];
    __shared__ T scratch[kLongBlock / 32];
    __shared__ T hs[kMaxOuterM + 1];
    const int nv = j + 1;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    const int nq = L.n / N;
    T *__restrict__ w = L.w;
    const T *__restrict__ V = L.V;
    const size_t ld = L.ld;
    T acc2[2] = {(T)0, (T)0};
    if (MODE >= 1) {
        const T *h = (MODE == 1 || passes == 1) ? L.hA() : L.hB();
        for (int l = threadIdx.x; l < nv; l += blockDim.x) hs[l] = h[l];
        __syncthreads();
        for (int q = tid; q < nq; q += nth) {
            Pack<T, N> wv = ldp<T, N>(w + (size_t)q * N);
            int l = 0;
            for (; l + 8 <= nv; l += 8) {
                Pack<T, N> v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = ldp<T, N>(V + (size_t)(l + u) * ld + (size_t)q * N);
#pragma unroll
                for (int u = 0; u < 8; ++u)
#pragma unroll
                    for (int e = 0; e < N; ++e) wv.v[e] = fma_rn(-hs[l + u], v[u].v[e], wv.v[e]);
            }
            for (; l < nv; ++l) {
                const Pack<T, N> v = ldp<T, N>(V + (size_t)l * ld + (size_t)q * N);
#pragma unroll
                for (int e = 0; e < N; ++e) wv.v[e] = fma_rn(-hs[l], v.v[e], wv.v[e]);
            }
            stp<T, N>(w + (size_t)q * N, wv);
            if (MODE == 2) {
#pragma unroll
                for (int e = 0; e < N; ++e) {
                    acc2[0] = fma_rn(wv.v[e], wv.v[e], acc2[0]);
                    acc2[1] = fmax(acc2[1], fabs(wv.v[e]));
                }
            }
        }
        for (int i = nq * N + tid; i < L.n; i += nth) {
            T wi = w[i];
            for (int l = 0; l < nv; ++l) wi = fma_rn(-hs[l], V[(size_t)l * ld + i], wi);
            w[i] = wi;
            if (MODE == 2) {
                acc2[0] = fma_rn(wi, wi, acc2[0]);
                acc2[1] = fmax(acc2[1], fabs(wi));
            }
        }
    }
    if (MODE <= 1) {
        for (int l0 = 0; l0 < nv; l0 += kLongGroup) {
            T acc[kLongGroup];
#pragma unroll
            for (int g = 0; g < kLongGroup; ++g) acc[g] = (T)0;
            for (int q = tid; q < nq; q += nth) {
                const Pack<T, N> wv = ldp<T, N>(w + (size_t)q * N);
#pragma unroll
                for (int g = 0; g < kLongGroup; ++g)
                    if (l0 + g < nv) {
                        const Pack<T, N> v = ldp<T, N>(V + (size_t)(l0 + g) * ld + (size_t)q * N);
#pragma unroll
                        for (int e = 0; e < N; ++e) acc[g] = fma_rn(v.v[e], wv.v[e], acc[g]);
                    }
            }
            for (int i = nq * N + tid; i < L.n; i += nth) {
                const T wi = w[i];
#pragma unroll
                for (int g = 0; g < kLongGroup; ++g)
                    if (l0 + g < nv) acc[g] = fma_rn(V[(size_t)(l0 + g) * ld + i], wi, acc[g]);
            }
#pragma unroll
            for (int g = 0; g < kLongGroup; ++g)
                if (l0 + g < nv) block_sum_into(acc[g], &bs[l0 + g], scratch);
        }
        grid_reduce_many(bs, nv, partials, ticket, [&](T *res) {
            T *h = (MODE == 0) ? L.hA() : L.hB();
            for (int l = 0; l < nv; ++l) h[l] = res[l];
        });
    } else {
        grid_reduce<T, 2>(acc2, 1, true, gr, [&](T *res) {
            T hcol[kMaxOuterM + 1];
            const T *hA = L.hA(), *hB = L.hB();
            for (int l = 0; l < nv; ++l) hcol[l] = (passes == 2) ? add_rn(hA[l], hB[l]) : hA[l];
            const T hn = sqrt_rn(res[0]);
            givens_column(L, j, hcol, hn, last_iter != 0);
            T *ms = L.misc();
            if (want_sigma && hn > (T)0) {
                const T sig = pow2_scale_for(mul_rn(res[1], ms[MS_INV]));
                ms[MS_SIGMA] = sig;
                ms[MS_INV_SIGMA] = div_rn((T)1, sig);
            } else {
                ms[MS_SIGMA] = (T)1;
                ms[MS_INV_SIGMA] = (T)1;
            }
        });
    }
}

// z = sum_{k < kdim} y_k Z[k] (fma in k order) into the parent's slot of a
// long level, times D^-1/2 when returning to level 0 (as k_combine)
template <class T, class TP>
__global__ void __launch_bounds__(kVecBlock) k_combine_long(LevelDev<T> L, TP *out, const double *dsc) {
    pdl_enter();
    if (stopped(L.flags, L.depth - 1)) return;
    const int *fl = L.fl();
    const int k = fl[IF_KDIM];
    const bool nonfinite = fl[IF_NONFINITE] != 0 && k == 0;
    __shared__ T ys[kMaxOuterM];
    for (int l = threadIdx.x; l < k; l += blockDim.x) ys[l] = L.y()[l];
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L.n; i += gridDim.x * blockDim.x) {
        T s = (T)0;
        for (int l = 0; l < k; ++l) s = fma_rn(ys[l], L.Z[(size_t)l * L.ld + i], s);
        if (nonfinite) s = (T)NAN;
        out[i] = dsc ? (TP)mul_rn(dsc[i], (double)s) : (TP)s;
    }
}

// x += sum_{k < kdim} y_k Z[k]
static __global__ void __launch_bounds__(kBlock) k_outer_update_x(LevelDev<double> L, double *x) {
    pdl_enter();
    __shared__ double ys[kMaxOuterM];
    const int k = L.fl()[IF_KDIM];
    for (int l = threadIdx.x; l < k; l += blockDim.x) ys[l] = L.y()[l];
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L.n; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int l = 0; l < k; ++l) s = fma_rn(ys[l], L.Z[(size_t)l * L.ld + i], s);
        x[i] = add_rn(x[i], s);
    }
}

}  // namespace f3r
