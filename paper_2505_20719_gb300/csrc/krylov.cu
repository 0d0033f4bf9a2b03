// The paper's Krylov comparators on the GPU (Sec. 5: preconditioned CG for
// symmetric and BiCGStab for nonsymmetric systems, all in fp64), with the
// same preconditioner the F3R nest wraps: P = D^-1/2 M D^-1/2, M the stored
// Jacobi preconditioner of A^ (m_prec storage), on the original fp64 matrix.
//
// CG (Saad, Iterative Methods for Sparse Linear Systems, Alg. 9.1), two
// kernels per iteration:
//   K_q  q = A p, (p, q) -> alpha                      (p of the gather:
//        p_c = z_c + beta p'_c from the previous z and p', double-buffered)
//   K_x  x += alpha p, r -= alpha q, z = P r, (r, z), (r, r) -> beta, done
// BiCGStab (van der Vorst; Saad Alg. 7.7 with right preconditioning), five:
//   B_p  p = r + beta (p - omega v), p^ = P p
//   B_v  v = A p^, (r0^, v) -> alpha
//   B_s  s = r - alpha v, s^ = P s
//   B_t  t = A s^, (t, s), (t, t) -> omega
//   B_x  x += alpha p^ + omega s^, r = s - omega t, (r0^, r), (r, r) -> beta, done
// Every reduction is the deterministic grid reduction; a device flag ends
// the iteration (later kernels of a captured batch return at once), and the
// host replays CUDA graphs of kKrylovBatch iterations.
#include <cmath>
#include <cstring>

#include "ctx.h"
#include "kernels.cuh"

namespace f3r {

namespace {

// fp64 row sum of a slice exactly W entries wide: W gathers, then W fused
// multiply-adds in CSR order (no slot past the width)
template <int W, class GX>
__device__ __forceinline__ double kry_row_w(const Sell &S, const double *__restrict__ a, int beg, GX gx) {
    int c[W];
    double v[W], xv[W];
#pragma unroll
    for (int q = 0; q < W; ++q) {
        c[q] = __ldg(S.col + beg + (q << 5));
        v[q] = __ldg(a + beg + (q << 5));
    }
#pragma unroll
    for (int q = 0; q < W; ++q) xv[q] = (c[q] >= 0) ? gx(c[q]) : 0.0;
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < W; ++q)
        if (c[q] >= 0) acc = fma_rn(v[q], xv[q], acc);
    return acc;
}

// the same row sum as sell_row, with exact-width code for slices up to 8 wide
template <class GX>
__device__ __forceinline__ double kry_row(const Sell &S, const double *__restrict__ a, int s, int lane, GX gx) {
    const int beg = __ldg(S.sptr + s) + lane;
    switch ((__ldg(S.sptr + s + 1) - __ldg(S.sptr + s)) >> 5) {
        case 0: return 0.0;
        case 1: return kry_row_w<1>(S, a, beg, gx);
        case 2: return kry_row_w<2>(S, a, beg, gx);
        case 3: return kry_row_w<3>(S, a, beg, gx);
        case 4: return kry_row_w<4>(S, a, beg, gx);
        case 5: return kry_row_w<5>(S, a, beg, gx);
        case 6: return kry_row_w<6>(S, a, beg, gx);
        case 7: return kry_row_w<7>(S, a, beg, gx);
        case 8: return kry_row_w<8>(S, a, beg, gx);
        default: return sell_row<double>(S, a, s, lane, gx);
    }
}

constexpr int kKrylovBatch = 16;  // iterations per graph replay
constexpr int kHistCap = 1 << 20;

enum { KS_RHO = 0, KS_ALPHA, KS_OMEGA, KS_BETA, KS_RR, KS_BB, KS_TOL2, KS_COUNT };
enum { KF_DONE = 0, KF_ITERS, KF_BREAK, KF_CAP, KF_COUNT };

struct KrylovDev {
    int n;
    const double *dsc;  // D^-1/2
    const void *mvec;   // M (m_prec)
    int m_prec;
    double *x, *r, *rh, *p[2], *ph, *v, *s, *sh, *t, *q, *z;
    double *sc;         // scalars
    int *fl;            // flags
    double *hist;       // ||r|| / ||b|| per iteration
};

__device__ __forceinline__ double mval(const KrylovDev &K, int i) {
    switch (K.m_prec) {
        case F3R_F64: return ((const double *)K.mvec)[i];
        case F3R_F32: return (double)((const float *)K.mvec)[i];
        case F3R_F16: return (double)__half2float(((const h16 *)K.mvec)[i]);
        default: return (double)__bfloat162float(((const b16 *)K.mvec)[i]);
    }
}
// (P y)_i = d_i (m_i (d_i y_i))
__device__ __forceinline__ double papply(const KrylovDev &K, int i, double y) {
    const double d = K.dsc[i];
    return mul_rn(d, mul_rn(mval(K, i), mul_rn(d, y)));
}

__device__ __forceinline__ bool kdone(const KrylovDev &K) { return ((volatile const int *)K.fl)[KF_DONE] != 0; }

// r = b - A x, z = P r, p = z (CG) / r^ = r, p = 0, v = 0 (BiCGStab); (r, z), (r, r), (b, b)
__global__ void __launch_bounds__(kBlock) k_kry_init(Sell S, const double *__restrict__ a, const double *b,
                                                     KrylovDev K, int method, double tol, int cap,
                                                     GridRed<double> gr) {
    double acc[3] = {0.0, 0.0, 0.0};
    const int lane = threadIdx.x & 31;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int s = wid; s < S.nslices; s += nw) {
        const double ax = kry_row(S, a, s, lane, [&](int c) { return __ldg(K.x + c); });
        const int i = s * kSlice + lane;
        if (i < K.n) {
            const double ri = sub_rn(b[i], ax);
            K.r[i] = ri;
            if (method == 1) {
                const double zi = papply(K, i, ri);
                K.z[i] = zi;
                K.p[1][i] = 0.0;  // the "previous" direction of iteration 0 (beta = 0)
                acc[0] = fma_rn(ri, zi, acc[0]);
            } else {
                K.rh[i] = ri;
                K.p[0][i] = 0.0;
                K.v[i] = 0.0;
                acc[0] = fma_rn(ri, ri, acc[0]);
            }
            acc[1] = fma_rn(ri, ri, acc[1]);
            acc[2] = fma_rn(b[i], b[i], acc[2]);
        }
    }
    grid_reduce<double, 3>(acc, 3, false, gr, [&](double *res) {
        K.sc[KS_RHO] = res[0];
        K.sc[KS_RR] = res[1];
        K.sc[KS_BB] = res[2];
        K.sc[KS_ALPHA] = 1.0;
        K.sc[KS_OMEGA] = 1.0;
        K.sc[KS_BETA] = 0.0;
        K.sc[KS_TOL2] = mul_rn(mul_rn(tol, tol), res[2]);
        K.fl[KF_ITERS] = 0;
        K.fl[KF_BREAK] = 0;
        K.fl[KF_CAP] = cap;
        K.fl[KF_DONE] = (res[1] <= K.sc[KS_TOL2] || cap <= 0) ? 1 : 0;
    });
}

// ---------------------------------------------------------------- CG
// Iteration k keeps its search direction p_k in p[k % 2].  q = A p_k with
// p_k = z + beta p_{k-1} formed in the gather from p[(k - 1) % 2] (every
// block writes p_k only for its own rows, into the other buffer), and
// (p_k, q) -> alpha.  Iteration 0 sees p_{-1} = 0 and beta = 0.
__global__ void __launch_bounds__(kBlock) k_cg_q(Sell S, const double *__restrict__ a, KrylovDev K, int cur,
                                                 GridRed<double> gr) {
    if (kdone(K)) return;
    const double beta = K.sc[KS_BETA];
    const double *__restrict__ pp = K.p[cur ^ 1];
    double *pn = K.p[cur];
    double acc[1] = {0.0};
    const int lane = threadIdx.x & 31;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    auto pdir = [&](int c) { return fma_rn(beta, __ldg(pp + c), __ldg(K.z + c)); };
    for (int s = wid; s < S.nslices; s += nw) {
        const double qi = kry_row(S, a, s, lane, pdir);
        const int i = s * kSlice + lane;
        if (i < K.n) {
            const double pi = pdir(i);
            K.q[i] = qi;
            pn[i] = pi;
            acc[0] = fma_rn(pi, qi, acc[0]);
        }
    }
    grid_reduce<double, 1>(acc, 1, false, gr, [&](double *res) {
        const double pq = res[0];
        if (!(pq != 0.0) || !isfinite(pq)) {
            K.fl[KF_BREAK] = 1;
            K.fl[KF_DONE] = 1;
            K.sc[KS_ALPHA] = 0.0;
        } else {
            K.sc[KS_ALPHA] = div_rn(K.sc[KS_RHO], pq);
        }
    });
}

// x += alpha p_k, r -= alpha q, z = P r; (r, z) -> beta, (r, r) -> done
__global__ void __launch_bounds__(kBlock) k_cg_x(KrylovDev K, int cur, GridRed<double> gr) {
    if (kdone(K)) return;
    const double alpha = K.sc[KS_ALPHA];
    const double *p = K.p[cur];
    double acc[2] = {0.0, 0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K.n; i += gridDim.x * blockDim.x) {
        K.x[i] = fma_rn(alpha, p[i], K.x[i]);
        const double ri = fma_rn(-alpha, K.q[i], K.r[i]);
        K.r[i] = ri;
        const double zi = papply(K, i, ri);
        K.z[i] = zi;
        acc[0] = fma_rn(ri, zi, acc[0]);
        acc[1] = fma_rn(ri, ri, acc[1]);
    }
    grid_reduce<double, 2>(acc, 2, false, gr, [&](double *res) {
        const double rho = K.sc[KS_RHO];
        K.sc[KS_BETA] = div_rn(res[0], rho);
        K.sc[KS_RHO] = res[0];
        K.sc[KS_RR] = res[1];
        const int it = K.fl[KF_ITERS] + 1;
        K.fl[KF_ITERS] = it;
        if (it - 1 < kHistCap) K.hist[it - 1] = sqrt_rn(div_rn(res[1], K.sc[KS_BB]));
        if (res[1] <= K.sc[KS_TOL2] || !isfinite(res[1]) || it >= K.fl[KF_CAP]) K.fl[KF_DONE] = 1;
    });
}

// ------------------------------------------------------------ BiCGStab
__global__ void __launch_bounds__(kBlock) k_bs_p(KrylovDev K) {
    if (kdone(K)) return;
    const double beta = K.sc[KS_BETA], omega = K.sc[KS_OMEGA];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K.n; i += gridDim.x * blockDim.x) {
        const double pi = fma_rn(beta, fma_rn(-omega, K.v[i], K.p[0][i]), K.r[i]);
        K.p[0][i] = pi;
        K.ph[i] = papply(K, i, pi);
    }
}

// y = A src; with mode 0: (r0^, y) -> alpha = rho / (r0^, y); mode 1: (y, s), (y, y) -> omega
__global__ void __launch_bounds__(kBlock) k_bs_spmv(Sell S, const double *__restrict__ a, KrylovDev K, int mode,
                                                    GridRed<double> gr) {
    if (kdone(K)) return;
    const double *__restrict__ src = mode == 0 ? K.ph : K.sh;
    double *y = mode == 0 ? K.v : K.t;
    double acc[2] = {0.0, 0.0};
    const int lane = threadIdx.x & 31;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int s = wid; s < S.nslices; s += nw) {
        const double yi = kry_row(S, a, s, lane, [&](int c) { return __ldg(src + c); });
        const int i = s * kSlice + lane;
        if (i < K.n) {
            y[i] = yi;
            if (mode == 0) {
                acc[0] = fma_rn(K.rh[i], yi, acc[0]);
            } else {
                acc[0] = fma_rn(yi, K.s[i], acc[0]);
                acc[1] = fma_rn(yi, yi, acc[1]);
            }
        }
    }
    grid_reduce<double, 2>(acc, mode == 0 ? 1 : 2, false, gr, [&](double *res) {
        if (mode == 0) {
            if (!(res[0] != 0.0) || !isfinite(res[0])) {
                K.fl[KF_BREAK] = 1;
                K.fl[KF_DONE] = 1;
            } else {
                K.sc[KS_ALPHA] = div_rn(K.sc[KS_RHO], res[0]);
            }
        } else {
            // omega = (t, s) / (t, t); t = 0 means s = 0 (then omega is not used)
            K.sc[KS_OMEGA] = (res[1] > 0.0) ? div_rn(res[0], res[1]) : 0.0;
        }
    });
}

__global__ void __launch_bounds__(kBlock) k_bs_s(KrylovDev K) {
    if (kdone(K)) return;
    const double alpha = K.sc[KS_ALPHA];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K.n; i += gridDim.x * blockDim.x) {
        const double si = fma_rn(-alpha, K.v[i], K.r[i]);
        K.s[i] = si;
        K.sh[i] = papply(K, i, si);
    }
}

__global__ void __launch_bounds__(kBlock) k_bs_x(KrylovDev K, GridRed<double> gr) {
    if (kdone(K)) return;
    const double alpha = K.sc[KS_ALPHA], omega = K.sc[KS_OMEGA];
    double acc[2] = {0.0, 0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K.n; i += gridDim.x * blockDim.x) {
        K.x[i] = fma_rn(omega, K.sh[i], fma_rn(alpha, K.ph[i], K.x[i]));
        const double ri = fma_rn(-omega, K.t[i], K.s[i]);
        K.r[i] = ri;
        acc[0] = fma_rn(K.rh[i], ri, acc[0]);
        acc[1] = fma_rn(ri, ri, acc[1]);
    }
    grid_reduce<double, 2>(acc, 2, false, gr, [&](double *res) {
        const double rho = K.sc[KS_RHO], alpha = K.sc[KS_ALPHA], omega = K.sc[KS_OMEGA];
        const int it = K.fl[KF_ITERS] + 1;
        K.fl[KF_ITERS] = it;
        K.sc[KS_RR] = res[1];
        if (it - 1 < kHistCap) K.hist[it - 1] = sqrt_rn(div_rn(res[1], K.sc[KS_BB]));
        if (res[1] <= K.sc[KS_TOL2] || !isfinite(res[1]) || it >= K.fl[KF_CAP]) {
            K.fl[KF_DONE] = 1;
        } else if (!(res[0] != 0.0) || !(omega != 0.0)) {
            K.fl[KF_BREAK] = 1;  // rho = 0 or omega = 0: BiCGStab breaks down
            K.fl[KF_DONE] = 1;
        } else {
            K.sc[KS_BETA] = mul_rn(div_rn(res[0], rho), div_rn(alpha, omega));
            K.sc[KS_RHO] = res[0];
        }
    });
}

// true relative residual ||b - A x|| / ||b|| into sc[KS_RR] (as a ratio)
__global__ void __launch_bounds__(kBlock) k_kry_true(Sell S, const double *__restrict__ a, const double *b,
                                                     KrylovDev K, GridRed<double> gr) {
    double acc[2] = {0.0, 0.0};
    const int lane = threadIdx.x & 31;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int s = wid; s < S.nslices; s += nw) {
        const double ax = kry_row(S, a, s, lane, [&](int c) { return __ldg(K.x + c); });
        const int i = s * kSlice + lane;
        if (i < K.n) {
            const double ri = sub_rn(b[i], ax);
            acc[0] = fma_rn(ri, ri, acc[0]);
            acc[1] = fma_rn(b[i], b[i], acc[1]);
        }
    }
    grid_reduce<double, 2>(acc, 2, false, gr, [&](double *res) {
        K.sc[KS_RR] = (res[1] > 0.0) ? sqrt_rn(div_rn(res[0], res[1])) : 0.0;
    });
}

struct KrylovHost {
    double *buf = nullptr;  // all vectors
    double *sc = nullptr, *hist = nullptr;
    int *fl = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // CG, BiCGStab batches
    const double *graph_x[2] = {nullptr, nullptr};  // the x each graph was captured with
    std::vector<void *> owned;
};

void kry_release(KrylovHost *k) {
    for (auto &g : k->graph)
        if (g) cudaGraphExecDestroy(g);
    for (void *p : k->owned) cudaFree(p);
    delete k;
}

constexpr int kKrylovVectors = 11;

KrylovHost *kry_state(Ctx &c) {
    static_assert(KS_COUNT <= 8 && KF_COUNT <= 4, "scalar blocks");
    if (c.krylov) return (KrylovHost *)c.krylov;
    KrylovHost *k = new (std::nothrow) KrylovHost;
    if (!k) return nullptr;
    const size_t sizes[4] = {sizeof(double) * (size_t)c.ld * kKrylovVectors, sizeof(double) * 8,
                             sizeof(int) * 4, sizeof(double) * kHistCap};
    void *ptr[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int q = 0; q < 4; ++q) {
        if (cudaMalloc(&ptr[q], sizes[q]) != cudaSuccess) {
            cudaGetLastError();
            kry_release(k);
            return nullptr;
        }
        k->owned.push_back(ptr[q]);
        c.bytes += (long long)sizes[q];
    }
    k->buf = (double *)ptr[0];
    k->sc = (double *)ptr[1];
    k->fl = (int *)ptr[2];
    k->hist = (double *)ptr[3];
    c.krylov = k;
    return k;
}

KrylovDev kry_dev(Ctx &c, KrylovHost &k, double *x) {
    KrylovDev K;
    K.n = c.n;
    K.dsc = c.dsc;
    K.mvec = c.mvec;
    K.m_prec = c.prm.m_prec;
    double *b = k.buf;
    const size_t ld = c.ld;
    K.x = x;
    K.r = b;
    K.rh = b + ld;
    K.p[0] = b + 2 * ld;
    K.p[1] = b + 3 * ld;
    K.ph = b + 4 * ld;
    K.v = b + 5 * ld;
    K.s = b + 6 * ld;
    K.sh = b + 7 * ld;
    K.t = b + 8 * ld;
    K.q = b + 9 * ld;
    K.z = b + 10 * ld;
    K.sc = k.sc;
    K.fl = k.fl;
    K.hist = k.hist;
    return K;
}

// kKrylovBatch iterations (an even number, so iteration parity = batch-local parity)
void kry_batch(Ctx &c, const KrylovDev &K, int method, cudaStream_t s) {
    const Sell S = sell_of(c);
    GridRed<double> gr{(double *)c.partials, c.ticket, kMaxDots};
    for (int it = 0; it < kKrylovBatch; ++it) {
        if (method == 1) {
            const int cur = it & 1;
            k_cg_q<<<c.Gs, kBlock, 0, s>>>(S, c.a64, K, cur, gr);
            k_cg_x<<<c.G, kBlock, 0, s>>>(K, cur, gr);
            c.launches += 2;
        } else {
            k_bs_p<<<c.G, kBlock, 0, s>>>(K);
            k_bs_spmv<<<c.Gs, kBlock, 0, s>>>(S, c.a64, K, 0, gr);
            k_bs_s<<<c.G, kBlock, 0, s>>>(K);
            k_bs_spmv<<<c.Gs, kBlock, 0, s>>>(S, c.a64, K, 1, gr);
            k_bs_x<<<c.G, kBlock, 0, s>>>(K, gr);
            c.launches += 5;
        }
    }
}

}  // namespace

void krylov_free(Ctx &c) {
    if (!c.krylov) return;
    kry_release((KrylovHost *)c.krylov);
    c.krylov = nullptr;
}

f3r_status krylov_solve(Ctx &c, cudaStream_t s, int method, const double *b, double *x, int max_iters,
                        f3r_stats *stats) {
    if (method != 1 && method != 2) return F3R_ERR_ARG;
    if (max_iters < 0) return F3R_ERR_ARG;
    KrylovHost *k = kry_state(c);
    if (!k) return F3R_ERR_NOMEM;
    const KrylovDev K = kry_dev(c, *k, x);
    GridRed<double> gr{(double *)c.partials, c.ticket, kMaxDots};
    const Sell S = sell_of(c);
    const long long launches0 = c.launches;
    // the batch graph holds x in its kernel arguments: captured again when x changes
    cudaGraphExec_t &ge = k->graph[method - 1];
    if (c.prm.use_graphs && (!ge || k->graph_x[method - 1] != x)) {
        if (ge) {
            cudaGraphExecDestroy(ge);
            ge = nullptr;
        }
        cudaGraph_t g = nullptr;
        const long long l0 = c.launches;
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return F3R_ERR_CUDA;
        kry_batch(c, K, method, s);
        if (cudaStreamEndCapture(s, &g) != cudaSuccess) return F3R_ERR_CUDA;
        const cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return F3R_ERR_CUDA;
        c.launches = l0;
        k->graph_x[method - 1] = x;
    }
    const long long per_batch = (method == 1 ? 2 : 5) * kKrylovBatch;
    int h_fl[KF_COUNT] = {0, 0, 0};
    int batches = 0, iters = 0, starts = 0;
    double rel = 0.0;
    // The recurrence's residual can drift from b - A x: when it claims
    // convergence the true residual decides, and the iteration starts again
    // from the current x (at most 3 times).
    for (; starts < 4; ++starts) {
        k_kry_init<<<c.Gs, kBlock, 0, s>>>(S, c.a64, b, K, method, c.prm.tol, max_iters - iters, gr);
        c.launches++;
        for (;;) {
            if (cudaMemcpyAsync(h_fl, k->fl, sizeof(int) * KF_COUNT, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return F3R_ERR_CUDA;
            if (h_fl[KF_DONE]) break;
            if (c.prm.use_graphs) {
                if (cudaGraphLaunch(ge, s) != cudaSuccess) return F3R_ERR_CUDA;
                c.launches += per_batch;
            } else {
                kry_batch(c, K, method, s);
            }
            ++batches;
        }
        iters += h_fl[KF_ITERS];
        k_kry_true<<<c.Gs, kBlock, 0, s>>>(S, c.a64, b, K, gr);
        c.launches++;
        cudaMemcpyAsync(&rel, k->sc + KS_RR, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return F3R_ERR_CUDA;
        if (!(rel >= c.prm.tol) || h_fl[KF_BREAK] || iters >= max_iters) break;
    }
    f3r_status status = F3R_OK;
    if (!std::isfinite(rel)) status = F3R_ERR_NONFINITE;
    else if (rel >= c.prm.tol) status = h_fl[KF_BREAK] ? F3R_ERR_BREAKDOWN : F3R_NOT_CONVERGED;
    if (stats) {
        stats->status = status;
        stats->outer_iters = iters;
        stats->restarts = starts < 4 ? starts : 3;
        stats->rel_res_true = rel;
        stats->m_applies = (int64_t)iters * (method == 1 ? 1 : 2);
        stats->r_calls = 0;
        stats->r_update_calls = 0;
        for (int q = 0; q < 8; ++q) stats->omega[q] = 0.0;
        const int nh = std::min(h_fl[KF_ITERS], std::min(stats->hist_cap, kHistCap));
        if (stats->hist && nh > 0) cudaMemcpy(stats->hist, k->hist, sizeof(double) * nh, cudaMemcpyDeviceToHost);
        stats->hist_len = h_fl[KF_ITERS];
        stats->true_len = 0;
        if (stats->true_hist && stats->true_cap > 0) {
            stats->true_hist[0] = rel;
            stats->true_len = 1;
        }
        stats->t_solve_ms = 0.0;
        stats->kernel_launches = c.launches - launches0;
        stats->graph_launches = c.prm.use_graphs ? batches : 0;
    }
    return cudaGetLastError() == cudaSuccess ? status : F3R_ERR_CUDA;
}

}  // namespace f3r
