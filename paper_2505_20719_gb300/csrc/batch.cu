// Batched F3R: many systems and right-hand sides in one persistent launch.
//
// Every (system, right-hand side) instance is solved entirely on the device
// by a team: one thread-block cluster, or for the large systems a wide team
// of several clusters.  A team runs the outer fp64 FGMRES(m1) with its
// convergence test and restarts, the fp32 FGMRES(m2), the FGMRES(m3) with
// fp16 A and the fp16 Richardson R_2 with adaptive weights (Sec. 4.2,
// Table 1, Algorithm 1) -- the same arithmetic as the single-system path.
// Kernel boundaries become cluster barriers (barrier.cluster), plus, in a
// wide team, a bounded barrier of the clusters in global memory; reductions
// sum per-block partials in distributed shared memory in a fixed rank order
// (and a wide team's cluster sums in cluster order); the small Givens /
// least-squares state of the inner levels is kept, and updated identically,
// in every block of the team.  Teams take instances from atomic work queues
// ordered by size (largest first).  All control decisions derive from values
// every block of a team holds identically, so every block reaches every
// barrier.
//
// Data written inside the launch is read with ld.global.cg (L2), never through
// the non-coherent read-only path.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <map>
#include <vector>

#include "ctx.h"
#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace f3r {
namespace bt {

constexpr int kBT = 512;          // threads per block at most (256 or 512, chosen by the autotuner)
constexpr int kBW = kBT / 32;     // warps per block at most
constexpr int kMaxCluster = 8;
constexpr int kRedMax = 16;       // sums per team reduction
constexpr int kMaxClustersPerSM = 4;  // clusters of a launch per SM at most (2048 threads per SM)

struct Sys {
    int n, nslices;
    const int *sptr, *col;
    const double *a64;   // original A
    const float *a32;    // A^ fp32
    const h16 *a16;      // A^ fp16
    const double *dsc;   // D^-1/2
    const h16 *m16;      // Jacobi M
    int m_unit;          // every entry of M is exactly 1: M v = v, M is not loaded
};

struct Inst {
    int sys;
    const double *b;
    double *x;
    double *V1, *Z1, *w1, *H1;  // H1: (m1+1) m1 + 4 m1 + 2 doubles (H, cs, sn, g, y)
    float *V2, *Z2, *w2;
    float *V3, *Z3, *w3;
    h16 *rin, *rz, *rr;
    int ld;
};

struct Out {
    int status, outer_iters, restarts;
    double rel;
    long long m_applies, r_calls;
};

struct BP {
    int m1, m2, m3, c, max_outer, cgs_passes, scale_cast;
    double tol;
    float omega_fixed;
};

// per-level least-squares state of an inner level, replicated in every block
struct LS {
    float H[(kMaxInnerM + 1) * kMaxInnerM];
    float cs[kMaxInnerM], sn[kMaxInnerM], g[kMaxInnerM + 1], y[kMaxInnerM];
    float hA[kMaxDots], hB[kMaxDots];
    float beta, inv, sigma, inv_sigma;
    int kdim, stop, nonfinite;
};

struct Shared {
    double red_blk[2][kRedMax];  // this block's partial sums (two buffers, alternating)
    double red_res[kRedMax];     // the team's sums, formed by every block itself
    double wred[kRedMax][kBW];
    int red_buf;                 // buffer of the next reduction
    LS ls2, ls3;
    float omega[2];
    long long c_ntr;
    // rank 0: outer-level decisions broadcast to the team
    double o_inv, o_est, o_beta, o_rel;
    int o_stop, o_kdim, o_nonfinite, inst;
};

// A team solves one instance: one cluster, or (a wide team, for the large
// systems) k clusters that meet at a barrier in global memory.  rank / size
// count the team's blocks (cluster kidx holds ranks kidx * csize ..), crank /
// csize the blocks of this cluster.
struct Team {
    unsigned rank, size;
    unsigned crank, csize;
    int k, kidx;
    int tid, nthr, wid, nwarps, lane;
    unsigned *bar;   // wide teams: [0] arrivals, [1] generation
    double *part;    // wide teams: [2][k][kRedMax] cluster sums of the reductions
    double *dec;     // wide teams: decisions of the team's rank 0 ([0..7]) and the instance ([8])
    int *abort;      // set when a wide barrier gave up; later wide barriers do not wait
};

constexpr long long kWideWaitCycles = 8000000000LL;  // ~4 s at the 2.07 GHz SM clock

__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// The k clusters of a wide team meet (one thread of each, after its cluster
// barrier): arrivals counted in bar[0], the last arriver resets it and
// advances the generation bar[1] the others poll.  The wait is bounded: on
// giving up it sets *abort, and no later wide barrier waits (the launch then
// ends with unreliable results for the wide instances, reported as
// F3R_ERR_TIMEOUT, instead of hanging).
__device__ void wide_barrier(const Team &tm) {
    unsigned *cnt = tm.bar, *gen = tm.bar + 1;
    const unsigned g = ld_acquire_gpu(gen);
    __threadfence();  // this cluster's writes (ordered by its cluster barrier) before the arrival
    if (atomicAdd(cnt, 1u) == (unsigned)tm.k - 1) {
        atomicExch(cnt, 0u);
        __threadfence();
        atomicAdd(gen, 1u);
    } else {
        const long long t0 = clock64();
        while (ld_acquire_gpu(gen) == g) {
            if (*(volatile int *)tm.abort) break;
            if (clock64() - t0 > kWideWaitCycles) {
                atomicExch(tm.abort, 1);
                break;
            }
            __nanosleep(100);
        }
    }
    __threadfence();
}

// barrier of the whole team
__device__ __forceinline__ void team_sync(const Team &tm) {
    cluster_sync();
    if (tm.k > 1) {
        if (tm.crank == 0 && threadIdx.x == 0) wide_barrier(tm);
        cluster_sync();
    }
}

template <class T> __device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }
__device__ __forceinline__ h16 ldcg(const h16 *p) {
    unsigned short u = __ldcg(reinterpret_cast<const unsigned short *>(p));
    return __ushort_as_half(u);
}

// Deterministic team reduction of nd sums (nd <= kRedMax), or maxima where
// is_max; every thread of the team returns the results in out[].  Each block
// writes its partials, one cluster barrier, then every block sums all ranks'
// partials in rank order itself (the same order everywhere, so the same
// result).  The partials alternate between two buffers: a block still
// reading the previous reduction's buffer cannot be overtaken, because the
// next write to that buffer follows one more cluster barrier.
template <class T>
__device__ void team_reduce(const Team &tm, Shared &sh, T *acc, int nd, T *out, const bool *is_max = nullptr) {
    cg::cluster_group cl = cg::this_cluster();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int buf = sh.red_buf;
    for (int d = 0; d < nd; ++d) {
        const bool mx = is_max && is_max[d];
        T v = mx ? warp_max(acc[d]) : warp_sum(acc[d]);
        if (lane == 0) sh.wred[d][warp] = (double)v;
    }
    __syncthreads();
    if (threadIdx.x < nd) {
        const int d = threadIdx.x;
        const bool mx = is_max && is_max[d];
        T s = (T)sh.wred[d][0];
        const int nw = (int)(blockDim.x >> 5);  // 256 or 512 threads per block
        for (int w = 1; w < nw; ++w) s = mx ? fmax(s, (T)sh.wred[d][w]) : add_rn(s, (T)sh.wred[d][w]);
        sh.red_blk[buf][d] = (double)s;
    }
    cluster_sync();
    if (threadIdx.x < nd) {
        const int d = threadIdx.x;
        const bool mx = is_max && is_max[d];
        T s = (T)0;
        for (unsigned r = 0; r < tm.csize; ++r) {
            const double *rb = cl.map_shared_rank(&sh.red_blk[buf][0], r);
            s = (r == 0) ? (T)rb[d] : (mx ? fmax(s, (T)rb[d]) : add_rn(s, (T)rb[d]));
        }
        sh.red_res[d] = (double)s;
    }
    if (tm.k > 1) {
        // the cluster sums through global memory, summed in cluster order by every block
        double *pb = tm.part + (size_t)buf * tm.k * kRedMax;
        if (tm.crank == 0 && threadIdx.x < nd) pb[(size_t)tm.kidx * kRedMax + threadIdx.x] = sh.red_res[threadIdx.x];
        team_sync(tm);
        if (threadIdx.x < nd) {
            const int d = threadIdx.x;
            const bool mx = is_max && is_max[d];
            T s = (T)0;
            for (int c = 0; c < tm.k; ++c) {
                const T v = (T)__ldcg(pb + (size_t)c * kRedMax + d);
                s = (c == 0) ? v : (mx ? fmax(s, v) : add_rn(s, v));
            }
            sh.red_res[d] = (double)s;
        }
    }
    __syncthreads();
    for (int d = 0; d < nd; ++d) out[d] = (T)sh.red_res[d];
    __syncthreads();
    if (threadIdx.x == 0) sh.red_buf = buf ^ 1;
    __syncthreads();
}

// ---------------------------------------------------------------- Givens
// Saad 6.5.3 update of an inner level with column j; identical in every block.
__device__ void ls_column(LS &L, int m, int j, const float *hcol, float hn, bool last) {
    const int ldh = m + 1;
    bool finite = isfinite(hn);
    for (int i = 0; i <= j; ++i) finite = finite && isfinite(hcol[i]);
    bool ok = finite;
    if (ok) {
        for (int i = 0; i <= j; ++i) L.H[i + ldh * j] = hcol[i];
        L.H[j + 1 + ldh * j] = hn;
        for (int i = 0; i < j; ++i) {
            const float t = add_rn(mul_rn(L.cs[i], L.H[i + ldh * j]), mul_rn(L.sn[i], L.H[i + 1 + ldh * j]));
            L.H[i + 1 + ldh * j] = add_rn(mul_rn(-L.sn[i], L.H[i + ldh * j]), mul_rn(L.cs[i], L.H[i + 1 + ldh * j]));
            L.H[i + ldh * j] = t;
        }
        const float a = L.H[j + ldh * j], b = L.H[j + 1 + ldh * j];
        const float rho = sqrt_rn(add_rn(mul_rn(a, a), mul_rn(b, b)));
        ok = rho > 0.0f && isfinite(rho);
        if (ok) {
            L.cs[j] = div_rn(a, rho);
            L.sn[j] = div_rn(b, rho);
            L.H[j + ldh * j] = rho;
            L.H[j + 1 + ldh * j] = 0.0f;
            L.g[j + 1] = mul_rn(-L.sn[j], L.g[j]);
            L.g[j] = mul_rn(L.cs[j], L.g[j]);
        }
    }
    if (!finite) L.nonfinite = 1;
    bool stop = !ok;
    if (ok) {
        L.kdim = j + 1;
        if (!(hn > 0.0f)) stop = true;
        else L.inv = div_rn(1.0f, hn);
    }
    if (stop) L.stop = 1;
    if (stop || last) {
        const int k = L.kdim;
        for (int r = k - 1; r >= 0; --r) {
            float s = L.g[r];
            for (int l = r + 1; l < k; ++l) s = fma_rn(-L.H[r + ldh * l], L.y[l], s);
            L.y[r] = div_rn(s, L.H[r + ldh * r]);
        }
    }
}

__device__ __forceinline__ float pow2_scale_f(float a) { return pow2_scale_for(a); }

// ----------------------------------------------------------- team kernels
// row sum of a slice exactly W entries wide: W gathers, then W fused
// multiply-adds in CSR order (no slot past the width)
template <class TC, int W, class TA, class GX>
__device__ __forceinline__ TC row_sum_w(const Sys &S, const TA *val, int beg, GX gx) {
    int c[W];
    TC a[W], xv[W];
#pragma unroll
    for (int q = 0; q < W; ++q) {
        c[q] = __ldg(S.col + beg + (q << 5));
        a[q] = to_c<TC>(__ldg(val + beg + (q << 5)));
    }
#pragma unroll
    for (int q = 0; q < W; ++q) xv[q] = (c[q] >= 0) ? gx(c[q]) : (TC)0;
    TC acc = (TC)0;
#pragma unroll
    for (int q = 0; q < W; ++q)
        if (c[q] >= 0) acc = fma_rn(a[q], xv[q], acc);
    return acc;
}

// row sum of slice row i over A (CSR order, fused multiply-add), x from gx
template <class TC, class TA, class GX>
__device__ __forceinline__ TC row_sum(const Sys &S, const TA *val, int s, int lane, GX gx) {
    const int beg = __ldg(S.sptr + s) + lane;
    const int w = (__ldg(S.sptr + s + 1) - __ldg(S.sptr + s)) >> 5;
    switch (w) {  // slices up to 8 wide: exact-width code
        case 0: return (TC)0;
        case 1: return row_sum_w<TC, 1>(S, val, beg, gx);
        case 2: return row_sum_w<TC, 2>(S, val, beg, gx);
        case 3: return row_sum_w<TC, 3>(S, val, beg, gx);
        case 4: return row_sum_w<TC, 4>(S, val, beg, gx);
        case 5: return row_sum_w<TC, 5>(S, val, beg, gx);
        case 6: return row_sum_w<TC, 6>(S, val, beg, gx);
        case 7: return row_sum_w<TC, 7>(S, val, beg, gx);
        case 8: return row_sum_w<TC, 8>(S, val, beg, gx);
        default: break;
    }
    TC acc = (TC)0;
    constexpr int U = 4;  // loads of a group of entries issued before its multiply-adds
    for (int k0 = 0; k0 < w; k0 += U) {
        int c[U];
        TC a[U], xv[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int idx = beg + ((k0 + q) << 5);
            c[q] = (k0 + q < w) ? __ldg(S.col + idx) : -1;
            a[q] = (k0 + q < w) ? to_c<TC>(__ldg(val + idx)) : (TC)0;
        }
#pragma unroll
        for (int q = 0; q < U; ++q) xv[q] = (c[q] >= 0) ? gx(c[q]) : (TC)0;
#pragma unroll
        for (int q = 0; q < U; ++q)
            if (c[q] >= 0) acc = fma_rn(a[q], xv[q], acc);
    }
    return acc;
}

struct Ctx2 {
    const Team &tm;
    Shared &sh;
    const Sys &S;
    const Inst &I;
    const BP &P;
    Out &o;
};

// Richardson call (Algorithm 1, m4 = 2) on rin (scaled by sigma) into out = z / sigma
__device__ void rich_call(Ctx2 &C, float inv_sigma, float *out) {
    const Team &tm = C.tm;
    Shared &sh = C.sh;
    const Sys &S = C.S;
    const Inst &I = C.I;
    const int n = S.n;
    const bool fixed = C.P.omega_fixed > 0.0f;
    const bool update = !fixed && (sh.c_ntr % C.P.c) == 0;
    if (!update) {
        const float w1 = sh.omega[0], w2 = sh.omega[1];
        for (int s = tm.wid; s < S.nslices; s += tm.nwarps) {
            const bool unit = S.m_unit != 0;
            const float acc = row_sum<float>(S, S.a16, s, tm.lane, [&](int c) {
                const float vc = to_c<float>(ldcg(I.rin + c));
                return rnd<h16>(fma_rn(w1, unit ? vc : mul_rn(to_c<float>(__ldg(S.m16 + c)), vc), 0.0f));
            });
            const int i = s * kSlice + tm.lane;
            if (i < n) {
                const float vi = to_c<float>(ldcg(I.rin + i));
                const float z1 = rnd<h16>(fma_rn(w1, unit ? vi : mul_rn(to_c<float>(__ldg(S.m16 + i)), vi), 0.0f));
                const float ri = rnd<h16>(sub_rn(vi, acc));
                const float z2 = rnd<h16>(fma_rn(w2, unit ? ri : mul_rn(to_c<float>(__ldg(S.m16 + i)), ri), z1));
                out[i] = mul_rn(z2, inv_sigma);
            }
        }
        C.o.m_applies += 2;
    } else {
        // two steps, each computing w' = (r, AMr)/(AMr, AMr) in fp32
        const long long l_ = sh.c_ntr / C.P.c;
        for (int k = 0; k < 2; ++k) {
            const h16 *r = (k == 0) ? I.rin : I.rr;
            if (k == 1) {
                for (int s = tm.wid; s < S.nslices; s += tm.nwarps) {
                    const float acc =
                        row_sum<float>(S, S.a16, s, tm.lane, [&](int c) { return to_c<float>(ldcg(I.rz + c)); });
                    const int i = s * kSlice + tm.lane;
                    if (i < n) I.rr[i] = Store<h16>::from(sub_rn(to_c<float>(ldcg(I.rin + i)), acc));
                }
                team_sync(tm);
            }
            float acc[2] = {0.0f, 0.0f};
            for (int s = tm.wid; s < S.nslices; s += tm.nwarps) {
                const float w = row_sum<float>(S, S.a16, s, tm.lane, [&](int c) {
                    return mul_rn(to_c<float>(__ldg(S.m16 + c)), to_c<float>(ldcg(r + c)));
                });
                const int i = s * kSlice + tm.lane;
                if (i < n) {
                    acc[0] = fma_rn(to_c<float>(ldcg(r + i)), w, acc[0]);
                    acc[1] = fma_rn(w, w, acc[1]);
                }
            }
            float res[2];
            team_reduce<float>(tm, sh, acc, 2, res);
            const float wk = sh.omega[k];
            const float q = div_rn(res[0], res[1]);
            const bool ok = res[1] > 0.0f && isfinite(q);
            const float wp = ok ? q : wk;
            __syncthreads();
            if (threadIdx.x == 0 && ok) {
                const float l = (float)l_;
                sh.omega[k] = div_rn(add_rn(mul_rn(l, wk), q), add_rn(l, 1.0f));
            }
            for (int i = tm.tid; i < n; i += tm.nthr) {
                const float zp = (k == 0) ? 0.0f : to_c<float>(ldcg(I.rz + i));
                const float z = rnd<h16>(fma_rn(wp, mul_rn(to_c<float>(__ldg(S.m16 + i)), to_c<float>(ldcg(r + i))), zp));
                if (k == 1) out[i] = mul_rn(z, inv_sigma);
                else I.rz[i] = Store<h16>::from(z);
            }
            team_sync(tm);
        }
        C.o.m_applies += 2;
    }
    C.o.r_calls += 1;
    __syncthreads();
    if (threadIdx.x == 0) sh.c_ntr += 1;
    __syncthreads();
}

// Inner FGMRES level with fp32 vectors: levels 2 (A fp32) and 3 (A fp16).
// On entry V[0] holds the input and L.beta / L.inv / L.sigma are set (or
// L.stop); on exit out = sum_k y_k Z[k] (fp32, or fp64 * dsc for level 2).
template <int LEVEL>
__device__ void inner_level(Ctx2 &C, float *V, float *Z, float *w, LS &L, int m, float *out32, double *out64) {
    const Team &tm = C.tm;
    Shared &sh = C.sh;
    const Sys &S = C.S;
    const Inst &I = C.I;
    const int n = S.n, ld = I.ld;
    const bool half_child = (LEVEL == 3);
    if (!L.stop) {
        // V[0] = x / beta; the child's input from it
        for (int i = tm.tid; i < n; i += tm.nthr) {
            const float v = mul_rn(ldcg(V + i), L.inv);
            V[i] = v;
            if (LEVEL == 2) I.V3[i] = v;
            else I.rin[i] = Store<h16>::from(mul_rn(L.sigma, v));
        }
        if (LEVEL == 2) {
            // F3 start: ||V2[0]||, max -> beta3, sigma3
            float acc[2] = {0.0f, 0.0f};
            for (int i = tm.tid; i < n; i += tm.nthr) {
                const float v = ldcg(I.V3 + i);
                acc[0] = fma_rn(v, v, acc[0]);
                acc[1] = fmax(acc[1], fabs(v));
            }
            const bool mx[2] = {false, true};
            float res[2];
            team_reduce<float>(tm, sh, acc, 2, res, mx);
            if (threadIdx.x == 0) {
                LS &L3 = sh.ls3;
                const float beta = sqrt_rn(res[0]);
                L3.kdim = 0;
                L3.nonfinite = isfinite(beta) ? 0 : 1;
                L3.stop = (beta > 0.0f && isfinite(beta)) ? 0 : 1;
                L3.beta = beta;
                if (!L3.stop) {
                    L3.inv = div_rn(1.0f, beta);
                    L3.g[0] = beta;
                    L3.sigma = C.P.scale_cast ? pow2_scale_f(mul_rn(res[1], L3.inv)) : 1.0f;
                    L3.inv_sigma = div_rn(1.0f, L3.sigma);
                }
            }
            __syncthreads();
        } else {
            team_sync(tm);
        }
    }
    for (int j = 0; j < m && !L.stop; ++j) {
        // child -> Z[j]
        if (LEVEL == 2) inner_level<3>(C, I.V3, I.Z3, I.w3, sh.ls3, C.P.m3, Z + (size_t)j * ld, nullptr);
        else rich_call(C, L.inv_sigma, Z + (size_t)j * ld);
        team_sync(tm);
        // w = A Z[j], hA = V^T w
        const float *zj = Z + (size_t)j * ld;
        float acc[kRedMax];
        for (int l = 0; l < kRedMax; ++l) acc[l] = 0.0f;
        for (int s = tm.wid; s < S.nslices; s += tm.nwarps) {
            float y = (LEVEL == 2) ? row_sum<float>(S, S.a32, s, tm.lane, [&](int c) { return ldcg(zj + c); })
                                   : row_sum<float>(S, S.a16, s, tm.lane, [&](int c) { return ldcg(zj + c); });
            const int i = s * kSlice + tm.lane;
            if (i < n) {
                w[i] = y;
                for (int l = 0; l <= j; ++l) acc[l] = fma_rn(ldcg(V + (size_t)l * ld + i), y, acc[l]);
            }
        }
        float hA[kRedMax], hB[kRedMax];
        team_reduce<float>(tm, sh, acc, j + 1, hA);
        const float *hl = hA;
        if (C.P.cgs_passes == 2) {
            for (int l = 0; l < kRedMax; ++l) acc[l] = 0.0f;
            for (int i = tm.tid; i < n; i += tm.nthr) {
                float wi = ldcg(w + i);
                float v[kRedMax];
                for (int l = 0; l <= j; ++l) {
                    v[l] = ldcg(V + (size_t)l * ld + i);
                    wi = fma_rn(-hA[l], v[l], wi);
                }
                w[i] = wi;
                for (int l = 0; l <= j; ++l) acc[l] = fma_rn(v[l], wi, acc[l]);
            }
            team_reduce<float>(tm, sh, acc, j + 1, hB);
            hl = hB;
        }
        float a2[2] = {0.0f, 0.0f};
        for (int i = tm.tid; i < n; i += tm.nthr) {
            float wi = ldcg(w + i);
            for (int l = 0; l <= j; ++l) wi = fma_rn(-hl[l], ldcg(V + (size_t)l * ld + i), wi);
            w[i] = wi;
            a2[0] = fma_rn(wi, wi, a2[0]);
            a2[1] = fmax(a2[1], fabs(wi));
        }
        const bool mx[2] = {false, true};
        float r2[2];
        team_reduce<float>(tm, sh, a2, 2, r2, mx);
        if (threadIdx.x == 0) {
            float hcol[kRedMax];
            for (int l = 0; l <= j; ++l) hcol[l] = (C.P.cgs_passes == 2) ? add_rn(hA[l], hB[l]) : hA[l];
            const float hn = sqrt_rn(r2[0]);
            ls_column(L, m, j, hcol, hn, j == m - 1);
            if (half_child && hn > 0.0f && C.P.scale_cast) {
                L.sigma = pow2_scale_f(mul_rn(r2[1], L.inv));
                L.inv_sigma = div_rn(1.0f, L.sigma);
            } else {
                L.sigma = 1.0f;
                L.inv_sigma = 1.0f;
            }
        }
        __syncthreads();
        if (L.stop || j == m - 1) break;
        // V[j+1] = w / ||w||; the child's next input
        float b3[2] = {0.0f, 0.0f};
        for (int i = tm.tid; i < n; i += tm.nthr) {
            const float v = mul_rn(ldcg(w + i), L.inv);
            V[(size_t)(j + 1) * ld + i] = v;
            if (LEVEL == 2) {
                I.V3[i] = v;
                b3[0] = fma_rn(v, v, b3[0]);
                b3[1] = fmax(b3[1], fabs(v));
            } else {
                I.rin[i] = Store<h16>::from(mul_rn(L.sigma, v));
            }
        }
        if (LEVEL == 2) {
            float r3[2];
            team_reduce<float>(tm, sh, b3, 2, r3, mx);
            if (threadIdx.x == 0) {
                LS &L3 = sh.ls3;
                const float beta = sqrt_rn(r3[0]);
                L3.kdim = 0;
                L3.nonfinite = isfinite(beta) ? 0 : 1;
                L3.stop = (beta > 0.0f && isfinite(beta)) ? 0 : 1;
                L3.beta = beta;
                if (!L3.stop) {
                    L3.inv = div_rn(1.0f, beta);
                    L3.g[0] = beta;
                    L3.sigma = C.P.scale_cast ? pow2_scale_f(mul_rn(r3[1], L3.inv)) : 1.0f;
                    L3.inv_sigma = div_rn(1.0f, L3.sigma);
                }
            }
            __syncthreads();
        } else {
            team_sync(tm);
        }
    }
    // out = sum_k y_k Z[k]
    const int k = L.stop && L.kdim == 0 ? 0 : L.kdim;
    const bool nan_out = L.nonfinite && L.kdim == 0;
    for (int i = tm.tid; i < n; i += tm.nthr) {
        float s = 0.0f;
        for (int l = 0; l < k; ++l) s = fma_rn(L.y[l], ldcg(Z + (size_t)l * ld + i), s);
        if (nan_out) s = NAN;
        if (LEVEL == 2) out64[i] = mul_rn(__ldg(S.dsc + i), (double)s);
        else out32[i] = s;
    }
}

// ------------------------------------------------------- one instance solve
__device__ void solve_instance(const Team &tm, Shared &sh, const Sys &S, const Inst &I, const BP &P, Out &o) {
    cg::cluster_group cl = cg::this_cluster();
    const int n = S.n, ld = I.ld, m1 = P.m1;
    Ctx2 C{tm, sh, S, I, P, o};
    double *H = I.H1, *cs = H + (m1 + 1) * m1, *sn = cs + m1, *g = sn + m1, *y = g + m1 + 1;
    const int ldh = m1 + 1;
    o = Out{F3R_NOT_CONVERGED, 0, 0, 0.0, 0, 0};
    // ||b||
    double accb[1] = {0.0};
    for (int i = tm.tid; i < n; i += tm.nthr) accb[0] = fma_rn(I.b[i], I.b[i], accb[0]);
    double nbv[1];
    team_reduce<double>(tm, sh, accb, 1, nbv);
    const double nb = sqrt_rn(nbv[0]);
    if (threadIdx.x == 0) {
        sh.c_ntr = 1;
        sh.omega[0] = sh.omega[1] = (P.omega_fixed > 0.0f) ? P.omega_fixed : 1.0f;
    }
    __syncthreads();
    if (!(nb > 0.0)) {
        for (int i = tm.tid; i < n; i += tm.nthr) I.x[i] = 0.0;
        o.status = isfinite(nb) ? F3R_OK : F3R_ERR_NONFINITE;
        return;
    }
    int total = 0, cycles = 0;
    for (;;) {
        // r = b - A x
        double ar[1] = {0.0};
        for (int s = tm.wid; s < S.nslices; s += tm.nwarps) {
            const double ax = row_sum<double>(S, S.a64, s, tm.lane, [&](int c) { return ldcg(I.x + c); });
            const int i = s * kSlice + tm.lane;
            if (i < n) {
                const double ri = sub_rn(I.b[i], ax);
                I.w1[i] = ri;
                ar[0] = fma_rn(ri, ri, ar[0]);
            }
        }
        double bb[1];
        team_reduce<double>(tm, sh, ar, 1, bb);
        const double beta = sqrt_rn(bb[0]);
        const double rel = div_rn(beta, nb);
        o.rel = rel;
        if (!isfinite(beta)) {
            o.status = F3R_ERR_NONFINITE;
            break;
        }
        if (rel < P.tol) {
            o.status = F3R_OK;
            break;
        }
        if (total >= P.max_outer) break;
        ++cycles;
        const double inv0 = div_rn(1.0, beta);
        if (tm.rank == 0 && threadIdx.x == 0) g[0] = beta;
        // V1[0] = r / beta, F2 input (fp32 of D^-1/2 V1[0]) in V2[0]
        double inv = inv0;
        int kdim = 0;
        bool nonfinite = false;
        for (int j = 0; j < m1; ++j) {
            float a2[2] = {0.0f, 0.0f};
            for (int i = tm.tid; i < n; i += tm.nthr) {
                const double v = mul_rn(ldcg(j == 0 ? I.w1 + i : I.w1 + i), inv);
                I.V1[(size_t)j * ld + i] = v;
                const float c = __double2float_rn(mul_rn(__ldg(S.dsc + i), v));
                I.V2[i] = c;
                a2[0] = fma_rn(c, c, a2[0]);
            }
            float r2[1];
            team_reduce<float>(tm, sh, a2, 1, r2);
            if (threadIdx.x == 0) {
                LS &L2 = sh.ls2;
                const float b2 = sqrt_rn(r2[0]);
                L2.kdim = 0;
                L2.nonfinite = isfinite(b2) ? 0 : 1;
                L2.stop = (b2 > 0.0f && isfinite(b2)) ? 0 : 1;
                L2.beta = b2;
                if (!L2.stop) {
                    L2.inv = div_rn(1.0f, b2);
                    L2.g[0] = b2;
                }
            }
            __syncthreads();
            // Z1[j] = D^-1/2 F2(D^-1/2 V1[j])
            double *zj = I.Z1 + (size_t)j * ld;
            inner_level<2>(C, I.V2, I.Z2, I.w2, sh.ls2, P.m2, nullptr, zj);
            team_sync(tm);
            // w = A Z1[j]; CGS2 against V1[0..j] in chunks of kRedMax
            for (int s = tm.wid; s < S.nslices; s += tm.nwarps) {
                const double yv = row_sum<double>(S, S.a64, s, tm.lane, [&](int c) { return ldcg(zj + c); });
                const int i = s * kSlice + tm.lane;
                if (i < n) I.w1[i] = yv;
            }
            team_sync(tm);
            double hsum[kMaxOuterM + 1];
            for (int p = 0; p < P.cgs_passes; ++p) {
                double h[kMaxOuterM + 1];
                for (int l0 = 0; l0 <= j; l0 += kRedMax) {
                    const int cnt = min(kRedMax, j + 1 - l0);
                    double acc[kRedMax];
                    for (int l = 0; l < kRedMax; ++l) acc[l] = 0.0;
                    for (int i = tm.tid; i < n; i += tm.nthr) {
                        const double wi = ldcg(I.w1 + i);
                        for (int l = 0; l < cnt; ++l) acc[l] = fma_rn(ldcg(I.V1 + (size_t)(l0 + l) * ld + i), wi, acc[l]);
                    }
                    team_reduce<double>(tm, sh, acc, cnt, h + l0);
                }
                for (int i = tm.tid; i < n; i += tm.nthr) {
                    double wi = ldcg(I.w1 + i);
                    for (int l = 0; l <= j; ++l) wi = fma_rn(-h[l], ldcg(I.V1 + (size_t)l * ld + i), wi);
                    I.w1[i] = wi;
                }
                for (int l = 0; l <= j; ++l) hsum[l] = (p == 0) ? h[l] : add_rn(hsum[l], h[l]);
                team_sync(tm);
            }
            double an[1] = {0.0};
            for (int i = tm.tid; i < n; i += tm.nthr) {
                const double wi = ldcg(I.w1 + i);
                an[0] = fma_rn(wi, wi, an[0]);
            }
            double rn[1];
            team_reduce<double>(tm, sh, an, 1, rn);
            const double hn = sqrt_rn(rn[0]);
            ++total;
            // outer Givens step (rank 0 owns H1), decisions broadcast
            if (tm.rank == 0 && threadIdx.x == 0) {
                bool finite = isfinite(hn);
                for (int l = 0; l <= j; ++l) finite = finite && isfinite(hsum[l]);
                bool ok = finite;
                if (ok) {
                    for (int l = 0; l <= j; ++l) H[l + ldh * j] = hsum[l];
                    H[j + 1 + ldh * j] = hn;
                    for (int l = 0; l < j; ++l) {
                        const double t = add_rn(mul_rn(cs[l], H[l + ldh * j]), mul_rn(sn[l], H[l + 1 + ldh * j]));
                        H[l + 1 + ldh * j] = add_rn(mul_rn(-sn[l], H[l + ldh * j]), mul_rn(cs[l], H[l + 1 + ldh * j]));
                        H[l + ldh * j] = t;
                    }
                    const double a = H[j + ldh * j], b = H[j + 1 + ldh * j];
                    const double rho = sqrt_rn(add_rn(mul_rn(a, a), mul_rn(b, b)));
                    ok = rho > 0.0 && isfinite(rho);
                    if (ok) {
                        cs[j] = div_rn(a, rho);
                        sn[j] = div_rn(b, rho);
                        H[j + ldh * j] = rho;
                        H[j + 1 + ldh * j] = 0.0;
                        g[j + 1] = mul_rn(-sn[j], g[j]);
                        g[j] = mul_rn(cs[j], g[j]);
                    }
                }
                sh.o_nonfinite = finite ? 0 : 1;
                sh.o_kdim = ok ? j + 1 : j;
                sh.o_stop = (!ok || !(hn > 0.0)) ? 1 : 0;
                sh.o_inv = (ok && hn > 0.0) ? div_rn(1.0, hn) : 0.0;
                sh.o_est = div_rn(fabs(g[sh.o_kdim]), nb);
                if (tm.k > 1) {  // the other clusters of a wide team read them from global memory
                    tm.dec[0] = (double)sh.o_kdim;
                    tm.dec[1] = (double)sh.o_stop;
                    tm.dec[2] = (double)sh.o_nonfinite;
                    tm.dec[3] = sh.o_est;
                    tm.dec[4] = sh.o_inv;
                }
            }
            team_sync(tm);
            int o_kdim, o_stop, o_nf;
            double o_est, o_inv;
            if (tm.k > 1) {
                o_kdim = (int)__ldcg(tm.dec + 0);
                o_stop = (int)__ldcg(tm.dec + 1);
                o_nf = (int)__ldcg(tm.dec + 2);
                o_est = __ldcg(tm.dec + 3);
                o_inv = __ldcg(tm.dec + 4);
            } else {
                const Shared *s0 = cl.map_shared_rank(&sh, 0);
                o_kdim = s0->o_kdim;
                o_stop = s0->o_stop;
                o_nf = s0->o_nonfinite;
                o_est = s0->o_est;
                o_inv = s0->o_inv;
            }
            team_sync(tm);
            kdim = o_kdim;
            if (o_nf) {
                nonfinite = true;
                break;
            }
            if (o_stop || o_est < P.tol || total >= P.max_outer) break;
            inv = o_inv;
            // V1[j+1] = w / ||w|| happens at the top of the next iteration (from w1)
        }
        // y = R^-1 g, x += Z1 y
        if (tm.rank == 0 && threadIdx.x == 0) {
            for (int r = kdim - 1; r >= 0; --r) {
                double s = g[r];
                for (int l = r + 1; l < kdim; ++l) s = fma_rn(-H[r + ldh * l], y[l], s);
                y[r] = div_rn(s, H[r + ldh * r]);
            }
        }
        team_sync(tm);
        for (int i = tm.tid; i < n; i += tm.nthr) {
            double s = 0.0;
            for (int l = 0; l < kdim; ++l) s = fma_rn(ldcg(y + l), ldcg(I.Z1 + (size_t)l * ld + i), s);
            I.x[i] = add_rn(ldcg(I.x + i), s);
        }
        team_sync(tm);
        if (nonfinite) {
            o.status = F3R_ERR_NONFINITE;
            break;
        }
    }
    o.outer_iters = total;
    o.restarts = cycles > 0 ? cycles - 1 : 0;
}

// One persistent launch over every instance.  Clusters [0, nteams * kw)
// first form nteams wide teams of kw clusters that take the large systems'
// instances (worder, largest first) from queue[1]; then every cluster, alone,
// takes the other instances (order) from queue[0].
__global__ void __launch_bounds__(kBT) k_batch(const Sys *sys, const Inst *inst, const int *order, int ninst,
                                               const int *worder, int nwide, int kw, int nteams, BP P, int *queue,
                                               unsigned *wbar, double *wpart, double *wdec, int *abort, Out *outs) {
    __shared__ Shared sh;
    cg::cluster_group cl = cg::this_cluster();
    Team tm;
    tm.crank = cl.block_rank();
    tm.csize = cl.num_blocks();
    tm.lane = threadIdx.x & 31;
    tm.abort = abort;
    const int cid = (int)(blockIdx.x / tm.csize);
    auto form = [&](int k, int kidx) {
        tm.k = k;
        tm.kidx = kidx;
        tm.rank = (unsigned)kidx * tm.csize + tm.crank;
        tm.size = (unsigned)k * tm.csize;
        tm.tid = (int)tm.rank * blockDim.x + threadIdx.x;
        tm.nthr = (int)tm.size * blockDim.x;
        tm.wid = tm.tid >> 5;
        tm.nwarps = tm.nthr >> 5;
    };
    if (threadIdx.x == 0) sh.red_buf = 0;  // every block of the team toggles it in step
    __syncthreads();
    if (cid < nteams * kw && nwide > 0) {
        const int t = cid / kw;
        form(kw, cid % kw);
        tm.bar = wbar + 2 * t;
        tm.part = wpart + (size_t)t * 2 * kw * kRedMax;
        tm.dec = wdec + (size_t)t * 16;
        for (;;) {
            if (tm.rank == 0 && threadIdx.x == 0) tm.dec[8] = (double)atomicAdd(queue + 1, 1);
            team_sync(tm);
            const int q = (int)__ldcg(tm.dec + 8);
            team_sync(tm);
            if (q >= nwide) break;
            const int k = worder[q];
            const Inst I = inst[k];
            const Sys S = sys[I.sys];
            Out o;
            solve_instance(tm, sh, S, I, P, o);
            if (*(volatile int *)abort) o.status = F3R_ERR_TIMEOUT;
            if (tm.rank == 0 && threadIdx.x == 0) outs[k] = o;
            team_sync(tm);
        }
    }
    form(1, 0);
    tm.bar = nullptr;
    tm.part = nullptr;
    tm.dec = nullptr;
    for (;;) {
        if (tm.rank == 0 && threadIdx.x == 0) sh.inst = atomicAdd(queue, 1);
        team_sync(tm);
        const int q = cl.map_shared_rank(&sh, 0)->inst;
        team_sync(tm);
        if (q >= ninst) break;
        const int k = order[q];
        const Inst I = inst[k];
        const Sys S = sys[I.sys];
        Out o;
        solve_instance(tm, sh, S, I, P, o);
        if (tm.rank == 0 && threadIdx.x == 0) outs[k] = o;
        team_sync(tm);
    }
}

}  // namespace bt
}  // namespace f3r

using namespace f3r;

struct f3r_batch {
    std::vector<Ctx *> sys;   // matrix of each system (set-up arrays only; none for a large system)
    std::vector<f3r_ctx *> full;  // large systems: a single-system context, else null
    std::vector<int> small;   // instances of the persistent launch on one cluster each, largest first
    std::vector<int> wide;    // instances of the large systems taken by wide teams, largest first
    std::vector<int> nrhs;
    std::vector<int> inst_sys, inst_rhs;
    bt::BP P{};
    f3r_params prm{};
    bt::Sys *d_sys = nullptr;
    bt::Inst *d_inst = nullptr;
    int *d_order = nullptr, *d_queue = nullptr, *d_worder = nullptr, *d_abort = nullptr;
    unsigned *d_wbar = nullptr;   // [team][2] barrier words of the wide teams
    double *d_wpart = nullptr;    // [team][2][kw][kRedMax] cluster sums
    double *d_wdec = nullptr;     // [team][16] broadcast slots
    int kw = 0, nteams = 0;       // clusters per wide team, wide teams (of the last launch)
    int kw_req = 0;               // clusters per wide team the autotuner chose (0: batch_wide's rule)
    bt::Out *d_out = nullptr;
    std::vector<bt::Inst> h_inst;
    std::vector<void *> allocs;
    int cluster = 8, threads = bt::kBT, grid = 0;
    long long bytes = 0;
    cudaStream_t cs = nullptr;
    // the persistent launch as a CUDA graph per (cluster, threads): the
    // instance table is copied from pinned memory, the queue reset, the
    // kernel run and the results copied back to pinned memory
    bt::Inst *pin_inst = nullptr;
    bt::Out *pin_out = nullptr;
    std::map<int, cudaGraphExec_t> graphs;
    std::map<int, int> graph_grid;  // blocks of each graph's launch
    std::map<int, std::pair<int, int>> graph_wide;  // clusters per wide team, wide teams of each graph
    long long graph_launches = 0;
};

namespace {
void *balloc(f3r_batch *b, size_t bytes) {
    void *p = nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) return nullptr;
    b->allocs.push_back(p);
    b->bytes += (long long)bytes;
    return p;
}
}  // namespace

extern "C" {

f3r_status f3r_setup_batched(f3r_batch **out, int nsys, const f3r_system_desc *desc, const f3r_params *params,
                             void *stream) {
    if (!out || nsys <= 0 || !desc) return F3R_ERR_ARG;
    *out = nullptr;
    f3r_params prm;
    if (params) prm = *params;
    else f3r_default_params(&prm);
    // the batched path runs the default F3R precision schedule
    if (prm.nlevels != 3 || prm.rich_m != 2 || prm.a_prec[1] != F3R_F32 || prm.a_prec[2] != F3R_F16 ||
        prm.v_prec[1] != F3R_F32 || prm.v_prec[2] != F3R_F32 || prm.rich_a_prec != F3R_F16 ||
        prm.rich_v_prec != F3R_F16 || prm.m_prec != F3R_F16 || prm.row_scale || prm.inner_rtol != 0.0f)
        return F3R_ERR_UNSUPPORTED;
    if (prm.m[0] < 1 || prm.m[0] > kMaxOuterM || prm.m[1] < 1 || prm.m[1] > kMaxInnerM || prm.m[2] < 1 ||
        prm.m[2] > kMaxInnerM || prm.c < 1 || prm.max_outer < 1 || (prm.cgs_passes != 1 && prm.cgs_passes != 2))
        return F3R_ERR_ARG;
    f3r_batch *b = new (std::nothrow) f3r_batch;
    if (!b) return F3R_ERR_NOMEM;
    b->prm = prm;
    auto fail = [&](f3r_status e) {
        f3r_destroy_batched(b);
        return e;
    };
    if (cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking) != cudaSuccess) return fail(F3R_ERR_CUDA);
    cudaStream_t s = b->cs;
    cudaEvent_t ev;
    cudaEventCreate(&ev);
    cudaEventRecord(ev, (cudaStream_t)stream);
    cudaStreamWaitEvent(s, ev, 0);
    cudaEventDestroy(ev);
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // systems of at least `split` rows are solved one after another by the
    // single-system path (the whole GPU each); in the persistent launch they
    // would run on one cluster and keep the launch waiting on them
    const long long split = prm.batch_split > 0 ? (long long)prm.batch_split
                                                : (prm.batch_split < 0 ? (1LL << 40) : 2048LL * nsm);
    // batch_wide < 0: the large systems on the single-system path; else in
    // the persistent launch, each instance on a wide team of clusters
    const bool single_path = prm.batch_wide < 0;
    b->full.assign(nsys, nullptr);
    std::vector<bt::Sys> hs(nsys);
    for (int k = 0; k < nsys; ++k) {
        const f3r_system_desc &d = desc[k];
        if (d.n <= 0 || d.nrhs < 1 || !d.rowptr || !d.colidx || !d.val) return fail(F3R_ERR_ARG);
        Ctx *c = new (std::nothrow) Ctx;
        if (!c) return fail(F3R_ERR_NOMEM);
        b->sys.push_back(c);
        c->dev = dev;
        c->nsm = nsm;
        c->zstream = s;  // the copies of A are allocated and built in the batch's stream
        c->prm = prm;
        c->n = d.n;
        c->nnz = d.nnz;
        c->ld = (int)(((long long)d.n + kTileRows - 1) / kTileRows * kTileRows);  // whole tiles
        if (d.n >= split && single_path) {
            const f3r_status st = f3r_setup(&b->full[k], d.n, d.nnz, d.rowptr, d.colidx, d.val, &prm, (void *)s);
            if (st != F3R_OK) return fail(st);
            hs[k] = bt::Sys{};
            hs[k].n = d.n;
            for (int r = 0; r < d.nrhs; ++r) {
                b->inst_sys.push_back(k);
                b->inst_rhs.push_back(r);
            }
            b->nrhs.push_back(d.nrhs);
            continue;
        }
        // upload the CSR arrays (host or device) and build the copies of A
        void *tmp[3] = {nullptr, nullptr, nullptr};
        const size_t sz[3] = {sizeof(int) * ((size_t)d.n + 1), sizeof(int) * (size_t)d.nnz, sizeof(double) * (size_t)d.nnz};
        const void *src[3] = {d.rowptr, d.colidx, d.val};
        const void *dp[3];
        for (int q = 0; q < 3; ++q) {
            cudaPointerAttributes a;
            const bool on_dev = cudaPointerGetAttributes(&a, src[q]) == cudaSuccess &&
                                (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
            cudaGetLastError();
            if (on_dev) {
                dp[q] = src[q];
            } else {
                if (cudaMalloc(&tmp[q], sz[q] ? sz[q] : 16) != cudaSuccess) return fail(F3R_ERR_NOMEM);
                cudaMemcpyAsync(tmp[q], src[q], sz[q], cudaMemcpyHostToDevice, s);
                dp[q] = tmp[q];
            }
        }
        f3r_status st = build_matrix(*c, (const int *)dp[0], (const int *)dp[1], (const double *)dp[2], s);
        for (void *p : tmp)
            if (p) cudaFree(p);
        if (st != F3R_OK) return fail(st);
        hs[k] = bt::Sys{c->n, c->nslices, c->sptr, c->col, c->a64, c->a32, c->a16, c->dsc, (const h16 *)c->mvec,
                        c->m_unit ? 1 : 0};
        for (int r = 0; r < d.nrhs; ++r) {
            b->inst_sys.push_back(k);
            b->inst_rhs.push_back(r);
        }
        b->nrhs.push_back(d.nrhs);
    }
    // per-instance workspace
    const int m1 = prm.m[0], m2 = prm.m[1], m3 = prm.m[2];
    const int ninst = (int)b->inst_sys.size();
    b->h_inst.resize(ninst);
    for (int q = 0; q < ninst; ++q) {
        const Ctx &c = *b->sys[b->inst_sys[q]];
        const size_t ld = c.ld;
        bt::Inst &I = b->h_inst[q];
        I = bt::Inst{};
        I.sys = b->inst_sys[q];
        I.ld = (int)ld;
        I.b = nullptr;
        I.x = nullptr;
        if (b->full[I.sys]) continue;  // solved by its single-system context
        I.V1 = (double *)balloc(b, sizeof(double) * ld * (m1 + 1));
        I.Z1 = (double *)balloc(b, sizeof(double) * ld * m1);
        I.w1 = (double *)balloc(b, sizeof(double) * ld);
        I.H1 = (double *)balloc(b, sizeof(double) * ((m1 + 1) * m1 + 4 * m1 + 2));
        I.V2 = (float *)balloc(b, sizeof(float) * ld * (m2 + 1));
        I.Z2 = (float *)balloc(b, sizeof(float) * ld * m2);
        I.w2 = (float *)balloc(b, sizeof(float) * ld);
        I.V3 = (float *)balloc(b, sizeof(float) * ld * (m3 + 1));
        I.Z3 = (float *)balloc(b, sizeof(float) * ld * m3);
        I.w3 = (float *)balloc(b, sizeof(float) * ld);
        I.rin = (h16 *)balloc(b, sizeof(h16) * ld);
        I.rz = (h16 *)balloc(b, sizeof(h16) * ld);
        I.rr = (h16 *)balloc(b, sizeof(h16) * ld);
        if (!I.V1 || !I.Z1 || !I.w1 || !I.H1 || !I.V2 || !I.Z2 || !I.w2 || !I.V3 || !I.Z3 || !I.w3 || !I.rin ||
            !I.rz || !I.rr)
            return fail(F3R_ERR_NOMEM);
    }
    b->d_sys = (bt::Sys *)balloc(b, sizeof(bt::Sys) * nsys);
    b->d_inst = (bt::Inst *)balloc(b, sizeof(bt::Inst) * ninst);
    b->d_order = (int *)balloc(b, sizeof(int) * ninst);
    b->d_queue = (int *)balloc(b, sizeof(int) * 4);
    b->d_out = (bt::Out *)balloc(b, sizeof(bt::Out) * ninst);
    if (!b->d_sys || !b->d_inst || !b->d_order || !b->d_queue || !b->d_out) return fail(F3R_ERR_NOMEM);
    if (cudaHostAlloc((void **)&b->pin_inst, sizeof(bt::Inst) * ninst, cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc((void **)&b->pin_out, sizeof(bt::Out) * ninst, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return fail(F3R_ERR_NOMEM);
    }
    std::memset(b->pin_out, 0, sizeof(bt::Out) * ninst);
    cudaMemcpyAsync(b->d_sys, hs.data(), sizeof(bt::Sys) * nsys, cudaMemcpyHostToDevice, s);
    // the persistent launch's instances, largest first: the large systems'
    // for the wide teams, the others for single clusters
    for (int q = 0; q < ninst; ++q) {
        if (b->full[b->inst_sys[q]]) continue;
        if (b->sys[b->inst_sys[q]]->n >= split) b->wide.push_back(q);
        else b->small.push_back(q);
    }
    auto larger = [&](int a, int c) { return b->sys[b->inst_sys[a]]->nnz > b->sys[b->inst_sys[c]]->nnz; };
    std::stable_sort(b->small.begin(), b->small.end(), larger);
    std::stable_sort(b->wide.begin(), b->wide.end(), larger);
    if (!b->small.empty())
        cudaMemcpyAsync(b->d_order, b->small.data(), sizeof(int) * b->small.size(), cudaMemcpyHostToDevice, s);
    if (!b->wide.empty()) {
        // barrier words, cluster sums and broadcast slots: a launch holds at
        // most kMaxClustersPerSM clusters per SM, each in at most one team
        const size_t maxc = (size_t)bt::kMaxClustersPerSM * nsm;
        b->d_worder = (int *)balloc(b, sizeof(int) * b->wide.size());
        b->d_wbar = (unsigned *)balloc(b, sizeof(unsigned) * 2 * maxc);
        b->d_wpart = (double *)balloc(b, sizeof(double) * 2 * maxc * bt::kRedMax);
        b->d_wdec = (double *)balloc(b, sizeof(double) * 16 * maxc);
        if (!b->d_worder || !b->d_wbar || !b->d_wpart || !b->d_wdec) return fail(F3R_ERR_NOMEM);
        cudaMemcpyAsync(b->d_worder, b->wide.data(), sizeof(int) * b->wide.size(), cudaMemcpyHostToDevice, s);
    }
    b->d_abort = (int *)balloc(b, sizeof(int) * 4);
    if (!b->d_abort) return fail(F3R_ERR_NOMEM);
    b->P = bt::BP{m1, m2, m3, prm.c, prm.max_outer, prm.cgs_passes, prm.scale_cast, prm.tol, (float)prm.omega_fixed};
    b->cluster = 8;
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(F3R_ERR_CUDA);
    *out = b;
    return F3R_OK;
}

f3r_status f3r_batched_set_cluster(f3r_batch *b, int cluster_size) {
    if (!b || cluster_size < 1 || cluster_size > bt::kMaxCluster || (cluster_size & (cluster_size - 1))) return F3R_ERR_ARG;
    b->cluster = cluster_size;
    return F3R_OK;
}

f3r_status f3r_batched_set_shape(f3r_batch *b, int cluster_size, int threads) {
    if (!b || (threads != 256 && threads != 512)) return F3R_ERR_ARG;
    const f3r_status st = f3r_batched_set_cluster(b, cluster_size);
    if (st != F3R_OK) return st;
    b->threads = threads;
    return F3R_OK;
}

}  // extern "C"

namespace {
// The persistent launch over the instances of the small systems; their
// statuses go to st[q] (and res[q] when given).  Replayed as a CUDA graph
// (one per cluster size and block size): the instances' b and x pointers go
// through a pinned host table that the graph copies to the device.
f3r_status launch_small(f3r_batch *b, const double *const *B, double *const *X, f3r_batch_result *res,
                        std::vector<int> &st, void *stream) {
    const int nsmall = (int)b->small.size(), nwide = (int)b->wide.size();
    if (nsmall + nwide == 0) return F3R_OK;
    cudaStream_t s = b->cs;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, (cudaStream_t)stream);
    cudaStreamWaitEvent(s, e0, 0);
    const int ninst = (int)b->h_inst.size();
    for (int q = 0; q < ninst; ++q) {
        b->h_inst[q].b = B[q];
        b->h_inst[q].x = X[q];
    }
    // the graph reads the table from pinned memory when it runs
    std::memcpy(b->pin_inst, b->h_inst.data(), sizeof(bt::Inst) * ninst);
    const int cl = b->cluster, nt = b->threads;
    const int kw_code = b->kw_req > 0 ? b->kw_req : std::max(0, b->prm.batch_wide);  // 0: automatic
    const int key = (kw_code * 16 + cl) * 1024 + nt;
    auto it = b->graphs.find(key);
    if (it == b->graphs.end()) {
        int dev = 0, nsm = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cl;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.blockDim = dim3(nt, 1, 1);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int ncl = 0;
        cfg.gridDim = dim3(cl, 1, 1);
        if (cudaOccupancyMaxActiveClusters(&ncl, (void *)bt::k_batch, &cfg) != cudaSuccess || ncl < 1) {
            cudaGetLastError();
            ncl = 1;
        }
        // every cluster resident at once (the wide teams' barriers need it)
        ncl = std::min(ncl, bt::kMaxClustersPerSM * nsm);
        if (nwide == 0) ncl = std::min(ncl, nsmall);
        // wide teams: batch_wide clusters each (0: an eighth of the clusters, at least 2)
        int kw = kw_code > 0 ? kw_code : std::max(2, ncl / 8);
        kw = std::max(1, std::min(kw, ncl));
        const int nteams = nwide > 0 ? std::max(1, std::min(nwide, ncl / kw)) : 0;
        b->graph_wide[key] = std::make_pair(nwide > 0 ? kw : 0, nteams);
        cfg.gridDim = dim3(ncl * cl, 1, 1);
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaMemcpyAsync(b->d_inst, b->pin_inst, sizeof(bt::Inst) * ninst, cudaMemcpyHostToDevice, s);
            cudaMemsetAsync(b->d_queue, 0, sizeof(int) * 4, s);
            cudaMemsetAsync(b->d_abort, 0, sizeof(int) * 4, s);
            if (nteams > 0) cudaMemsetAsync(b->d_wbar, 0, sizeof(unsigned) * 2 * nteams, s);
            cudaLaunchKernelEx(&cfg, bt::k_batch, (const bt::Sys *)b->d_sys, (const bt::Inst *)b->d_inst,
                               (const int *)b->d_order, nsmall, (const int *)b->d_worder, nwide, kw, nteams, b->P,
                               b->d_queue, b->d_wbar, b->d_wpart, b->d_wdec, b->d_abort, b->d_out);
            cudaMemcpyAsync(b->pin_out, b->d_out, sizeof(bt::Out) * ninst, cudaMemcpyDeviceToHost, s);
            e = cudaStreamEndCapture(s, &g);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return F3R_ERR_CUDA;
        }
        it = b->graphs.emplace(key, ge).first;
        b->graph_grid[key] = ncl * cl;
    }
    b->grid = b->graph_grid[key];
    b->kw = b->graph_wide[key].first;
    b->nteams = b->graph_wide[key].second;
    cudaEventRecord(e0, s);
    cudaError_t e = cudaGraphLaunch(it->second, s);
    b->graph_launches++;
    cudaEventRecord(e1, s);
    if (e != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaGetLastError();
        return F3R_ERR_CUDA;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    const bt::Out *ho = b->pin_out;
    std::vector<int> all(b->small);
    all.insert(all.end(), b->wide.begin(), b->wide.end());
    std::vector<char> iswide(ninst, 0);
    for (int q : b->wide) iswide[q] = 1;
    for (int q : all) {
        st[q] = ho[q].status;
        if (res) {
            res[q].status = ho[q].status;
            res[q].outer_iters = ho[q].outer_iters;
            res[q].restarts = ho[q].restarts;
            res[q].rel_res_true = ho[q].rel;
            res[q].m_applies = ho[q].m_applies;
            res[q].r_calls = ho[q].r_calls;
            res[q].t_solve_ms = ms;
            res[q].system = b->inst_sys[q];
            res[q].rhs = b->inst_rhs[q];
            res[q].path = iswide[q] ? 2 : 0;
        }
    }
    cudaEventRecord(e1, s);
    cudaStreamWaitEvent((cudaStream_t)stream, e1, 0);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return F3R_OK;
}
}  // namespace

extern "C" {

f3r_status f3r_solve_batched(f3r_batch *b, const double *const *B, double *const *X, f3r_batch_result *res,
                             void *stream) {
    if (!b || !B || !X) return F3R_ERR_ARG;
    const int ninst = (int)b->h_inst.size();
    std::vector<int> st(ninst, F3R_OK);
    // instances of the large systems, one after another on the whole GPU
    for (int q = 0; q < ninst; ++q) {
        f3r_ctx *h = b->full[b->inst_sys[q]];
        if (!h) continue;
        f3r_stats ss{};
        const f3r_status r = f3r_solve(h, B[q], X[q], &ss, stream);
        if (r != F3R_OK && r != F3R_NOT_CONVERGED && r != F3R_ERR_NONFINITE) return r;
        st[q] = r;
        if (res) {
            res[q].status = r;
            res[q].outer_iters = ss.outer_iters;
            res[q].restarts = ss.restarts;
            res[q].rel_res_true = ss.rel_res_true;
            res[q].m_applies = ss.m_applies;
            res[q].r_calls = ss.r_calls;
            res[q].t_solve_ms = ss.t_solve_ms;
            res[q].system = b->inst_sys[q];
            res[q].rhs = b->inst_rhs[q];
            res[q].path = 1;
        }
    }
    const f3r_status e = launch_small(b, B, X, res, st, stream);
    if (e != F3R_OK) return e;
    for (int q = 0; q < ninst; ++q)
        if (st[q] != F3R_OK) return (f3r_status)st[q];
    return F3R_OK;
}

// Autotuner of the batched launch shape: time one outer iteration of the
// persistent launch's instances (from x0 = 0) for every team shape -- blocks
// per instance (the cluster size: 1, 2, 4, 8) times threads per block (256,
// 512), i.e. the rows each thread of a team covers -- and, when the batch has
// large systems and batch_wide is automatic, clusters per wide team (2, 4,
// 8); keep the fastest.  X is zeroed again on return.
f3r_status f3r_batched_autotune(f3r_batch *b, const double *const *B, double *const *X, int *chosen, void *stream) {
    if (!b || !B || !X) return F3R_ERR_ARG;
    const int saved_outer = b->P.max_outer;
    const int cand[8][2] = {{1, 256}, {1, 512}, {2, 256}, {2, 512}, {4, 256}, {4, 512}, {8, 256}, {8, 512}};
    // clusters per wide team, when the batch has large systems and batch_wide is automatic
    std::vector<int> kws{0};
    if (!b->wide.empty() && b->prm.batch_wide == 0) kws = {2, 4, 8};
    float best = 3.0e38f;
    int best_c = b->cluster, best_t = b->threads, best_kw = b->kw_req;
    const int ninst = (int)b->h_inst.size();
    std::vector<int> in_launch(b->small);
    in_launch.insert(in_launch.end(), b->wide.begin(), b->wide.end());
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int ci = 0; ci < 8; ++ci) {
        for (int kw : kws) {
            b->cluster = cand[ci][0];
            b->threads = cand[ci][1];
            b->kw_req = kw;
            b->P.max_outer = 1;
            for (int q : in_launch)
                cudaMemsetAsync(X[q], 0, sizeof(double) * (size_t)b->sys[b->inst_sys[q]]->n, b->cs);
            cudaEventRecord(e0, b->cs);
            std::vector<int> stv(ninst, F3R_OK);
            f3r_status st = launch_small(b, B, X, nullptr, stv, stream);
            for (int q : in_launch)
                if (st == F3R_OK && stv[q] != F3R_OK) st = (f3r_status)stv[q];
            cudaEventRecord(e1, b->cs);
            cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if ((st == F3R_OK || st == F3R_NOT_CONVERGED) && ms < best) {
                best = ms;
                best_c = cand[ci][0];
                best_t = cand[ci][1];
                best_kw = kw;
            }
        }
    }
    b->P.max_outer = saved_outer;
    b->cluster = best_c;
    b->threads = best_t;
    b->kw_req = best_kw;
    // the graphs captured while tuning hold max_outer = 1: drop them
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
    b->graph_grid.clear();
    b->graph_wide.clear();
    for (int q = 0; q < ninst; ++q) cudaMemsetAsync(X[q], 0, sizeof(double) * (size_t)b->sys[b->inst_sys[q]]->n, b->cs);
    cudaStreamSynchronize(b->cs);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (chosen) *chosen = best_c;
    return F3R_OK;
}

int f3r_batched_instances(const f3r_batch *b) { return b ? (int)b->h_inst.size() : 0; }

f3r_status f3r_batched_info(const f3r_batch *b, int64_t *out) {
    if (!b || !out) return F3R_ERR_ARG;
    long long rows_small = 0, rows_full = 0, n_full = 0;
    for (size_t q = 0; q < b->h_inst.size(); ++q) {
        const long long n = b->sys[b->inst_sys[q]]->n;
        if (b->full[b->inst_sys[q]]) {
            rows_full += n;
            ++n_full;
        } else {
            rows_small += n;
        }
    }
    out[0] = b->cluster;
    out[1] = b->threads;
    out[2] = (int64_t)(b->small.size() + b->wide.size());
    out[3] = n_full;
    out[4] = rows_small;
    out[5] = rows_full;
    out[6] = b->grid;
    out[7] = b->graph_launches;
    return F3R_OK;
}

f3r_status f3r_batched_wide_info(const f3r_batch *b, int64_t *out) {
    if (!b || !out) return F3R_ERR_ARG;
    long long rows = 0;
    for (int q : b->wide) rows += b->sys[b->inst_sys[q]]->n;
    out[0] = b->kw;
    out[1] = b->nteams;
    out[2] = (int64_t)b->wide.size();
    out[3] = rows;
    return F3R_OK;
}

int64_t f3r_batched_device_bytes(const f3r_batch *b) {
    if (!b) return 0;
    long long t = b->bytes;
    for (Ctx *c : b->sys) t += c->bytes;
    for (f3r_ctx *h : b->full)
        if (h) t += f3r_device_bytes(h);
    return t;
}

void f3r_destroy_batched(f3r_batch *b) {
    if (!b) return;
    for (Ctx *c : b->sys) {
        for (void *p : c->allocs) pool_free(p, b->cs);
        delete c;
    }
    for (f3r_ctx *h : b->full)
        if (h) f3r_destroy(h);
    if (b->cs) cudaStreamSynchronize(b->cs);
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    for (void *p : b->allocs) cudaFree(p);
    if (b->pin_inst) cudaFreeHost(b->pin_inst);
    if (b->pin_out) cudaFreeHost(b->pin_out);
    if (b->cs) cudaStreamDestroy(b->cs);
    delete b;
}

}  // extern "C"
