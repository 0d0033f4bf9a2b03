// The tail of one inner FGMRES iteration in a single cooperative launch:
// second CGS pass, norm, Givens step and normalisation with the cast into
// the child's input (Sec. 4.2, Table 1), replacing k_cgs_pass, k_cgs_final and
// k_normalize.
//
// Every block owns one contiguous chunk of rows and keeps its part of w in
// shared memory across two grid-wide barriers:
//   phase A   w1 = w - V[0..j] hA,  hB = V[0..j]^T w1           | barrier 1
//   phase B   w2 = w1 - V[0..j] hB, ||w2||^2, max|w2|           | barrier 2
//   phase C   V[j+1] = w2 / ||w2||, child input (cast, sigma), child beta
// so w is read once from HBM (not three times and written twice), V[0..j] is
// read twice (the second time mostly from L2) and three launches become one.
// After each barrier every block sums the per-block partials itself, in the
// same fixed block order, so all blocks hold bit-identical h and ||w2||.
// Block 0 records hB and runs the Givens step.  The barriers are bounded: a
// block that waits about two seconds records an error and leaves, and the
// others follow at their next wait.
#pragma once
#include "kernels.cuh"
#include "stage.cuh"

namespace f3r {

#ifndef F3R_FUSED_THREADS
#define F3R_FUSED_THREADS 512
#endif
constexpr int kFusedThreads = F3R_FUSED_THREADS;
constexpr int kFusedWarps = kFusedThreads / 32;
constexpr int kFusedChunkAlign = 64;  // rows; keeps every chunk 256-byte aligned
enum { ERR_BARRIER_TIMEOUT = 2 };

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add_u32(unsigned *p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier of a cooperative launch: arrival number `target` on the
// monotone counter `arrive` (G per barrier).  Thread 0 arrives with a release
// reduction (cumulative over the block's writes ordered before it by the
// block barrier) and polls with acquire loads.  Returns false (in every
// thread of the block) when the wait gave up.
__device__ __forceinline__ bool coop_sync(unsigned *arrive, unsigned target, int *err) {
    __shared__ int ok_sh;
    __syncthreads();
    if (threadIdx.x == 0) {
        red_release_add_u32(arrive, 1u);
        int ok = 1;
        const long long t0 = clock64();
        while (ld_acquire_u32(arrive) < target) {
            if (clock64() - t0 > kWaitCycles) {
                ok = 0;
                atomicOr(err, ERR_BARRIER_TIMEOUT);
                break;
            }
            __nanosleep(32);
        }
        ok_sh = ok;
    }
    __syncthreads();
    return ok_sh != 0;
}

// every block leaves through here; the last one resets the counters
__device__ __forceinline__ void coop_exit(unsigned *bar) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(bar + 1, 1u) == gridDim.x - 1) {
            bar[0] = 0u;
            bar[1] = 0u;
            __threadfence();
        }
    }
}

template <class T> struct FusedScratch {
    T *part;        // [kMaxDots][G] phase-A partials, then [G][2] phase-B partials
    unsigned *bar;  // arrivals, exits (zero between launches)
    int *err;
    int chunk;      // rows per block (multiple of kFusedChunkAlign)
    const T *hpart; // [l][hG] block totals of hA from the SpMV + dots (null: hA is in the scalars)
    int hG;
};

// block-wide sums of acc[0..nd) (and a max in acc[nd] when with_max) in warp
// order; thread d < nd (+1) returns its total through out
template <class T, int ND, int NW = kFusedWarps>
__device__ __forceinline__ void block_reduce(T (&acc)[ND], int nd, bool with_max, T *out) {
    __shared__ T sm[ND][NW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ntot = nd + (with_max ? 1 : 0);
#pragma unroll
    for (int d = 0; d < ND; ++d)
        if (d < ntot) {
            const T v = (with_max && d == nd) ? warp_max(acc[d]) : warp_sum(acc[d]);
            if (lane == 0) sm[d][warp] = v;
        }
    __syncthreads();
    if (threadIdx.x < ntot) {
        const int d = threadIdx.x;
        T s = sm[d][0];
        for (int w = 1; w < NW; ++w) s = (with_max && d == nd) ? fmax(s, sm[d][w]) : add_rn(s, sm[d][w]);
        out[d] = s;
    }
    __syncthreads();
}

// sum (or max) over the G block partials p[b * stride] by one warp, fixed
// order: lane l takes b = l, l + 32, ... in turn, then the warp combines the
// lanes.  A lane issues the loads of 8 partials before it adds them, so their
// L2 latencies overlap instead of adding up.
template <class T>
__device__ __forceinline__ T warp_sum_partials(const T *p, int G, int stride, bool is_max) {
    constexpr int K = 8;
    const int lane = threadIdx.x & 31;
    T s = (T)0;
    for (int b0 = lane; b0 < G; b0 += 32 * K) {
        T v[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int b = b0 + 32 * k;
            v[k] = (b < G) ? __ldcg(p + (size_t)b * stride) : (T)0;
        }
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (b0 + 32 * k < G) s = is_max ? fmax(s, v[k]) : add_rn(s, v[k]);
    }
    return is_max ? warp_max(s) : warp_sum(s);
}

template <class T, class TC, int CHILD, int MAXD>
__global__ void __launch_bounds__(kFusedThreads, (MAXD <= 8 && kFusedThreads <= 512) ? 2 : 1)
    k_cgs_fused(LevelDev<T> L, int j, int passes, int last_iter, int want_sigma, int do_norm, ChildOut<TC> co,
                FusedScratch<T> fs, GridRed<TC> grc) {
    if (stopped(L.flags, L.depth)) return;  // the same answer in every block: no barrier is entered
    constexpr int N = PackN<T>::N;
    extern __shared__ __align__(16) unsigned char fused_dsm[];
    T *ws = reinterpret_cast<T *>(fused_dsm);
    __shared__ T hs[MAXD];
    __shared__ T tot[MAXD + 2];
    const int G = gridDim.x;
    const int r0 = blockIdx.x * fs.chunk;
    const int cnt = max(0, min(L.n - r0, fs.chunk));
    const int nq = cnt / N;
    const T *__restrict__ V = L.V + r0;
    const T *__restrict__ w = L.w + r0;
    bool ok = true;

    // hA: the sum of the SpMV's block totals (every block alike; block 0 keeps
    // it for the Givens step), or the value a grid reduction left
    auto load_hA = [&]() {
        if (fs.hpart) {
            const int warp = threadIdx.x >> 5;
            for (int l = warp; l <= j; l += kFusedWarps) {
                const T sm = warp_sum_partials(fs.hpart + (size_t)l * fs.hG, fs.hG, 1, false);
                if ((threadIdx.x & 31) == 0) {
                    hs[l] = sm;
                    if (blockIdx.x == 0) L.hA()[l] = sm;
                }
            }
        } else if (threadIdx.x <= j) {
            hs[threadIdx.x] = L.hA()[threadIdx.x];
        }
    };

    // ---- phase A: w1 = w - V hA, partial hB
    if (passes == 2) {
        load_hA();
        __syncthreads();
        T acc[MAXD];
#pragma unroll
        for (int l = 0; l < MAXD; ++l) acc[l] = (T)0;
        for (int q = threadIdx.x; q < nq; q += blockDim.x) {
            Pack<T, N> wv = ldp<T, N>(w + (size_t)q * N);
            Pack<T, N> v[MAXD];
#pragma unroll
            for (int l = 0; l < MAXD; ++l)
                if (l <= j) v[l] = ldp<T, N>(V + (size_t)l * L.ld + (size_t)q * N);
#pragma unroll
            for (int l = 0; l < MAXD; ++l)
                if (l <= j)
#pragma unroll
                    for (int e = 0; e < N; ++e) wv.v[e] = fma_rn(-hs[l], v[l].v[e], wv.v[e]);
            stp<T, N>(ws + (size_t)q * N, wv);
#pragma unroll
            for (int l = 0; l < MAXD; ++l)
                if (l <= j)
#pragma unroll
                    for (int e = 0; e < N; ++e) acc[l] = fma_rn(v[l].v[e], wv.v[e], acc[l]);
        }
        for (int i = nq * N + threadIdx.x; i < cnt; i += blockDim.x) {
            T wi = w[i];
            T v[MAXD];
#pragma unroll
            for (int l = 0; l < MAXD; ++l)
                if (l <= j) {
                    v[l] = V[(size_t)l * L.ld + i];
                    wi = fma_rn(-hs[l], v[l], wi);
                }
            ws[i] = wi;
#pragma unroll
            for (int l = 0; l < MAXD; ++l)
                if (l <= j) acc[l] = fma_rn(v[l], wi, acc[l]);
        }
        block_reduce<T, MAXD>(acc, j + 1, false, tot);
        if (threadIdx.x <= j) fs.part[(size_t)threadIdx.x * G + blockIdx.x] = tot[threadIdx.x];
        ok = coop_sync(fs.bar, (unsigned)G, fs.err);
        if (ok) {
            const int warp = threadIdx.x >> 5;
            if (warp <= j) {
                const T s = warp_sum_partials(fs.part + (size_t)warp * G, G, 1, false);
                if ((threadIdx.x & 31) == 0) {
                    hs[warp] = s;
                    if (blockIdx.x == 0) L.hB()[warp] = s;
                }
            }
            __syncthreads();
        }
    } else {
        load_hA();
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) ws[i] = w[i];
        __syncthreads();
    }

    // ---- phase B: w2 = w1 - V h, ||w2||^2 and max|w2|
    T *part2 = fs.part + (size_t)kMaxDots * G;
    if (ok) {
        T acc[2] = {(T)0, (T)0};
        for (int q = threadIdx.x; q < nq; q += blockDim.x) {
            Pack<T, N> wv = ldp<T, N>(ws + (size_t)q * N);
#pragma unroll
            for (int l = 0; l < MAXD; ++l)
                if (l <= j) {
                    const Pack<T, N> v = ldp<T, N>(V + (size_t)l * L.ld + (size_t)q * N);
#pragma unroll
                    for (int e = 0; e < N; ++e) wv.v[e] = fma_rn(-hs[l], v.v[e], wv.v[e]);
                }
            stp<T, N>(ws + (size_t)q * N, wv);
#pragma unroll
            for (int e = 0; e < N; ++e) {
                acc[0] = fma_rn(wv.v[e], wv.v[e], acc[0]);
                acc[1] = fmax(acc[1], fabs(wv.v[e]));
            }
        }
        for (int i = nq * N + threadIdx.x; i < cnt; i += blockDim.x) {
            T wi = ws[i];
#pragma unroll
            for (int l = 0; l < MAXD; ++l)
                if (l <= j) wi = fma_rn(-hs[l], V[(size_t)l * L.ld + i], wi);
            ws[i] = wi;
            acc[0] = fma_rn(wi, wi, acc[0]);
            acc[1] = fmax(acc[1], fabs(wi));
        }
        block_reduce<T, 2>(acc, 1, true, tot);
        if (threadIdx.x < 2) part2[(size_t)blockIdx.x * 2 + threadIdx.x] = tot[threadIdx.x];
        ok = coop_sync(fs.bar, (passes == 2 ? 2u : 1u) * (unsigned)G, fs.err);
    }
    // the next kernel (a programmatic launch) may start its prologue now
    pdl_trigger();

    // ---- Givens step (block 0) and phase C: normalise into V[j+1] and the child
    if (ok) {
        const int warp = threadIdx.x >> 5;
        if (warp < 2) {
            const T s = warp_sum_partials(part2 + warp, G, 2, warp == 1);
            if ((threadIdx.x & 31) == 0) tot[warp] = s;
        }
        __syncthreads();
        const T hn = sqrt_rn(tot[0]);
        const T amax = tot[1];
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            T hcol[MAXD];
            const T *hA = L.hA(), *hB = L.hB();
            for (int l = 0; l <= j; ++l) hcol[l] = (passes == 2) ? add_rn(hA[l], hB[l]) : hA[l];
            givens_column(L, j, hcol, hn, last_iter != 0);
            T *ms = L.misc();
            if (want_sigma && hn > (T)0) {
                const T sig = pow2_scale_for(mul_rn(amax, ms[MS_INV]));
                ms[MS_SIGMA] = sig;
                ms[MS_INV_SIGMA] = div_rn((T)1, sig);
            } else {
                ms[MS_SIGMA] = (T)1;
                ms[MS_INV_SIGMA] = (T)1;
            }
        }
        if (do_norm && hn > (T)0 && isfinite(hn)) {
            // the same scalars block 0 derives in givens_column / above
            const T inv = div_rn((T)1, hn);
            const T sig = want_sigma ? pow2_scale_for(mul_rn(amax, inv)) : (T)1;
            T *out = L.V + (size_t)(j + 1) * L.ld + r0;
            if constexpr (CHILD == CHILD_F) {
                TC cacc[2] = {(TC)0, (TC)0};
                TC *cx = co.x + r0;
                for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
                    const T v = vstore(L.vround, mul_rn(ws[i], inv));
                    const TC c = Store<TC>::from(v);
                    out[i] = v;
                    cx[i] = c;
                    cacc[0] = fma_rn(c, c, cacc[0]);
                    cacc[1] = fmax(cacc[1], fabs(c));
                }
                grid_reduce<TC, 2>(cacc, 1, true, grc, [&](TC *res) {
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
                });
            } else {
                for (int q = threadIdx.x; q < nq; q += blockDim.x) {
                    const Pack<T, N> sv = ldp<T, N>(ws + (size_t)q * N);
                    Pack<T, N> op;
#pragma unroll
                    for (int e = 0; e < N; ++e) op.v[e] = vstore(L.vround, mul_rn(sv.v[e], inv));
                    stp<T, N>(out + (size_t)q * N, op);
                    if constexpr (CHILD == CHILD_R) {
                        Pack<TC, N> cp;
#pragma unroll
                        for (int e = 0; e < N; ++e) cp.v[e] = Store<TC>::from(mul_rn(sig, op.v[e]));
                        stp<TC, N>(co.x + r0 + (size_t)q * N, cp);
                    }
                }
                for (int i = nq * N + threadIdx.x; i < cnt; i += blockDim.x) {
                    const T v = vstore(L.vround, mul_rn(ws[i], inv));
                    out[i] = v;
                    if constexpr (CHILD == CHILD_R) co.x[r0 + i] = Store<TC>::from(mul_rn(sig, v));
                }
            }
        }
    }
    coop_exit(fs.bar);
}

// ---------------------------------------------------------------------------
// The outer (fp64) level after w = A z_j: CGS2 against V[0..j], the Givens
// step with the convergence estimate, and the normalisation of V[j+1] with
// the cast (times D^-1/2) into the first inner level's V[0] and its beta, in
// one cooperative launch with w kept in shared memory (j read on the device):
//   phase 0  hA = V^T w                                           | barrier 1
//   phase 1  w1 = w - V hA (row sweep), hB = V^T w1 (vector sweep)| barrier 2
//   phase 2  w2 = w1 - V hB, ||w2||^2                             | barrier 3
//   phase 3  V[j+1] = w2 / ||w2||, child input and beta; j += 1
// Dot products sweep the vectors in groups of 8 with per-block partial sums
// [vector][block]; phase-0 and phase-1 partials use separate regions so that a
// block still reading one never races a block writing the next.
constexpr int kOuterGroup = 8;
constexpr int kOuterUnroll = 4;  // 16-byte packs per thread in flight in the outer sweeps

template <class TC, int CHILD>
__global__ void __launch_bounds__(kFusedThreads, kFusedThreads <= 512 ? 2 : 1)
    k_outer_cgs_fused(LevelDev<double> L, int passes, ChildOut<TC> co, FusedScratch<double> fs, GridRed<TC> grc) {
    constexpr int N = 2;  // double2 packs
    extern __shared__ __align__(16) unsigned char fused_dsm[];
    double *ws = reinterpret_cast<double *>(fused_dsm);
    __shared__ double hs[kMaxOuterM + 1];
    __shared__ double tot[kOuterGroup + 1];
    __shared__ double wsum[kOuterGroup][kFusedWarps];  // the warps' sums of up to kOuterGroup dot products
    const int j = *L.jptr;
    const int nv = j + 1;
    const int G = gridDim.x;
    const int r0 = blockIdx.x * fs.chunk;
    const int cnt = max(0, min(L.n - r0, fs.chunk));
    const int nq = cnt / N;
    const double *__restrict__ V = L.V + r0;
    double *partA = fs.part;
    double *partB = fs.part + (size_t)(kMaxOuterM + 1) * G;
    double *partC = fs.part + (size_t)2 * (kMaxOuterM + 1) * G;
    unsigned target = 0;
    bool ok = true;

    for (int i = threadIdx.x; i < cnt; i += blockDim.x) ws[i] = L.w[r0 + i];
    __syncthreads();

    // The block's rows of each basis vector are streamed one vector at a time
    // (one contiguous run per block in flight, kOuterUnroll packs per thread),
    // with the same fma order per sum and per element as a row-major sweep.
    // dots V[0..nv)^T ws into part[l * G + block]: a thread's sum over its
    // packs, the warp's butterfly sum, the warps' sums in warp order (one
    // vector loop, so that the sweep's code is not repeated per vector)
    auto dots = [&](double *part) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll 1
        for (int l = 0; l < nv; ++l) {
            const double *__restrict__ Vl = V + (size_t)l * L.ld;
            double a = 0.0;
            for (int q0 = threadIdx.x; q0 < nq; q0 += blockDim.x * kOuterUnroll) {
                Pack<double, N> v[kOuterUnroll];
#pragma unroll
                for (int u = 0; u < kOuterUnroll; ++u) {
                    const int q = q0 + u * (int)blockDim.x;
                    if (q < nq) v[u] = ldp<double, N>(Vl + (size_t)q * N);
                }
#pragma unroll
                for (int u = 0; u < kOuterUnroll; ++u) {
                    const int q = q0 + u * (int)blockDim.x;
                    if (q < nq) {
                        const Pack<double, N> wv = ldp<double, N>(ws + (size_t)q * N);
#pragma unroll
                        for (int e = 0; e < N; ++e) a = fma_rn(v[u].v[e], wv.v[e], a);
                    }
                }
            }
            for (int i = nq * N + threadIdx.x; i < cnt; i += blockDim.x) a = fma_rn(Vl[i], ws[i], a);
            a = warp_sum(a);
            const int k = l % kOuterGroup;
            if (lane == 0) wsum[k][warp] = a;
            if (k == kOuterGroup - 1 || l == nv - 1) {
                __syncthreads();
                if ((int)threadIdx.x <= k) {
                    double sm = wsum[threadIdx.x][0];
                    for (int w = 1; w < kFusedWarps; ++w) sm = add_rn(sm, wsum[threadIdx.x][w]);
                    part[(size_t)(l - k + threadIdx.x) * G + blockIdx.x] = sm;
                }
                __syncthreads();
            }
        }
    };
    // hs[l] = sum over blocks of part[l * G + b] (fixed order, every block alike)
    auto gather = [&](const double *part, double *rec) {
        const int warp = threadIdx.x >> 5;
        for (int l = warp; l < nv; l += kFusedWarps) {
            const double sm = warp_sum_partials(part + (size_t)l * G, G, 1, false);
            if ((threadIdx.x & 31) == 0) {
                hs[l] = sm;
                if (blockIdx.x == 0) rec[l] = sm;
            }
        }
        __syncthreads();
    };
    // ws -= V hs (fma in l order per element; a thread owns the same
    // positions of ws for every l)
    auto update = [&]() {
        for (int l = 0; l < nv; ++l) {
            const double h = hs[l];
            const double *__restrict__ Vl = V + (size_t)l * L.ld;
            for (int q0 = threadIdx.x; q0 < nq; q0 += blockDim.x * kOuterUnroll) {
                Pack<double, N> v[kOuterUnroll];
#pragma unroll
                for (int u = 0; u < kOuterUnroll; ++u) {
                    const int q = q0 + u * (int)blockDim.x;
                    if (q < nq) v[u] = ldp<double, N>(Vl + (size_t)q * N);
                }
#pragma unroll
                for (int u = 0; u < kOuterUnroll; ++u) {
                    const int q = q0 + u * (int)blockDim.x;
                    if (q < nq) {
                        Pack<double, N> wv = ldp<double, N>(ws + (size_t)q * N);
#pragma unroll
                        for (int e = 0; e < N; ++e) wv.v[e] = fma_rn(-h, v[u].v[e], wv.v[e]);
                        stp<double, N>(ws + (size_t)q * N, wv);
                    }
                }
            }
            for (int i = nq * N + threadIdx.x; i < cnt; i += blockDim.x) ws[i] = fma_rn(-h, Vl[i], ws[i]);
        }
        __syncthreads();
    };

    // phase 0
    dots(partA);
    target += G;
    ok = coop_sync(fs.bar, target, fs.err);
    if (ok) gather(partA, L.hA());
    // phase 1
    if (ok && passes == 2) {
        update();
        dots(partB);
        target += G;
        ok = coop_sync(fs.bar, target, fs.err);
        if (ok) gather(partB, L.hB());
    }
    // phase 2
    if (ok) {
        update();
        double acc[1] = {0.0};
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) acc[0] = fma_rn(ws[i], ws[i], acc[0]);
        block_reduce<double, 1>(acc, 1, false, tot);
        if (threadIdx.x == 0) partC[blockIdx.x] = tot[0];
        target += G;
        ok = coop_sync(fs.bar, target, fs.err);
    }
    // Givens (block 0) and phase 3
    if (ok) {
        if (threadIdx.x < 32) {
            const double sm = warp_sum_partials(partC, G, 1, false);
            if (threadIdx.x == 0) tot[0] = sm;
        }
        __syncthreads();
        const double hn = sqrt_rn(tot[0]);
        // 1/||w|| as the Givens step records it; a breakdown keeps the previous value
        const double inv_prev = L.misc()[MS_INV];
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            double hcol[kMaxOuterM + 1];
            const double *hA = L.hA(), *hB = L.hB();
            for (int l = 0; l < nv; ++l) hcol[l] = (passes == 2) ? add_rn(hA[l], hB[l]) : hA[l];
            givens_column(L, j, hcol, hn, false);
            double *ms = L.misc();
            ms[MS_EST] = div_rn(fabs(L.g()[L.fl()[IF_KDIM]]), ms[MS_NB]);
        }
        const double inv = (hn > 0.0 && isfinite(hn)) ? div_rn(1.0, hn) : inv_prev;
        double *out = L.V + (size_t)(j + 1) * L.ld + r0;
        // block 0's thread 0 runs the Givens step (a serial chain of fp64
        // operations) above while its other warps take the block's rows
        const int r_first = (blockIdx.x == 0) ? (int)threadIdx.x - 32 : (int)threadIdx.x;
        const int r_step = (blockIdx.x == 0) ? (int)blockDim.x - 32 : (int)blockDim.x;
        if constexpr (CHILD == CHILD_F) {
            TC cacc[2] = {(TC)0, (TC)0};
            for (int i = r_first; i >= 0 && i < cnt; i += r_step) {
                const double v = mul_rn(ws[i], inv);
                const TC c = co.dsc ? Store<TC>::from(mul_rn(co.dsc[r0 + i], v)) : Store<TC>::from(v);
                out[i] = v;
                co.x[r0 + i] = c;
                cacc[0] = fma_rn(c, c, cacc[0]);
                cacc[1] = fmax(cacc[1], fabs(c));
            }
            grid_reduce<TC, 2>(cacc, 1, true, grc, [&](TC *res) {
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
            });
        } else {
            for (int i = r_first; i >= 0 && i < cnt; i += r_step) out[i] = mul_rn(ws[i], inv);
        }
        // every block read j at its start: close outer iteration j
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(const_cast<int *>(L.jptr), 1);
    }
    coop_exit(fs.bar);
}

}  // namespace f3r
