// One whole iteration j of the innermost FGMRES level of F3R in a single
// cooperative launch (fp16 A and Richardson storage, fp32 vectors, Jacobi M,
// m4 = 2, a plain Richardson call):
//   phase R   Z[j] = R(v16_j): the fused two-step Richardson call      | barrier
//   phase S   w = A16 Z[j] (into shared memory), hA = V[0..j]^T w      | barrier
//   phase A   w1 = w - V hA, hB = V^T w1                               | barrier
//   phase B   w2 = w1 - V hB, ||w2||^2, max|w2|                         | barrier
//   phase C   Givens (block 0); V[j+1] = w2 / ||w2||, v16_{j+1} = fp16(sigma V[j+1])
// Phases R and S stream the block's own contiguous range of 256-row tiles
// through the shared-memory ring of stage.cuh (bulk copies + mbarriers, a
// producer warp), so the rows whose w phase S produces are the rows the
// vector phases own; w never leaves the SM.  Every row sum, rounding point
// and dot-product order is that of k_rich2_st, k_spmv_dots_st and
// k_cgs_fused, except that the partial dot products are per block of this
// grid.  The kernel replaces three launches (and their ramps and tails) per
// iteration; a stopped level returns at once.
#pragma once
#include "fused.cuh"
#include "staged.cuh"

namespace f3r {

struct StepArgs {
    Sell A;
    const h16 *a16;
    const float *rs;       // row scales (null without row scaling)
    const h16 *v16;        // R input of this iteration (sigma-scaled fp16)
    const h16 *m16;        // Jacobi M
    float *zout;           // Z[j]
    const float *omega;    // w_1, w_2
    unsigned long long *counters;
    h16 *v16_next;         // R input of the next iteration
    int stage_bytes;
    int *err;
    unsigned *bar;         // grid barrier counters (zero between launches)
    float *part;           // [kMaxDots][G] hA partials, [kMaxDots][G] hB partials, [G][2] norm / max
};

template <int S, int MAXD>
__global__ void __launch_bounds__(kStagedThreads) k_f3_step(StepArgs a, LevelDev<float> L, int j, int last_iter,
                                                            int want_sigma, int do_norm) {
    if (stopped(L.flags, L.depth)) return;  // uniform: no barrier entered
    extern __shared__ __align__(128) char dsm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int G = gridDim.x;
    const int2 tr = tile_range(a.A);
    const int r0 = tr.x * kTileRows;
    const int cnt = max(0, min(L.n, tr.y * kTileRows) - r0);
    // shared memory: [2 x (S full + S empty) mbarriers][ring][w chunk]
    uint64_t *barR = reinterpret_cast<uint64_t *>(dsm);
    uint64_t *barS = barR + 2 * S;
    char *ring = dsm + kBarBytes;
    float *ws = reinterpret_cast<float *>(ring + (size_t)S * a.stage_bytes);
    __shared__ float hs[MAXD];
    __shared__ float tot[MAXD + 2];
    unsigned target = 0;
    bool ok = true;

    // ---- phase R: Z[j] = R(v16) for this block's rows
    {
        const float w1 = a.omega[0], w2 = a.omega[1];
        const float inv_sigma = L.misc()[MS_INV_SIGMA];
        const bool sok = staged_tiles<h16, S>(a.A, a.a16, tr.x, tr.y, ring, a.stage_bytes, barR, barR + S, Extra(), a.err,
                                  [&](int s, const StageView<h16> &st) {
                                      float acc = staged_row<float>(st, lane, [&](int c) {
                                          return rnd<h16>(fma_rn(w1, mul_rn(__half2float(__ldg(a.m16 + c)),
                                                                            __half2float(__ldg(a.v16 + c))),
                                                                 0.0f));
                                      });
                                      const int i = s * kSlice + lane;
                                      if (a.rs) acc = mul_rn(acc, __ldg(a.rs + i));
                                      if (i < L.n) {
                                          const float vi = __half2float(a.v16[i]), mi = __half2float(a.m16[i]);
                                          const float z1 = rnd<h16>(fma_rn(w1, mul_rn(mi, vi), 0.0f));
                                          const float ri = rnd<h16>(sub_rn(vi, acc));
                                          const float z2 = rnd<h16>(fma_rn(w2, mul_rn(mi, ri), z1));
                                          a.zout[i] = mul_rn(z2, inv_sigma);
                                      }
                                  });
        ok = __syncthreads_and(sok) != 0;  // block-uniform from here on
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            atomicAdd(a.counters + 0, 2ull);
            atomicAdd(a.counters + 1, 1ull);
        }
    }
    target += G;
    ok = coop_sync(a.bar, target, a.err) && ok;

    // ---- phase S: w = A16 Z[j] into shared memory, hA partials
    if (ok) {
        float acc[MAXD];
#pragma unroll
        for (int l = 0; l < MAXD; ++l) acc[l] = 0.0f;
        const float *x = a.zout;  // written in phase R by other blocks: L1-cached loads of fresh lines
        Extra ex;
        ex.base = L.V;
        ex.count = j + 1;
        ex.ld = L.ld;
        ex.esize = sizeof(float);
        const bool sok = staged_tiles<h16, S>(a.A, a.a16, tr.x, tr.y, ring, a.stage_bytes, barS, barS + S, ex, a.err,
                                  [&](int s, const StageView<h16> &v) {
                                      float y = staged_row<float>(v, lane, [&](int c) { return __ldca(x + c); });
                                      const int i = s * kSlice + lane;
                                      if (a.rs) y = mul_rn(y, __ldg(a.rs + i));
                                      if (i < L.n) {
                                          ws[i - r0] = y;
#pragma unroll
                                          for (int l = 0; l < MAXD; ++l)
                                              if (l <= j) acc[l] = fma_rn(v.template ext<float>(l)[lane], y, acc[l]);
                                      }
                                  });
        ok = __syncthreads_and(sok) != 0;
        block_reduce<float, MAXD, kStagedThreads / 32>(acc, j + 1, false, tot);
        if (threadIdx.x <= j) a.part[(size_t)threadIdx.x * G + blockIdx.x] = tot[threadIdx.x];
    }
    target += G;
    ok = coop_sync(a.bar, target, a.err) && ok;
    if (ok) {
        for (int l = warp; l <= j; l += kStagedThreads / 32) {
            const float sm = warp_sum_partials(a.part + (size_t)l * G, G, 1, false);
            if (lane == 0) {
                hs[l] = sm;
                if (blockIdx.x == 0) L.hA()[l] = sm;
            }
        }
        __syncthreads();
    }

    // ---- phase A: w1 = w - V hA, hB partials (V rows from global / L2); the
    // hB partials go to their own region: a block may still be reading hA's
    const float *__restrict__ V = L.V + r0;
    float *partB = a.part + (size_t)kMaxDots * G;
    if (ok) {
        float acc[MAXD];
#pragma unroll
        for (int l = 0; l < MAXD; ++l) acc[l] = 0.0f;
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            float wi = ws[i];
            float v[MAXD];
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
        block_reduce<float, MAXD, kStagedThreads / 32>(acc, j + 1, false, tot);
        if (threadIdx.x <= j) partB[(size_t)threadIdx.x * G + blockIdx.x] = tot[threadIdx.x];
        __syncthreads();
    }
    target += G;
    ok = coop_sync(a.bar, target, a.err) && ok;
    if (ok) {
        for (int l = warp; l <= j; l += kStagedThreads / 32) {
            const float sm = warp_sum_partials(partB + (size_t)l * G, G, 1, false);
            if (lane == 0) {
                hs[l] = sm;
                if (blockIdx.x == 0) L.hB()[l] = sm;
            }
        }
        __syncthreads();
    }

    // ---- phase B: w2 = w1 - V hB, ||w2||^2, max|w2|
    float *part2 = a.part + (size_t)2 * kMaxDots * G;
    if (ok) {
        float acc[2] = {0.0f, 0.0f};
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            float wi = ws[i];
#pragma unroll
            for (int l = 0; l < MAXD; ++l)
                if (l <= j) wi = fma_rn(-hs[l], V[(size_t)l * L.ld + i], wi);
            ws[i] = wi;
            acc[0] = fma_rn(wi, wi, acc[0]);
            acc[1] = fmaxf(acc[1], fabsf(wi));
        }
        block_reduce<float, 2, kStagedThreads / 32>(acc, 1, true, tot);
        if (threadIdx.x < 2) part2[(size_t)blockIdx.x * 2 + threadIdx.x] = tot[threadIdx.x];
        __syncthreads();
    }
    target += G;
    ok = coop_sync(a.bar, target, a.err) && ok;

    // ---- phase C: Givens (block 0), normalise and cast into the next R input
    if (ok) {
        if (warp < 2) {
            const float sm = warp_sum_partials(part2 + warp, G, 2, warp == 1);
            if (lane == 0) tot[warp] = sm;
        }
        __syncthreads();
        const float hn = sqrt_rn(tot[0]);
        const float amax = tot[1];
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            float hcol[MAXD];
            const float *hA = L.hA(), *hB = L.hB();
            for (int l = 0; l <= j; ++l) hcol[l] = add_rn(hA[l], hB[l]);
            givens_column(L, j, hcol, hn, last_iter != 0);
            float *ms = L.misc();
            if (want_sigma && hn > 0.0f) {
                const float sig = pow2_scale_for(mul_rn(amax, ms[MS_INV]));
                ms[MS_SIGMA] = sig;
                ms[MS_INV_SIGMA] = div_rn(1.0f, sig);
            } else {
                ms[MS_SIGMA] = 1.0f;
                ms[MS_INV_SIGMA] = 1.0f;
            }
        }
        if (do_norm && hn > 0.0f && isfinite(hn)) {
            const float inv = div_rn(1.0f, hn);
            const float sig = want_sigma ? pow2_scale_for(mul_rn(amax, inv)) : 1.0f;
            float *out = L.V + (size_t)(j + 1) * L.ld + r0;
            h16 *vo = a.v16_next + r0;
            for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
                const float v = mul_rn(ws[i], inv);
                out[i] = v;
                vo[i] = __float2half_rn(mul_rn(sig, v));
            }
        }
    }
    coop_exit(a.bar);
}

}  // namespace f3r
