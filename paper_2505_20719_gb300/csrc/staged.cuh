// SELL kernels whose matrix slices are staged into shared memory by bulk
// asynchronous copies (stage.cuh): the inner-level SpMV with fused CGS dot
// products, the fused m4 = 2 Richardson call, the stand-alone SpMV and the
// outer fp64 SpMV.  Each lane still sums its row in CSR order with fused
// multiply-add, so results equal the unstaged kernels bit for bit.
//
// Blocks have kWarps consumer warps plus one producer warp (kStagedThreads).
// Dynamic shared memory per block: [S full + S empty mbarriers, padded to
// 256 B][ring of S stages of `stage_bytes`].  Block b owns the contiguous tiles
// [b * per, (b + 1) * per), per = ceil(tiles / gridDim.x).
#pragma once
#include "kernels.cuh"
#include "rich.cuh"
#include "stage.cuh"

namespace f3r {

constexpr int kBarBytes = 256;
constexpr int kStagedThreads = kBlock + 32;

struct StageCfg {
    int stage_bytes;
    int *err;
};

__device__ __forceinline__ char *block_ring(char *dsm) { return dsm + kBarBytes; }
__device__ __forceinline__ uint64_t *block_full(char *dsm) { return reinterpret_cast<uint64_t *>(dsm); }
__device__ __forceinline__ uint64_t *block_empty(char *dsm) { return reinterpret_cast<uint64_t *>(dsm) + 8; }

// this block's contiguous range of tiles
__device__ __forceinline__ int2 tile_range(const Sell &A) {
    const int ntiles = (A.nslices + kTileSlices - 1) / kTileSlices;
    const int per = (ntiles + gridDim.x - 1) / gridDim.x;
    const int b = blockIdx.x * per;
    return make_int2(min(b, ntiles), min(b + per, ntiles));
}

// one row of a staged slice: sum_k a_k x(c_k) in CSR order.  Entries go in
// groups of kRowGroup: all gathers of a group are issued before its first
// fused multiply-add, so a row of up to kRowGroup entries waits for one
// round of gather latency, not one per entry (the accumulation order is
// unchanged).
constexpr int kRowGroup = 8;

// index of entry q of the lane's row: the int32 column (-1 for padding) or,
// for windowed tiles, the 16-bit window index (padding: the zero slot, so
// every windowed entry is gathered and multiplied; never negative)
template <bool WIN, class TA>
__device__ __forceinline__ int entry_index(const StageView<TA> &v, int q, int lane) {
    if constexpr (WIN) return (int)v.lcol[q * kSlice + lane];
    else return v.col[q * kSlice + lane];
}

// a slice exactly W entries wide: W gathers issued, then W fused multiply-adds
// (no slot of the group is spent on entries past the width).  gx(c) gets the
// column (plain tiles) or the window index (WIN).
template <class TC, int W, bool WIN, class TA, class GX>
__device__ __forceinline__ TC staged_row_w(const StageView<TA> &v, int lane, GX gx) {
    int c[W];
    TC a[W], xv[W];
#pragma unroll
    for (int q = 0; q < W; ++q) {
        c[q] = entry_index<WIN>(v, q, lane);
        a[q] = to_c<TC>(v.val[q * kSlice + lane]);
    }
#pragma unroll
    for (int q = 0; q < W; ++q) xv[q] = (c[q] >= 0) ? gx(c[q]) : (TC)0;
    TC acc = (TC)0;
#pragma unroll
    for (int q = 0; q < W; ++q)
        if (c[q] >= 0) acc = fma_rn(a[q], xv[q], acc);
    return acc;
}

template <class TC, bool WIN = false, class TA, class GX>
__device__ __forceinline__ TC staged_row(const StageView<TA> &v, int lane, GX gx) {
    switch (v.w) {  // slice widths up to one group: exact-width code
        case 0: return (TC)0;
        case 1: return staged_row_w<TC, 1, WIN>(v, lane, gx);
        case 2: return staged_row_w<TC, 2, WIN>(v, lane, gx);
        case 3: return staged_row_w<TC, 3, WIN>(v, lane, gx);
        case 4: return staged_row_w<TC, 4, WIN>(v, lane, gx);
        case 5: return staged_row_w<TC, 5, WIN>(v, lane, gx);
        case 6: return staged_row_w<TC, 6, WIN>(v, lane, gx);
        case 7: return staged_row_w<TC, 7, WIN>(v, lane, gx);
        case 8: return staged_row_w<TC, 8, WIN>(v, lane, gx);
        default: break;
    }
    TC acc = (TC)0;
    for (int k0 = 0; k0 < v.w; k0 += kRowGroup) {
        int c[kRowGroup];
        TC a[kRowGroup], xv[kRowGroup];
#pragma unroll
        for (int q = 0; q < kRowGroup; ++q) {
            const int k = k0 + q;
            c[q] = (k < v.w) ? entry_index<WIN>(v, k, lane) : -1;
            a[q] = (k < v.w) ? to_c<TC>(v.val[k * kSlice + lane]) : (TC)0;
        }
#pragma unroll
        for (int q = 0; q < kRowGroup; ++q) xv[q] = (c[q] >= 0) ? gx(c[q]) : (TC)0;
#pragma unroll
        for (int q = 0; q < kRowGroup; ++q)
            if (c[q] >= 0) acc = fma_rn(a[q], xv[q], acc);
    }
    return acc;
}

// w = A Z[j] (times the row scale), hA = V[0..j]^T w; V rows staged with the
// slice.  hpart != null: the block totals of hA go to hpart[l * grid + block]
// for the fused CGS2 launch that follows to sum; else a grid reduction
// leaves hA itself in the level's scalars.
template <class TA, class T, int S, int MAXD, bool WIN = false>
__global__ void __launch_bounds__(kStagedThreads) k_spmv_dots_st(Sell A, const TA *__restrict__ val,
                                                         const float *__restrict__ rs, LevelDev<T> L, int j,
                                                         GridRed<T> gr, StageCfg cfg, T *hpart,
                                                         Window wn = Window()) {
    // programmatic launch: the matrix and basis tiles of the first stages are
    // requested before the wait for the Richardson call that writes z
    extern __shared__ __align__(128) char dsm[];
    const int lane = threadIdx.x & 31;
    const T *__restrict__ x = L.Z + (size_t)j * L.ld;
    T acc[MAXD];
#pragma unroll
    for (int l = 0; l < MAXD; ++l) acc[l] = (T)0;
    Extra ex;
    ex.base = L.V;
    ex.count = j + 1;
    ex.ld = L.ld;
    ex.esize = sizeof(T);
    const int2 tr = tile_range(A);
    bool go = false;  // the gate passed (the same in every thread)
    wn.x = x;
    staged_tiles_gated<TA, S, true, WIN>(A, val, tr.x, tr.y, block_ring(dsm), cfg.stage_bytes, block_full(dsm), block_empty(dsm), ex, cfg.err,
                        [&](int s, const StageView<TA> &v) {
                             const int i = s * kSlice + lane;
                             const T rsi = rs ? (T)__ldg(rs + i) : (T)1;  // requested before the row sum
                             T y;
                             if constexpr (WIN) y = staged_row<T, true>(v, lane, [&](int c) { return v.template xwin<T>()[c]; });
                             else y = staged_row<T>(v, lane, [&](int c) { return __ldg(x + c); });
                             if (rs) y = mul_rn(y, rsi);
                             if (i < L.n) {
                                 L.w[i] = y;
#pragma unroll
                                 for (int l = 0; l < MAXD; ++l)
                                     if (l <= j) acc[l] = fma_rn(v.template ext<T>(l)[lane], y, acc[l]);
                             }
                         },
                        [&] {
                            pdl_wait();
                            go = !stopped(L.flags, L.depth);
                            return go;
                        }, wn);
    if (!go) return;  // a stopped level, in every block alike
    pdl_trigger();
    if (hpart) {
        block_partials<T, MAXD>(acc, j + 1, hpart);
        return;
    }
    grid_reduce<T, MAXD>(acc, j + 1, false, gr, [&](T *res) {
        T *hA = L.hA();
        for (int l = 0; l <= j; ++l) hA[l] = res[l];
    });
}

// fused plain Richardson call with m4 = 2 (see k_rich2).  UNIT: every entry
// of M is 1, so M v is v itself (mul(1, v) = v) and M is not loaded.
// WIN (with UNIT): windowed tiles, v gathered from the stage's x window.
template <class TA, class VS, class TC, class TP, int S, bool UNIT = false, bool WIN = false>
__global__ void __launch_bounds__(kStagedThreads) k_rich2_st(Sell A, const TA *__restrict__ val, const float *__restrict__ rs,
                                                     const VS *__restrict__ v, const VS *__restrict__ mv, TP *out,
                                                     const TP *par_misc, RichDev<TC> R, const int *flags,
                                                     int check_depth, int n, StageCfg cfg, Window wn = Window()) {
    static_assert(!WIN || UNIT, "windowed Richardson calls gather v alone (M = I)");
    // programmatic launch: the first stages' matrix tiles are requested
    // before the wait for the kernel that writes v, the weights and sigma
    extern __shared__ __align__(128) char dsm[];
    const int lane = threadIdx.x & 31;
    TC w1 = (TC)0, w2 = (TC)0;
    TP inv_sigma = (TP)1;
    const int2 tr = tile_range(A);
    bool go = false;  // the gate passed (the same in every thread)
    wn.x = v;
    staged_tiles_gated<TA, S, false, WIN>(A, val, tr.x, tr.y, block_ring(dsm), cfg.stage_bytes, block_full(dsm), block_empty(dsm), Extra(), cfg.err,
                        [&](int s, const StageView<TA> &st) {
                             const int i = s * kSlice + lane;
                             const TC rsi = rs ? (TC)__ldg(rs + i) : (TC)1;  // requested before the row sum
                             TC acc;
                             if constexpr (WIN) {
                                 const VS *xw = st.template xwin<VS>();
                                 acc = staged_row<TC, true>(st, lane, [&](int c) {
                                     return rnd<VS>(fma_rn(w1, to_c<TC>(xw[c]), (TC)0));
                                 });
                             } else {
                                 acc = staged_row<TC>(st, lane, [&](int c) {
                                     const TC vc = to_c<TC>(__ldg(v + c));
                                     return rnd<VS>(fma_rn(w1, UNIT ? vc : mul_rn(to_c<TC>(__ldg(mv + c)), vc), (TC)0));
                                 });
                             }
                             if (rs) acc = mul_rn(acc, rsi);
                             if (i < n) {
                                 TC vi;  // the row's own v: from the window (it holds the tile's rows)
                                 if constexpr (WIN) vi = to_c<TC>(st.template xwin<VS>()[st.own + st.row0 + lane]);
                                 else vi = to_c<TC>(v[i]);
                                 const TC z1 = rnd<VS>(fma_rn(w1, UNIT ? vi : mul_rn(to_c<TC>(mv[i]), vi), (TC)0));
                                 const TC ri = rnd<VS>(sub_rn(vi, acc));
                                 const TC z2 = rnd<VS>(fma_rn(w2, UNIT ? ri : mul_rn(to_c<TC>(mv[i]), ri), z1));
                                 out[i] = mul_rn((TP)z2, inv_sigma);
                             }
                         },
                        [&] {
                            pdl_wait();
                            if (stopped(flags, check_depth)) return false;
                            w1 = R.omega[0];
                            w2 = R.omega[1];
                            inv_sigma = par_misc[MS_INV_SIGMA];
                            go = true;
                            return true;
                        }, wn);
    if (!go) return;
    pdl_trigger();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        atomicAdd(R.counters + 0, 2ull);
        atomicAdd(R.counters + 1, 1ull);
    }
}

// stand-alone y = A x
template <class TA, class TX, class TY, int S, bool WIN = false>
__global__ void __launch_bounds__(kStagedThreads) k_spmv_st(Sell A, const TA *__restrict__ val, const float *__restrict__ rs,
                                                    const TX *__restrict__ x, TY *y, StageCfg cfg,
                                                    Window wn = Window()) {
    pdl_enter();
    extern __shared__ __align__(128) char dsm[];
    const int lane = threadIdx.x & 31;
    const int2 tr = tile_range(A);
    wn.x = x;
    staged_tiles<TA, S, false, WIN>(A, val, tr.x, tr.y, block_ring(dsm), cfg.stage_bytes, block_full(dsm), block_empty(dsm), Extra(), cfg.err,
                        [&](int s, const StageView<TA> &st) {
                             const int i = s * kSlice + lane;
                             const TY rsi = rs ? (TY)__ldg(rs + i) : (TY)1;  // requested before the row sum
                             TY acc;
                             if constexpr (WIN) acc = staged_row<TY, true>(st, lane, [&](int c) { return to_c<TY>(st.template xwin<TX>()[c]); });
                             else acc = staged_row<TY>(st, lane, [&](int c) { return to_c<TY>(__ldg(x + c)); });
                             if (rs) acc = mul_rn(acc, rsi);
                             if (i < A.n) y[i] = acc;
                         }, wn);
}

// outer level: Z[j] = z (the inner nest's output) and w = A z, original fp64 A
template <int S, bool WIN = false>
__global__ void __launch_bounds__(kStagedThreads) k_outer_spmv_st(Sell A, const double *__restrict__ a, LevelDev<double> L,
                                                          const double *__restrict__ z, StageCfg cfg,
                                                          Window wn = Window()) {
    pdl_enter();
    extern __shared__ __align__(128) char dsm[];
    const int lane = threadIdx.x & 31;
    const int j = *L.jptr;
    double *zj = L.Z + (size_t)j * L.ld;
    const int2 tr = tile_range(A);
    wn.x = z;
    staged_tiles<double, S, false, WIN>(A, a, tr.x, tr.y, block_ring(dsm), cfg.stage_bytes, block_full(dsm), block_empty(dsm), Extra(), cfg.err,
                            [&](int s, const StageView<double> &st) {
                                 double y;
                                 if constexpr (WIN) y = staged_row<double, true>(st, lane, [&](int c) { return st.template xwin<double>()[c]; });
                                 else y = staged_row<double>(st, lane, [&](int c) { return __ldg(z + c); });
                                 const int i = s * kSlice + lane;
                                 if (i < L.n) {
                                     L.w[i] = y;
                                     zj[i] = z[i];
                                 }
                             }, wn);
}

}  // namespace f3r
