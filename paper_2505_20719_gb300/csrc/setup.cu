// Setup: validate the CSR matrix, symmetric diagonal scaling
// (Sec. 5), conversion to sliced ELLPACK with 32-row slices (Sec. 5.2) and the
// fp64 / fp32 / fp16 / bf16 copies of the scaled matrix (Table 1).  Runs on
// the device after one upload of the CSR arrays.
#include <algorithm>
#include <cstdlib>

#include "ctx.h"
#include "stage.cuh"

namespace f3r {

__global__ void k_validate(const int *rp, const int *ci, int n, long long nnz, int *err) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int b = rp[i], e = rp[i + 1];
        if (i == 0 && b != 0) atomicOr(err, 1);
        if (i == n - 1 && (long long)e != nnz) atomicOr(err, 2);
        if (e < b) atomicOr(err, 4);
        if (e >= b && b >= 0 && (long long)e <= nnz) {
            for (int k = b; k < e; ++k) {
                const int c = ci[k];
                if (c < 0 || c >= n) {
                    atomicOr(err, 8);
                    break;
                }
            }
        } else {
            atomicOr(err, 16);
        }
    }
}

// D^-1/2 from the (last stored) diagonal entry; ones without scaling or
// when the diagonal is zero / missing.
__global__ void k_diag_scale(const int *rp, const int *ci, const double *val, int n, int scale, double *dsc) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double di = 0.0;
        for (int k = rp[i]; k < rp[i + 1]; ++k)
            if (ci[k] == i) di = val[k];
        dsc[i] = (scale && di != 0.0) ? div_rn(1.0, sqrt_rn(fabs(di))) : 1.0;
    }
}

// width of every slice = longest row in it
__global__ void k_slice_width(const int *rp, int n, int nslices, int *width) {
    const int lane = threadIdx.x & 31;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int s = wid; s < nslices; s += nw) {
        const int i = s * kSlice + lane;
        int len = (i < n) ? rp[i + 1] - rp[i] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, o));
        if (lane == 0) width[s] = len;
    }
}

// s_i = 2^ceil(log2 max_j |A^_ij|) (1 for an empty or zero row)
__device__ __forceinline__ double row_scale_pow2(double mx) {
    if (!(mx > 0.0) || isinf(mx)) return 1.0;
    int e;
    const double f = frexp(mx, &e);
    return ldexp(1.0, (f == 0.5) ? e - 1 : e);
}

// One thread per row: fill the row's entries of the slice and its copies.
__global__ void k_fill(const int *rp, const int *ci, const double *val, int n, int nslices, const int *sptr,
                       const double *dsc, int row_scale, int precond, int m_prec, int *col, double *a64,
                       double *ah64, float *a32, h16 *a16, b16 *abf, float *rs, void *mvec) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nslices * kSlice; t += gridDim.x * blockDim.x) {
        const int s = t / kSlice, lane = t % kSlice;
        const int i = t;
        const int base = sptr[s] + lane;
        const int w = (sptr[s + 1] - sptr[s]) / kSlice;
        const int b = (i < n) ? rp[i] : 0;
        const int len = (i < n) ? rp[i + 1] - b : 0;
        const double di = (i < n) ? dsc[i] : 1.0;
        double mx = 0.0, diag = 0.0;
        for (int k = 0; k < len; ++k) {
            const int c = ci[b + k];
            const double ah = (val[b + k] * di) * dsc[c];
            mx = fmax(mx, fabs(ah));
            if (c == i) diag = ah;
        }
        const double sc = row_scale ? row_scale_pow2(mx) : 1.0;
        for (int k = 0; k < w; ++k) {
            const int idx = base + k * kSlice;
            if (k < len) {
                const int c = ci[b + k];
                const double a = val[b + k];
                const double ah = (a * di) * dsc[c];
                col[idx] = c;
                if (a64) a64[idx] = a;
                if (ah64) ah64[idx] = ah;
                if (a32) a32[idx] = __double2float_rn(ah);
                if (a16) a16[idx] = __double2half(ah / sc);
                if (abf) abf[idx] = __double2bfloat16(ah / sc);
            } else {
                col[idx] = -1;
                if (a64) a64[idx] = 0.0;
                if (ah64) ah64[idx] = 0.0;
                if (a32) a32[idx] = 0.0f;
                if (a16) a16[idx] = __double2half(0.0);
                if (abf) abf[idx] = __double2bfloat16(0.0);
            }
        }
        if (i < n) {
            if (rs) rs[i] = (float)sc;
            const double m = (precond == F3R_PC_JACOBI && diag != 0.0) ? div_rn(1.0, diag) : 1.0;
            switch (m_prec) {
                case F3R_F64: ((double *)mvec)[i] = m; break;
                case F3R_F32: ((float *)mvec)[i] = __double2float_rn(m); break;
                case F3R_F16: ((h16 *)mvec)[i] = __double2half(m); break;
                default: ((b16 *)mvec)[i] = __double2bfloat16(m); break;
            }
        }
    }
}

// flag = 1 when some stored entry of M differs from 1
template <class S> __global__ void k_m_nonunit(const S *m, int n, int *flag) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (!(to_c<double>(m[i]) == 1.0)) atomicOr(flag, 1);
}

// Factors of the approximate inverse M = (I - Dt^-1 U) Dt^-1 (I - L Dt^-1) of
// A^ = L + D + U, Dt = alpha D: entry (i, c) of L Dt^-1 is A^_ic / dt_c
// (c < i), of Dt^-1 U it is A^_ic / dt_i (c > i), both rounded to fp16 once
// from fp64 (zero elsewhere on the SELL pattern); Dt^-1 in fp16.  A^_ic is
// formed as (a_ic d_i) d_c, the set-up's own rounding of the scaled matrix.
__global__ void k_ainv_fill(const int *rp, const int *ci, const double *val, int n, const int *sptr,
                            const double *dsc, double alpha, h16 *wl, h16 *wu, h16 *dinv) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int s = i / kSlice, lane = i % kSlice;
        const int base = sptr[s] + lane;
        const int w = (sptr[s + 1] - sptr[s]) / kSlice;
        const int b = rp[i], len = rp[i + 1] - b;
        const double di = dsc[i];
        double dii = 0.0;
        for (int k = 0; k < len; ++k)
            if (ci[b + k] == i) dii = (val[b + k] * di) * di;
        const double dti = (dii != 0.0) ? alpha * dii : alpha;
        dinv[i] = __double2half(div_rn(1.0, dti));
        for (int k = 0; k < w; ++k) {
            const int idx = base + k * kSlice;
            double l = 0.0, u = 0.0;
            if (k < len) {
                const int c = ci[b + k];
                const double ah = (val[b + k] * di) * dsc[c];
                if (c < i) {
                    double dcc = 0.0;
                    for (int q = rp[c]; q < rp[c + 1]; ++q)
                        if (ci[q] == c) dcc = (val[q] * dsc[c]) * dsc[c];
                    const double dtc = (dcc != 0.0) ? alpha * dcc : alpha;
                    l = div_rn(ah, dtc);
                } else if (c > i) {
                    u = div_rn(ah, dti);
                }
            }
            wl[idx] = __double2half(l);
            wu[idx] = __double2half(u);
        }
    }
}

template <class S>
__global__ void k_export(const int *rp, int n, const int *sptr, const S *src, S *dst) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int s = i / kSlice, lane = i % kSlice;
        const int b = rp[i], len = rp[i + 1] - b;
        for (int k = 0; k < len; ++k) dst[b + k] = src[sptr[s] + lane + k * kSlice];
    }
}

// windowed tiles: the column each entry's window index stands for, in CSR
// order (the tile's runs concatenated in column order)
__global__ void k_export_win(const int *rp, int n, const int *sptr, const uint16_t *lcol, const int *rec, int *dst) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int s = i / kSlice, lane = i % kSlice;
        const int *r = rec + (size_t)(i / kTileRows) * kWinRec;
        const int b = rp[i], len = rp[i + 1] - b;
        for (int k = 0; k < len; ++k) {
            const int l = lcol[sptr[s] + lane + k * kSlice];
            int c = -1;
            for (int q = 0; q < r[0]; ++q) {
                const int c0 = r[kWinRecRun + 3 * q], ln = r[kWinRecRun + 3 * q + 1], pos = r[kWinRecRun + 3 * q + 2];
                if (l >= pos && l < pos + ln) c = c0 + (l - pos);
            }
            dst[b + k] = c;
        }
    }
}

static void *dalloc(Ctx &c, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void *p = pool_alloc(c.dev, bytes, c.zstream);
    if (!p) return nullptr;
    c.allocs.push_back(p);
    c.bytes += (long long)bytes;
    return p;
}

f3r_status build_matrix(Ctx &c, const int *rp, const int *ci, const double *val, cudaStream_t s) {
    const int n = c.n;
    const int grid = std::min(ceil_div(n, kBlock), c.nsm * 8);
    int *err = (int *)dalloc(c, sizeof(int));
    if (!err) return F3R_ERR_NOMEM;
    cudaMemsetAsync(err, 0, sizeof(int), s);
    k_validate<<<grid, kBlock, 0, s>>>(rp, ci, n, c.nnz, err);
    int herr = 0;
    cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return F3R_ERR_CUDA;
    if (herr) return F3R_ERR_ARG;

    c.dsc = (double *)dalloc(c, sizeof(double) * n);
    if (!c.dsc) return F3R_ERR_NOMEM;
    k_diag_scale<<<grid, kBlock, 0, s>>>(rp, ci, val, n, c.prm.diag_scale, c.dsc);

    c.nslices = ceil_div(n, kSlice);
    int *width = (int *)dalloc(c, sizeof(int) * c.nslices);
    if (!width) return F3R_ERR_NOMEM;
    const int gs = std::max(1, std::min(ceil_div(c.nslices, kWarps), c.nsm * 8));
    k_slice_width<<<gs, kBlock, 0, s>>>(rp, n, c.nslices, width);
    std::vector<int> hw(c.nslices);
    cudaMemcpyAsync(hw.data(), width, sizeof(int) * c.nslices, cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return F3R_ERR_CUDA;
    std::vector<int> hp(c.nslices + 1, 0);
    long long tot = 0;
    for (int k = 0; k < c.nslices; ++k) {
        hp[k] = (int)tot;
        tot += (long long)hw[k] * kSlice;
        if (tot >= (1LL << 31)) return F3R_ERR_ARG;  // padded entry offsets are int32
    }
    hp[c.nslices] = (int)tot;
    c.nsell = tot;
    c.wmax = 0;
    for (int k = 0; k < c.nslices; ++k) c.wmax = std::max(c.wmax, hw[k]);
    c.sptr = (int *)dalloc(c, sizeof(int) * (c.nslices + 1));
    c.col = (int *)dalloc(c, sizeof(int) * tot);
    if (!c.sptr || !c.col) return F3R_ERR_NOMEM;
    cudaMemcpyAsync(c.sptr, hp.data(), sizeof(int) * (c.nslices + 1), cudaMemcpyHostToDevice, s);

    // which copies of A the configured levels read (Table 1)
    bool need[4] = {false, false, false, false};
    for (int d = 1; d < c.prm.nlevels; ++d) need[c.prm.a_prec[d]] = true;
    if (c.prm.rich_m > 0) need[c.prm.rich_a_prec] = true;
    c.a64 = (double *)dalloc(c, sizeof(double) * tot);
    if (need[F3R_F64]) c.ah64 = (double *)dalloc(c, sizeof(double) * tot);
    if (need[F3R_F32]) c.a32 = (float *)dalloc(c, sizeof(float) * tot);
    if (need[F3R_F16]) c.a16 = (h16 *)dalloc(c, sizeof(h16) * tot);
    if (need[F3R_BF16]) c.abf = (b16 *)dalloc(c, sizeof(b16) * tot);
    if (c.prm.row_scale) c.rs = (float *)dalloc(c, sizeof(float) * (size_t)c.nslices * kSlice);
    c.mvec = dalloc(c, (size_t)prec_bytes(c.prm.m_prec) * n);
    if (!c.a64 || !c.mvec || (need[F3R_F64] && !c.ah64) || (need[F3R_F32] && !c.a32) ||
        (need[F3R_F16] && !c.a16) || (need[F3R_BF16] && !c.abf) || (c.prm.row_scale && !c.rs))
        return F3R_ERR_NOMEM;
    if (c.rs) cudaMemsetAsync(c.rs, 0, sizeof(float) * (size_t)c.nslices * kSlice, s);
    const int gf = std::max(1, std::min(ceil_div((long long)c.nslices * kSlice, kBlock), c.nsm * 8));
    k_fill<<<gf, kBlock, 0, s>>>(rp, ci, val, n, c.nslices, c.sptr, c.dsc, c.prm.row_scale, c.prm.precond,
                                 c.prm.m_prec, c.col, c.a64, c.ah64, c.a32, c.a16, c.abf, c.rs, c.mvec);
    if (c.prm.precond == F3R_PC_AINV) {
        c.ainv_l = (h16 *)dalloc(c, sizeof(h16) * tot);
        c.ainv_u = (h16 *)dalloc(c, sizeof(h16) * tot);
        c.ainv_dinv = (h16 *)dalloc(c, sizeof(h16) * (size_t)c.nslices * kSlice);
        c.ainv_t = (float *)dalloc(c, sizeof(float) * (size_t)c.nslices * kSlice);
        c.ainv_m = (float *)dalloc(c, sizeof(float) * (size_t)c.nslices * kSlice);
        if (!c.ainv_l || !c.ainv_u || !c.ainv_dinv || !c.ainv_t || !c.ainv_m) return F3R_ERR_NOMEM;
        cudaMemsetAsync(c.ainv_l, 0, sizeof(h16) * tot, s);
        cudaMemsetAsync(c.ainv_u, 0, sizeof(h16) * tot, s);
        k_ainv_fill<<<grid, kBlock, 0, s>>>(rp, ci, val, n, c.sptr, c.dsc, (double)c.prm.ainv_alpha, c.ainv_l,
                                            c.ainv_u, c.ainv_dinv);
    }
    c.rowptr = (int *)dalloc(c, sizeof(int) * (n + 1));
    int *nonunit = (int *)dalloc(c, sizeof(int));
    if (!c.rowptr || !nonunit) return F3R_ERR_NOMEM;
    cudaMemcpyAsync(c.rowptr, rp, sizeof(int) * (n + 1), cudaMemcpyDeviceToDevice, s);
    // M = I exactly (Jacobi of a matrix whose scaled diagonal is 1, or no M):
    // the Richardson kernels then skip the loads of M; mul(1, v) = v, so the
    // results are the same bits.
    cudaMemsetAsync(nonunit, 0, sizeof(int), s);
    switch (c.prm.m_prec) {
        case F3R_F64: k_m_nonunit<<<gf, kBlock, 0, s>>>((const double *)c.mvec, n, nonunit); break;
        case F3R_F32: k_m_nonunit<<<gf, kBlock, 0, s>>>((const float *)c.mvec, n, nonunit); break;
        case F3R_F16: k_m_nonunit<<<gf, kBlock, 0, s>>>((const h16 *)c.mvec, n, nonunit); break;
        default: k_m_nonunit<<<gf, kBlock, 0, s>>>((const b16 *)c.mvec, n, nonunit); break;
    }
    int nonunit_h = 1;
    cudaMemcpyAsync(&nonunit_h, nonunit, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return F3R_ERR_CUDA;
    const char *e = getenv("F3R_UNIT_M");  // 0: keep loading M (for the bit-identity test)
    c.m_unit = (nonunit_h == 0) && !(e && e[0] == '0');
    return build_window(c, s);
}

f3r_status export_array(Ctx &c, int which, void *out, cudaStream_t s) {
    const int n = c.n;
    const int grid = std::max(1, std::min(ceil_div(n, kBlock), c.nsm * 8));
    void *tmp = nullptr;
    size_t bytes = 0;
    f3r_status st = F3R_OK;
    auto run = [&](auto *src, size_t elem) {
        typedef typename std::remove_cv<typename std::remove_pointer<decltype(src)>::type>::type S;
        bytes = elem * (size_t)c.nnz;
        if (cudaMalloc(&tmp, bytes) != cudaSuccess) {
            st = F3R_ERR_NOMEM;
            return;
        }
        k_export<S><<<grid, kBlock, 0, s>>>(c.rowptr, n, c.sptr, src, (S *)tmp);
    };
    switch (which) {
        case 0:
            cudaMemcpyAsync(out, c.dsc, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
            return cudaStreamSynchronize(s) == cudaSuccess ? F3R_OK : F3R_ERR_CUDA;
        case 1:
            if (!c.ah64) return F3R_ERR_ARG;
            run(c.ah64, sizeof(double));
            break;
        case 2:
            if (!c.a32) return F3R_ERR_ARG;
            run(c.a32, sizeof(float));
            break;
        case 3:
            if (!c.a16) return F3R_ERR_ARG;
            run(c.a16, sizeof(h16));
            break;
        case 4:
            if (!c.abf) return F3R_ERR_ARG;
            run(c.abf, sizeof(b16));
            break;
        case 5:
            if (!c.rs) return F3R_ERR_ARG;
            cudaMemcpyAsync(out, c.rs, sizeof(float) * n, cudaMemcpyDeviceToHost, s);
            return cudaStreamSynchronize(s) == cudaSuccess ? F3R_OK : F3R_ERR_CUDA;
        case 6:
            cudaMemcpyAsync(out, c.mvec, (size_t)prec_bytes(c.prm.m_prec) * n, cudaMemcpyDeviceToHost, s);
            return cudaStreamSynchronize(s) == cudaSuccess ? F3R_OK : F3R_ERR_CUDA;
        case 7:
            if (!c.ainv_l) return F3R_ERR_ARG;
            run(c.ainv_l, sizeof(h16));
            break;
        case 8:
            if (!c.ainv_u) return F3R_ERR_ARG;
            run(c.ainv_u, sizeof(h16));
            break;
        case 9:
            if (!c.ainv_dinv) return F3R_ERR_ARG;
            cudaMemcpyAsync(out, c.ainv_dinv, sizeof(h16) * n, cudaMemcpyDeviceToHost, s);
            return cudaStreamSynchronize(s) == cudaSuccess ? F3R_OK : F3R_ERR_CUDA;
        case 10:
            if (!c.win) return F3R_ERR_ARG;
            bytes = sizeof(int) * (size_t)c.nnz;
            if (cudaMalloc(&tmp, bytes ? bytes : 16) != cudaSuccess) return F3R_ERR_NOMEM;
            k_export_win<<<grid, kBlock, 0, s>>>(c.rowptr, n, c.sptr, c.lcol, c.wrec, (int *)tmp);
            break;
        default:
            return F3R_ERR_ARG;
    }
    if (st != F3R_OK) return st;
    cudaMemcpyAsync(out, tmp, bytes, cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(tmp);
    return e == cudaSuccess ? F3R_OK : F3R_ERR_CUDA;
}

StagePlan plan_stage(const Ctx &c, int asize, int n_extra, int esize, int xsize) {
    StagePlan p;
    if (!c.staged) return p;
    const bool win = c.win && xsize > 0;
    const int sb = stage_bytes_for(c.wmax, asize, n_extra, esize, win ? c.win_max : 0, win ? xsize : 0);
    // 3 stages if four blocks fit an SM, else 2 stages with two blocks, else
    // 2 stages with one block; wider tiles run unstaged.  Windowed kernels
    // (smaller stages) may take 4 stages.
    static const int force_s = [] {
        const char *e = getenv("F3R_STAGES");  // 2 or 3: ring depth override for tuning runs
        return e ? atoi(e) : 0;
    }();
    static const int win_s = [] {
        const char *e = getenv("F3R_WSTAGES");  // 2, 3 or 4: ring depth of windowed kernels (tuning)
        const int v = e ? atoi(e) : 0;
        return (v >= 2 && v <= 4) ? v : kWinStages;
    }();
    const int cand[4][2] = {{4, 56 * 1024}, {3, 56 * 1024}, {2, 110 * 1024}, {2, 220 * 1024}};
    for (auto &cs : cand) {
        if (cs[0] == 4 && !(win && win_s == 4)) continue;
        if (cs[0] == 3 && (force_s == 2 || (win && win_s == 2))) continue;
        const int smem = 256 + cs[0] * sb;
        if (smem <= cs[1]) {
            p.S = cs[0];
            p.stage_bytes = sb;
            p.smem = smem;
            return p;
        }
    }
    return p;
}

bool pdl_enabled() {
    static const bool on = [] {
        const char *e = getenv("F3R_PDL");  // 0: plain stream order for every launch
        return !(e && e[0] == '0');
    }();
    return on;
}

int maxd_bucket(int m) { return m <= 4 ? 4 : (m <= 8 ? 8 : 16); }

int prec_bytes(int p) {
    switch (p) {
        case F3R_F64: return 8;
        case F3R_F32: return 4;
        default: return 2;
    }
}

}  // namespace f3r
