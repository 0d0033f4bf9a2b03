// Richardson with adaptive weights (Algorithm 1, Eqs. 4-5):
//   z_0 = 0, z_k = z_{k-1} + w_k M (v - A z_{k-1}),  k = 1..m4
// with w'_k = (r, AMr)/(AMr, AMr) used on every c-th call and folded into
// w_k := (l w_k + w'_k)/(l + 1), l = c_ntr / c.
//
// Storage VS (fp16 / bf16 / fp32 / fp64) for v, z, r and M; arithmetic TC
// (fp32, fp64 for fp64 storage).  Rounding points: r = VS(v - A z) with the
// row sum in TC, u = m * r in TC, z_k = VS(fma(w, u, z_{k-1})).
//
// k_rich2 runs a whole plain call with m4 = 2 in one pass over A: z_1 at a
// neighbour c is recomputed from v_c and m_c on the fly with the same
// rounding, so the result equals the two-step recurrence bit for bit.
#pragma once
#include "kernels.cuh"

namespace f3r {

template <class TC> struct RichDev {
    TC *omega;                    // w_1..w_m4
    TC *wcur;                     // w'_k of the running update step
    unsigned long long *counters; // [0] M applications, [1] calls, [2] update calls
    const long long *c_ntr_base;  // c_ntr of the first call of the current outer iteration
};

template <class TA, class VS, class TC, class TP>
__global__ void __launch_bounds__(kBlock) k_rich2(Sell S, const TA *__restrict__ val, const float *__restrict__ rs,
                                                  const VS *__restrict__ v, const VS *__restrict__ mv, TP *out,
                                                  const TP *par_misc, RichDev<TC> R, const int *flags, int check_depth,
                                                  int n) {
    pdl_enter();
    if (stopped(flags, check_depth)) return;
    const TC w1 = R.omega[0], w2 = R.omega[1];
    const TP inv_sigma = par_misc[MS_INV_SIGMA];
    const int lane = threadIdx.x & 31;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int s = wid; s < S.nslices; s += nw) {
        TC acc = sell_row<TC>(S, val, s, lane, [&](int c) {
            return rnd<VS>(fma_rn(w1, mul_rn(to_c<TC>(__ldg(mv + c)), to_c<TC>(__ldg(v + c))), (TC)0));
        });
        const int i = s * kSlice + lane;
        if (rs) acc = mul_rn(acc, (TC)__ldg(rs + i));
        if (i < n) {
            const TC vi = to_c<TC>(v[i]), mi = to_c<TC>(mv[i]);
            const TC z1 = rnd<VS>(fma_rn(w1, mul_rn(mi, vi), (TC)0));
            const TC ri = rnd<VS>(sub_rn(vi, acc));
            const TC z2 = rnd<VS>(fma_rn(w2, mul_rn(mi, ri), z1));
            out[i] = mul_rn((TP)z2, inv_sigma);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        atomicAdd(R.counters + 0, 2ull);
        atomicAdd(R.counters + 1, 1ull);
    }
}

// Plain step k of the generic recurrence (m4 != 2, or the non-fused path):
//   k == 0 : z = VS(fma(w_1, m v, 0))
//   k >= 1 : z = VS(fma(w_k, m VS(v - A z_prev), z_prev))
// The last step writes the parent's output z / sigma, earlier steps z (VS).
template <class TA, class VS, class TC, class TP>
__global__ void __launch_bounds__(kBlock) k_rich_step(Sell S, const TA *__restrict__ val, const float *__restrict__ rs,
                                                      const VS *__restrict__ v, const VS *__restrict__ mv,
                                                      const VS *__restrict__ zprev, VS *znext, TP *out,
                                                      const TP *par_misc, RichDev<TC> R, int k, int last,
                                                      const int *flags, int check_depth, int n) {
    pdl_enter();
    if (stopped(flags, check_depth)) return;
    const TC wk = R.omega[k];
    const TP inv_sigma = par_misc[MS_INV_SIGMA];
    const int lane = threadIdx.x & 31;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int s = wid; s < S.nslices; s += nw) {
        TC acc = (TC)0;
        if (k > 0) acc = sell_row<TC>(S, val, s, lane, [&](int c) { return to_c<TC>(__ldg(zprev + c)); });
        const int i = s * kSlice + lane;
        if (k > 0 && rs) acc = mul_rn(acc, (TC)__ldg(rs + i));
        if (i < n) {
            const TC vi = to_c<TC>(v[i]), mi = to_c<TC>(mv[i]);
            TC z;
            if (k == 0) {
                z = rnd<VS>(fma_rn(wk, mul_rn(mi, vi), (TC)0));
            } else {
                const TC ri = rnd<VS>(sub_rn(vi, acc));
                z = rnd<VS>(fma_rn(wk, mul_rn(mi, ri), to_c<TC>(zprev[i])));
            }
            if (last) out[i] = mul_rn((TP)z, inv_sigma);
            else znext[i] = Store<VS>::from(z);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        atomicAdd(R.counters + 0, 1ull);
        if (last) atomicAdd(R.counters + 1, 1ull);
    }
}

// Update call, step k >= 1: r = VS(v - A z) (stored)
template <class TA, class VS, class TC>
__global__ void __launch_bounds__(kBlock) k_rich_upd_r(Sell S, const TA *__restrict__ val, const float *__restrict__ rs,
                                                       const VS *__restrict__ v, const VS *__restrict__ z, VS *r,
                                                       const int *flags, int check_depth, int n) {
    pdl_enter();
    if (stopped(flags, check_depth)) return;
    const int lane = threadIdx.x & 31;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int s = wid; s < S.nslices; s += nw) {
        TC acc = sell_row<TC>(S, val, s, lane, [&](int c) { return to_c<TC>(__ldg(z + c)); });
        const int i = s * kSlice + lane;
        if (rs) acc = mul_rn(acc, (TC)__ldg(rs + i));
        if (i < n) r[i] = Store<VS>::from(sub_rn(to_c<TC>(v[i]), acc));
    }
}

// Update call, step k: w = A (M r) in TC, (r, w) and (w, w);
// w'_k = (r, w)/(w, w) (kept w_k if (w, w) = 0), w_k := (l w_k + w'_k)/(l + 1).
template <class TA, class VS, class TC>
__global__ void __launch_bounds__(kBlock) k_rich_upd_w(Sell S, const TA *__restrict__ val, const float *__restrict__ rs,
                                                       const VS *__restrict__ r, const VS *__restrict__ mv,
                                                       RichDev<TC> R, int k, int pos, int c, GridRed<TC> gr,
                                                       const int *flags, int check_depth, int n) {
    pdl_enter();
    if (stopped(flags, check_depth)) return;
    TC acc[2] = {(TC)0, (TC)0};
    const int lane = threadIdx.x & 31;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int s = wid; s < S.nslices; s += nw) {
        TC w = sell_row<TC>(S, val, s, lane, [&](int cc) {
            return mul_rn(to_c<TC>(__ldg(mv + cc)), to_c<TC>(__ldg(r + cc)));
        });
        const int i = s * kSlice + lane;
        if (rs) w = mul_rn(w, (TC)__ldg(rs + i));
        if (i < n) {
            acc[0] = fma_rn(to_c<TC>(r[i]), w, acc[0]);
            acc[1] = fma_rn(w, w, acc[1]);
        }
    }
    grid_reduce<TC, 2>(acc, 2, false, gr, [&](TC *res) {
        const TC num = res[0], den = res[1];
        const TC wk = R.omega[k];
        const TC q = div_rn(num, den);
        const bool ok = den > (TC)0 && isfinite(q);
        *R.wcur = ok ? q : wk;
        if (ok) {
            const long long cn = *R.c_ntr_base + pos;
            const TC l = (TC)(cn / c);
            R.omega[k] = div_rn(add_rn(mul_rn(l, wk), q), add_rn(l, (TC)1));
        }
    });
}

// Update call, step k: z = VS(fma(w'_k, m r, z_prev)) (z_prev = 0 at k = 0)
template <class VS, class TC, class TP>
__global__ void __launch_bounds__(kBlock) k_rich_upd_z(const VS *__restrict__ r, const VS *__restrict__ mv,
                                                       const VS *__restrict__ zprev, VS *znext, TP *out,
                                                       const TP *par_misc, RichDev<TC> R, int last,
                                                       const int *flags, int check_depth, int n) {
    pdl_enter();
    if (stopped(flags, check_depth)) return;
    const TC wp = *R.wcur;
    const TP inv_sigma = par_misc[MS_INV_SIGMA];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const TC zp = zprev ? to_c<TC>(zprev[i]) : (TC)0;
        const TC z = rnd<VS>(fma_rn(wp, mul_rn(to_c<TC>(mv[i]), to_c<TC>(r[i])), zp));
        if (last) out[i] = mul_rn((TP)z, inv_sigma);
        else znext[i] = Store<VS>::from(z);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        atomicAdd(R.counters + 0, 1ull);
        if (last) {
            atomicAdd(R.counters + 1, 1ull);
            atomicAdd(R.counters + 2, 1ull);
        }
    }
}

// Richardson input for a stand-alone call: sigma from max|v| (reduction), then
// the 16-bit cast; used by the instrumentation entry f3r_apply.
template <class TP>
__global__ void __launch_bounds__(kBlock) k_amax_sigma(const TP *v, int n, TP *misc, int want_sigma,
                                                       GridRed<TP> gr) {
    pdl_enter();
    TP acc[1] = {(TP)0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        acc[0] = fmax(acc[0], fabs(v[i]));
    grid_reduce<TP, 1>(acc, 0, true, gr, [&](TP *res) {
        const TP sg = want_sigma ? pow2_scale_for(res[0]) : (TP)1;
        misc[MS_SIGMA] = sg;
        misc[MS_INV_SIGMA] = div_rn((TP)1, sg);
    });
}

template <class TP, class VS>
__global__ void __launch_bounds__(kBlock) k_cast_scaled(const TP *v, VS *out, int n, const TP *misc) {
    pdl_enter();
    const TP sg = misc[MS_SIGMA];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = Store<VS>::from(mul_rn(sg, v[i]));
}

}  // namespace f3r
