// Richardson steps (Algorithm 1, Eqs. 4-5) for a primary preconditioner that
// is not diagonal: its output u = M r is computed first (the learned net, the
// approximate inverse) into an fp32 vector, then these kernels finish the
// step in the fp16 storage of the Richardson level.
#pragma once
#include "kernels.cuh"

namespace f3r {

// Richardson step with the preconditioner's output u = M r given (fp32):
// z = fp16(fma(w, u, z_prev)); the last step writes the parent's output
// z / sigma.  With use_wcur, w is the locally optimal weight of the update
// step (k_rich_upd_w_u), else omega[k].
static __global__ void __launch_bounds__(kBlock) k_rich_z_u(const float *u, const h16 *zprev, h16 *znext, float *out,
                                                      const float *par_misc, const float *omega, const float *wcur,
                                                      int k, int last, int use_wcur, const int *flags,
                                                      int check_depth, int n, unsigned long long *counters) {
    pdl_enter();
    if (stopped(flags, check_depth)) return;
    const float w = use_wcur ? *wcur : omega[k];
    const float inv_sigma = par_misc[MS_INV_SIGMA];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float zp = zprev ? __half2float(zprev[i]) : 0.0f;
        const float z = rnd<h16>(fma_rn(w, u[i], zp));
        if (last) out[i] = mul_rn(z, inv_sigma);
        else znext[i] = __float2half_rn(z);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        atomicAdd(counters + 0, 1ull);
        if (last) {
            atomicAdd(counters + 1, 1ull);
            if (use_wcur) atomicAdd(counters + 2, 1ull);
        }
    }
}

// update step (Algorithm 1) with u = M r given: w = A^ u, w' = (r, w)/(w, w),
// and the weight average w_k := (l w_k + w')/(l + 1), l = c_ntr / c
static __global__ void __launch_bounds__(kBlock) k_rich_upd_w_u(Sell S, const h16 *__restrict__ a16, const float *__restrict__ rs,
                                                     const h16 *__restrict__ r, const float *__restrict__ u, float *omega,
                                                     float *wcur, const long long *c_ntr_base, int k, int pos, int c,
                                                     GridRed<float> gr, const int *flags, int check_depth, int n) {
    pdl_enter();
    if (stopped(flags, check_depth)) return;
    float acc[2] = {0.0f, 0.0f};
    const int lane = threadIdx.x & 31;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int s = wid; s < S.nslices; s += nw) {
        float w = sell_row<float>(S, a16, s, lane, [&](int cc) { return u[cc]; });
        const int i = s * kSlice + lane;
        if (rs) w = mul_rn(w, rs[i]);
        if (i < n) {
            acc[0] = fma_rn(__half2float(r[i]), w, acc[0]);
            acc[1] = fma_rn(w, w, acc[1]);
        }
    }
    grid_reduce<float, 2>(acc, 2, false, gr, [&](float *res) {
        const float wk = omega[k];
        const float q = div_rn(res[0], res[1]);
        const bool ok = res[1] > 0.0f && isfinite(q);
        *wcur = ok ? q : wk;
        if (ok) {
            const float l = (float)((*c_ntr_base + pos) / c);
            omega[k] = div_rn(add_rn(mul_rn(l, wk), q), add_rn(l, 1.0f));
        }
    });
}

}  // namespace f3r
