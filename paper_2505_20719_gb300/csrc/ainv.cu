// Approximate inverse as the primary preconditioner M of the Richardson level
// (the paper's GPU runs use SD-AINV, a simplified approximate inverse that
// costs two SpMVs per application, Sec. 5.2; its construction is in a cited
// work).  The approximate inverse here truncates the inverse of the
// triangular factors of A^ ~ (Dt + L) Dt^-1 (Dt + U) after the first term:
//     M = (I - Dt^-1 U) Dt^-1 (I - L Dt^-1),   Dt = alpha diag(A^),
// with L Dt^-1, Dt^-1 U and Dt^-1 stored in fp16 on the SELL pattern of A^.
// One application u = M r (r fp16, arithmetic fp32, CSR-order fused
// multiply-adds):
//     t = Dt^-1 (r - (L Dt^-1) r)          k_ainv_lower
//     u = t - (Dt^-1 U) t                   k_ainv_upper
// The Richardson step then finishes with the shared k_rich_z_u /
// k_rich_upd_w_u (rich_u.cuh).
#include "ctx.h"
#include "rich.cuh"
#include "rich_u.cuh"

namespace f3r {

namespace {

__global__ void __launch_bounds__(kBlock) k_ainv_lower(Sell S, const h16 *__restrict__ wl, const h16 *__restrict__ dinv,
                                                       const h16 *__restrict__ r, float *t, const int *flags,
                                                       int check_depth, int n) {
    pdl_enter();
    if (stopped(flags, check_depth)) return;
    const int lane = threadIdx.x & 31;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int s = wid; s < S.nslices; s += nw) {
        const float lr = sell_row<float>(S, wl, s, lane, [&](int c) { return __half2float(__ldg(r + c)); });
        const int i = s * kSlice + lane;
        if (i < n) t[i] = mul_rn(__half2float(dinv[i]), sub_rn(__half2float(r[i]), lr));
    }
}

__global__ void __launch_bounds__(kBlock) k_ainv_upper(Sell S, const h16 *__restrict__ wu, const float *__restrict__ t,
                                                       float *u, const int *flags, int check_depth, int n) {
    pdl_enter();
    if (stopped(flags, check_depth)) return;
    const int lane = threadIdx.x & 31;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int s = wid; s < S.nslices; s += nw) {
        const float ut = sell_row<float>(S, wu, s, lane, [&](int c) { return __ldg(t + c); });
        const int i = s * kSlice + lane;
        if (i < n) u[i] = sub_rn(t[i], ut);
    }
}

}  // namespace

// One Richardson call (Algorithm 1) with the approximate inverse as M, fp16
// storage: r_0 = v, r_k = fp16(v - A^ z_{k-1}); u = M r_k; plain steps
// z_k = fp16(fma(w_k, u, z_{k-1})), update steps with w'_k from w = A^ u.
void ainv_rich_call(Ctx &c, bool update, int pos, void *out, const void *par_misc, cudaStream_t s) {
    const Sell S = sell_of(c);
    const int cd = c.prm.nlevels - 1, n = c.n, m4 = c.prm.rich_m;
    h16 *zb[2] = {(h16 *)c.rz[0], (h16 *)c.rz[1]};
    for (int k = 0; k < m4; ++k) {
        const bool last = (k == m4 - 1);
        const h16 *zp = (k > 0) ? zb[(k - 1) & 1] : nullptr;
        const h16 *rk = (const h16 *)c.rin;
        if (k > 0) {
            launch_pdl(k_rich_upd_r<h16, h16, float>, dim3(c.Gs), dim3(kBlock), 0, s, S, (const h16 *)c.a16,
                       (const float *)nullptr, (const h16 *)c.rin, zp, (h16 *)c.rr, (const int *)c.flags, cd, n);
            rk = (const h16 *)c.rr;
            c.launches++;
        }
        launch_pdl(k_ainv_lower, dim3(c.Gs), dim3(kBlock), 0, s, S, (const h16 *)c.ainv_l,
                   (const h16 *)c.ainv_dinv, rk, c.ainv_t, (const int *)c.flags, cd, n);
        launch_pdl(k_ainv_upper, dim3(c.Gs), dim3(kBlock), 0, s, S, (const h16 *)c.ainv_u, (const float *)c.ainv_t,
                   c.ainv_m, (const int *)c.flags, cd, n);
        c.launches += 2;
        if (update) {
            launch_pdl(k_rich_upd_w_u, dim3(c.Gs), dim3(kBlock), 0, s, S, (const h16 *)c.a16, (const float *)nullptr, rk,
                       (const float *)c.ainv_m, (float *)c.omega, (float *)c.wcur, (const long long *)c.c_ntr_base, k,
                       pos, c.prm.c, GridRed<float>{(float *)c.partials, c.ticket, kMaxDots}, (const int *)c.flags, cd,
                       n);
            c.launches++;
        }
        launch_pdl(k_rich_z_u, dim3(c.G), dim3(kBlock), 0, s, (const float *)c.ainv_m, zp, zb[k & 1], (float *)out,
                   (const float *)par_misc, (const float *)c.omega, (const float *)c.wcur, k, last ? 1 : 0,
                   update ? 1 : 0, (const int *)c.flags, cd, n, c.counters);
        c.launches++;
    }
}

}  // namespace f3r
