// Learned preconditioner M_theta: inference, training (forward, backward,
// Adam) and its use as M inside the Richardson level.  See learned.cuh for
// the network.  Aggregation runs over the sliced-ELLPACK copy of A^ in fp16
// (the off-diagonal entries), so the net sees exactly the matrix of the
// fp16 level; training needs A^ symmetric (the backward aggregation uses row
// j of A^ for column j).
#include <algorithm>
#include <cmath>
#include <vector>

#include "ctx.h"
#include "learned.cuh"
#include "rich.cuh"
#include "rich_u.cuh"

namespace f3r {
namespace lm {

constexpr int LDT = 2 * W + kPadH;   // row pitch of [h | g] tiles
constexpr int LDW = 2 * W + kPadH;   // row pitch of wcat in shared memory
constexpr int LDWT = W + kPadH;      // row pitch of wcat^T
constexpr int LDK = 16 + kPadH;      // row pitch of transposed 16-node tiles

// ------------------------------------------------------------ parameters
__global__ void k_lm_prepare(const float *theta, b16 *wcat, b16 *wcatT, b16 *e_bf, b16 *wo_bf) {
    for (int idx = threadIdx.x; idx < NL * W * 2 * W; idx += blockDim.x) {
        const int l = idx / (W * 2 * W), rem = idx % (W * 2 * W), a = rem / (2 * W), k = rem % (2 * W);
        const float v = (k < W) ? theta[OFF_WS + l * W * W + a * W + k] : theta[OFF_WM + l * W * W + a * W + (k - W)];
        const b16 q = __float2bfloat16_rn(v);
        wcat[idx] = q;
        wcatT[l * 2 * W * W + k * W + a] = q;
    }
    for (int c = threadIdx.x; c < W; c += blockDim.x) {
        e_bf[c] = __float2bfloat16_rn(theta[OFF_E + c]);
        wo_bf[c] = __float2bfloat16_rn(theta[OFF_WO + c]);
    }
}

// s = 2^ceil(log2 max|r|) and 1/s (1 when r = 0)
__global__ void __launch_bounds__(kBlock) k_lm_scale(const float *r, int n, float *misc, GridRed<float> gr) {
    pdl_enter();
    float acc[1] = {0.0f};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        acc[0] = fmax(acc[0], fabs(r[i]));
    grid_reduce<float, 1>(acc, 0, true, gr, [&](float *res) {
        const float mx = res[0];
        float s = 1.0f;
        if (mx > 0.0f && isfinite(mx)) {
            int e;
            const float f = frexpf(mx, &e);  // mx = f 2^e, f in [0.5, 1)
            s = ldexpf(1.0f, (f == 0.5f) ? e - 1 : e);
        }
        misc[0] = s;
        misc[1] = div_rn(1.0f, s);
    });
}

__global__ void __launch_bounds__(kBlock) k_lm_embed(const float *r, int n, const float *misc, NetDev net, b16 *H0) {
    pdl_enter();
    const float inv_s = misc[1];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * (W / 8); t += gridDim.x * blockDim.x) {
        const int i = t / (W / 8), ch = t % (W / 8);
        const float rt = mul_rn(r[i], inv_s);
        Pack<b16, 8> out;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int c = ch * 8 + e;
            const float p = fma_rn(__bfloat162float(net.e_bf[c]), rt, net.theta[OFF_B0 + c]);
            out.v[e] = __float2bfloat16_rn(fmax(p, 0.0f));
        }
        stp<b16, 8>(H0 + (size_t)i * W + ch * 8, out);
    }
}

// g_i = sum_{j != i} A^_ij X_j over the 16 features [16 hf, 16 hf + 16) of
// node i (fp32, CSR order), bf16 rows X of width W
__device__ __forceinline__ void aggregate16(const Sell &A, const h16 *__restrict__ a16, const float *__restrict__ rs,
                                            const b16 *__restrict__ X, int i, int hf, float (&acc)[16]) {
#pragma unroll
    for (int e = 0; e < 16; ++e) acc[e] = 0.0f;
    const int s = i >> 5, li = i & 31;
    const int beg = __ldg(A.sptr + s) + li;
    const int w = (__ldg(A.sptr + s + 1) - __ldg(A.sptr + s)) >> 5;
    // neighbours in groups of kAggGroup: their rows are loaded before the
    // multiply-adds (each feature still sums in CSR order)
    constexpr int kAggGroup = 4;
    for (int k0 = 0; k0 < w; k0 += kAggGroup) {
        int c[kAggGroup];
        float a[kAggGroup];
        Pack<b16, 8> x0[kAggGroup], x1[kAggGroup];
#pragma unroll
        for (int q = 0; q < kAggGroup; ++q) {
            const int idx = beg + ((k0 + q) << 5);
            const int cc = (k0 + q < w) ? __ldg(A.col + idx) : -1;
            c[q] = (cc >= 0 && cc != i) ? cc : -1;
            a[q] = (c[q] >= 0) ? __half2float(a16[idx]) : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < kAggGroup; ++q)
            if (c[q] >= 0) {
                x0[q] = ldp<b16, 8>(X + (size_t)c[q] * W + hf * 16);
                x1[q] = ldp<b16, 8>(X + (size_t)c[q] * W + hf * 16 + 8);
            }
#pragma unroll
        for (int q = 0; q < kAggGroup; ++q)
            if (c[q] >= 0) {
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    acc[e] = fma_rn(a[q], __bfloat162float(x0[q].v[e]), acc[e]);
                    acc[8 + e] = fma_rn(a[q], __bfloat162float(x1[q].v[e]), acc[8 + e]);
                }
            }
    }
    if (rs) {
        const float sc = rs[i];
#pragma unroll
        for (int e = 0; e < 16; ++e) acc[e] = mul_rn(acc[e], sc);
    }
}

// One message-passing layer for groups of 16 nodes per warp.
// MODE 0: store h (and g when G is given); MODE 1: read-out z only (last
// layer, inference); MODE 2: store h and g and read out z (last layer, training).
template <int MODE>
__global__ void __launch_bounds__(kLB) k_lm_layer(Sell A, const h16 *__restrict__ a16, const float *__restrict__ rs,
                                                  int n, const b16 *__restrict__ Hin, int l, NetDev net, b16 *Hout,
                                                  b16 *Gout, float *zout, const float *__restrict__ r,
                                                  const float *misc) {
    pdl_enter();
    __shared__ __align__(16) b16 Wt[W * LDW];
    __shared__ float bs[W];
    __shared__ __align__(16) b16 T[kLB / 32][16 * LDT];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int idx = threadIdx.x; idx < W * 2 * W; idx += blockDim.x)
        Wt[(idx / (2 * W)) * LDW + idx % (2 * W)] = net.wcat[(size_t)l * W * 2 * W + idx];
    for (int c = threadIdx.x; c < W; c += blockDim.x) bs[c] = net.theta[OFF_B + l * W + c];
    __syncthreads();
    b16 *Tw = T[warp];
    const int g = lane >> 2, t = lane & 3;
    const int ngroups = (n + 15) >> 4;
    for (int gi = blockIdx.x * (kLB / 32) + warp; gi < ngroups; gi += gridDim.x * (kLB / 32)) {
        const int i0 = gi * 16;
        // own rows h_i -> columns [0, W) of the tile
        for (int q = lane; q < 16 * (W / 8); q += 32) {
            const int rr = q / (W / 8), ch = q % (W / 8), i = i0 + rr;
            Pack<b16, 8> v;
            if (i < n) v = ldp<b16, 8>(Hin + (size_t)i * W + ch * 8);
            else
#pragma unroll
                for (int e = 0; e < 8; ++e) v.v[e] = __float2bfloat16_rn(0.0f);
            stp<b16, 8>(Tw + rr * LDT + ch * 8, v);
        }
        // messages g_i -> columns [W, 2W)
        {
            const int rr = lane >> 1, hf = lane & 1, i = i0 + rr;
            float acc[16];
            if (i < n) aggregate16(A, a16, rs, Hin, i, hf, acc);
            else
#pragma unroll
                for (int e = 0; e < 16; ++e) acc[e] = 0.0f;
            Pack<b16, 8> p0, p1;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                p0.v[e] = __float2bfloat16_rn(acc[e]);
                p1.v[e] = __float2bfloat16_rn(acc[8 + e]);
            }
            stp<b16, 8>(Tw + rr * LDT + W + hf * 16, p0);
            stp<b16, 8>(Tw + rr * LDT + W + hf * 16 + 8, p1);
            if (MODE != 1 && Gout && i < n) {
                stp<b16, 8>(Gout + (size_t)i * W + hf * 16, p0);
                stp<b16, 8>(Gout + (size_t)i * W + hf * 16 + 8, p1);
            }
        }
        __syncwarp();
        // p = [h | g] [Ws | Wm]^T  (16 x 64 by 64 x 32, fp32 accumulation)
        float d[4][4];
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) d[nt][e] = 0.0f;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
            uint32_t a[4];
            frag_a(a, Tw, LDT, ks, lane);
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                uint32_t b0, b1;
                frag_b(b0, b1, Wt, LDW, nt, ks, lane);
                mma_bf16(d[nt], a, b0, b1);
            }
        }
        __syncwarp();
        // h = bf16(relu(p + b)); read-out y = omega_j r~ + wo . h
        float part[2] = {0.0f, 0.0f};
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int hr = 0; hr < 2; ++hr)
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int col = 8 * nt + 2 * t + e;
                    const b16 hv = __float2bfloat16_rn(fmax(add_rn(d[nt][hr * 2 + e], bs[col]), 0.0f));
                    if (MODE != 1) Tw[(g + 8 * hr) * LDT + col] = hv;
                    if (MODE != 0)
                        part[hr] = fma_rn(__bfloat162float(net.wo_bf[col]), __bfloat162float(hv), part[hr]);
                }
        if (MODE != 0) {
#pragma unroll
            for (int hr = 0; hr < 2; ++hr) {
                part[hr] = add_rn(part[hr], __shfl_xor_sync(0xffffffffu, part[hr], 1));
                part[hr] = add_rn(part[hr], __shfl_xor_sync(0xffffffffu, part[hr], 2));
            }
            if (t == 0) {
                const float s = misc[0], inv_s = misc[1], oj = net.theta[OFF_OJ];
#pragma unroll
                for (int hr = 0; hr < 2; ++hr) {
                    const int i = i0 + g + 8 * hr;
                    if (i < n) zout[i] = mul_rn(s, fma_rn(oj, mul_rn(r[i], inv_s), part[hr]));
                }
            }
        }
        __syncwarp();
        if (MODE != 1)
            for (int q = lane; q < 16 * (W / 8); q += 32) {
                const int rr = q / (W / 8), ch = q % (W / 8), i = i0 + rr;
                if (i < n) stp<b16, 8>(Hout + (size_t)i * W + ch * 8, ldp<b16, 8>(Tw + rr * LDT + ch * 8));
            }
        __syncwarp();
    }
}

// ------------------------------------------------------------- backward
// Block-level sum of per-thread vectors v[K] into out[K] (fixed order).
template <int K>
__device__ __forceinline__ void block_vec_sum(float (&v)[K], float *smem /* kLB/32 * K */, float *out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float s = warp_sum(v[k]);
        if (lane == 0) smem[warp * K + k] = s;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        float s = smem[k];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) s = add_rn(s, smem[w * K + k]);
        out[k] = s;
    }
    __syncthreads();
}

// dy = s coef (z - e); dP_L = bf16((wo dy) * [h_L > 0]); per-block partials
// of [dwo (W) | domega_j | loss] in part[block][W + 2].
// With gdir (residual loss) dy = s coef gdir and the loss term is lossv^2.
__global__ void __launch_bounds__(kLB) k_lm_out_bwd(const float *z, const float *e, const float *r, int n,
                                                    const float *misc, const float *coef, NetDev net,
                                                    const b16 *HL, b16 *dP, float *part, const float *gdir,
                                                    const float *lossv) {
    pdl_enter();
    __shared__ float sm[(kLB / 32) * (W + 2)];
    const float s = misc[0], inv_s = misc[1], cf = *coef;
    float acc[W + 2];
#pragma unroll
    for (int k = 0; k < W + 2; ++k) acc[k] = 0.0f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float dif = gdir ? gdir[i] : sub_rn(z[i], e[i]);
        const float lt = gdir ? lossv[i] : dif;
        const float dy = mul_rn(mul_rn(s, cf), dif);
        const float rt = mul_rn(r[i], inv_s);
        acc[W] = fma_rn(rt, dy, acc[W]);
        acc[W + 1] = fma_rn(mul_rn(0.5f, cf), mul_rn(lt, lt), acc[W + 1]);
#pragma unroll
        for (int ch = 0; ch < W / 8; ++ch) {
            const Pack<b16, 8> h = ldp<b16, 8>(HL + (size_t)i * W + ch * 8);
            Pack<b16, 8> o;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int c = ch * 8 + q;
                const float hv = __bfloat162float(h.v[q]);
                acc[c] = fma_rn(hv, dy, acc[c]);
                const float dh = mul_rn(__bfloat162float(net.wo_bf[c]), dy);
                o.v[q] = __float2bfloat16_rn(hv > 0.0f ? dh : 0.0f);
            }
            stp<b16, 8>(dP + (size_t)i * W + ch * 8, o);
        }
    }
    block_vec_sum<W + 2>(acc, sm, part + (size_t)blockIdx.x * (W + 2));
}

// Weight gradient of one layer: dW = dP^T [h_prev | g] (32 x 64, tensor cores,
// K = nodes) and db = sum dP; per-block partials part[block][kGradLayer].
__global__ void __launch_bounds__(kLB) k_lm_wgrad(const b16 *__restrict__ dP, const b16 *__restrict__ Hprev,
                                                  const b16 *__restrict__ G, int n, float *part) {
    pdl_enter();
    __shared__ __align__(16) b16 PT[kLB / 32][W * LDK];      // dP^T tiles (32 features x 16 nodes)
    __shared__ __align__(16) b16 HT[kLB / 32][2 * W * LDK];  // [h | g]^T tiles (64 x 16 nodes)
    __shared__ float red[kLB / 32][W];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float d[2][8][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) d[mt][nt][e] = 0.0f;
    float db = 0.0f;  // lane = feature
    b16 *P = PT[warp], *H = HT[warp];
    const int ngroups = (n + 15) >> 4;
    for (int gi = blockIdx.x * (kLB / 32) + warp; gi < ngroups; gi += gridDim.x * (kLB / 32)) {
        const int i0 = gi * 16;
        // transposed tiles: lane = feature c; 16 nodes each
        for (int k = 0; k < 16; ++k) {
            const int i = i0 + k;
            const b16 zero = __float2bfloat16_rn(0.0f);
            const b16 pv = (i < n) ? dP[(size_t)i * W + lane] : zero;
            P[lane * LDK + k] = pv;
            H[lane * LDK + k] = (i < n) ? Hprev[(size_t)i * W + lane] : zero;
            H[(W + lane) * LDK + k] = (i < n) ? G[(size_t)i * W + lane] : zero;
            db = add_rn(db, __bfloat162float(pv));
        }
        __syncwarp();
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            uint32_t a[4];
            frag_a(a, P + 16 * mt * LDK, LDK, 0, lane);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                uint32_t b0, b1;
                frag_b(b0, b1, H, LDK, nt, 0, lane);
                mma_bf16(d[mt][nt], a, b0, b1);
            }
        }
        __syncwarp();
    }
    // reduce the warps' accumulators in a fixed order through shared memory
    __shared__ float acc_sm[W * 2 * W];
    const int g = lane >> 2, t = lane & 3;
    for (int w = 0; w < kLB / 32; ++w) {
        if (warp == w) {
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int m = 16 * mt + g + 8 * (e >> 1), c = 8 * nt + 2 * t + (e & 1);
                        acc_sm[m * 2 * W + c] = (w == 0) ? d[mt][nt][e] : add_rn(acc_sm[m * 2 * W + c], d[mt][nt][e]);
                    }
            red[w][lane] = db;
        }
        __syncthreads();
    }
    float *out = part + (size_t)blockIdx.x * kGradLayer;
    for (int k = threadIdx.x; k < W * 2 * W; k += blockDim.x) out[k] = acc_sm[k];
    if (threadIdx.x < W) {
        float s = red[0][threadIdx.x];
        for (int w = 1; w < kLB / 32; ++w) s = add_rn(s, red[w][threadIdx.x]);
        out[W * 2 * W + threadIdx.x] = s;
    }
}

// [dh_self | u] = dP [Ws | Wm]  (per node, 16 x 32 by 32 x 64, tensor cores):
// dh_self fp32 -> dHs, u bf16 -> U
__global__ void __launch_bounds__(kLB) k_lm_bprod(const b16 *__restrict__ dP, int n, int l, NetDev net, float *dHs,
                                                  b16 *U) {
    pdl_enter();
    __shared__ __align__(16) b16 WT[2 * W * LDWT];
    __shared__ __align__(16) b16 T[kLB / 32][16 * LDWT];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int idx = threadIdx.x; idx < 2 * W * W; idx += blockDim.x)
        WT[(idx / W) * LDWT + idx % W] = net.wcatT[(size_t)l * 2 * W * W + idx];
    __syncthreads();
    b16 *Tw = T[warp];
    const int g = lane >> 2, t = lane & 3;
    const int ngroups = (n + 15) >> 4;
    for (int gi = blockIdx.x * (kLB / 32) + warp; gi < ngroups; gi += gridDim.x * (kLB / 32)) {
        const int i0 = gi * 16;
        for (int q = lane; q < 16 * (W / 8); q += 32) {
            const int rr = q / (W / 8), ch = q % (W / 8), i = i0 + rr;
            Pack<b16, 8> v;
            if (i < n) v = ldp<b16, 8>(dP + (size_t)i * W + ch * 8);
            else
#pragma unroll
                for (int e = 0; e < 8; ++e) v.v[e] = __float2bfloat16_rn(0.0f);
            stp<b16, 8>(Tw + rr * LDWT + ch * 8, v);
        }
        __syncwarp();
        float d[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) d[nt][e] = 0.0f;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            uint32_t a[4];
            frag_a(a, Tw, LDWT, ks, lane);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                uint32_t b0, b1;
                frag_b(b0, b1, WT, LDWT, nt, ks, lane);
                mma_bf16(d[nt], a, b0, b1);
            }
        }
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int i = i0 + g + 8 * (e >> 1), c = 8 * nt + 2 * t + (e & 1);
                if (i < n) {
                    if (c < W) dHs[(size_t)i * W + c] = d[nt][e];
                    else U[(size_t)i * W + (c - W)] = __float2bfloat16_rn(d[nt][e]);
                }
            }
        __syncwarp();
    }
}

// dh_prev_j = dHs_j + sum_{i != j} A^_ij u_i (A^ symmetric), then
// dP_prev = bf16(dh_prev * [h_prev > 0]); for the embedding layer also
// per-block partials [de (W) | db0 (W)] in part[block][2W].
template <bool EMBED>
__global__ void __launch_bounds__(kLB) k_lm_bspmm(Sell A, const h16 *__restrict__ a16, const float *__restrict__ rs,
                                                  int n, const float *__restrict__ dHs, const b16 *__restrict__ U,
                                                  const b16 *__restrict__ Hprev, b16 *dPprev, const float *r,
                                                  const float *misc, float *part) {
    pdl_enter();
    __shared__ float sm[EMBED ? (kLB / 32) * 2 * W : 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rr = lane >> 1, hf = lane & 1;
    float acc2[EMBED ? 2 * W : 1];
    if constexpr (EMBED)
#pragma unroll
        for (int k = 0; k < 2 * W; ++k) acc2[k] = 0.0f;
    const float inv_s = misc ? misc[1] : 1.0f;
    const int ngroups = (n + 15) >> 4;
    for (int gi = blockIdx.x * (kLB / 32) + warp; gi < ngroups; gi += gridDim.x * (kLB / 32)) {
        const int j = gi * 16 + rr;
        if (j < n) {
            float acc[16];
            aggregate16(A, a16, rs, U, j, hf, acc);
            const Pack<b16, 8> h0 = ldp<b16, 8>(Hprev + (size_t)j * W + hf * 16);
            const Pack<b16, 8> h1 = ldp<b16, 8>(Hprev + (size_t)j * W + hf * 16 + 8);
            Pack<b16, 8> o0, o1;
            const float rt = EMBED ? mul_rn(r[j], inv_s) : 0.0f;
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int c = hf * 16 + e;
                const float dh = add_rn(dHs[(size_t)j * W + c], acc[e]);
                const float hv = __bfloat162float(e < 8 ? h0.v[e] : h1.v[e - 8]);
                const b16 q = __float2bfloat16_rn(hv > 0.0f ? dh : 0.0f);
                if (e < 8) o0.v[e] = q;
                else o1.v[e - 8] = q;
            }
            stp<b16, 8>(dPprev + (size_t)j * W + hf * 16, o0);
            stp<b16, 8>(dPprev + (size_t)j * W + hf * 16 + 8, o1);
            if constexpr (EMBED) {
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int c = hf * 16 + e;
                    const float pv = __bfloat162float(e < 8 ? o0.v[e] : o1.v[e - 8]);
                    acc2[c] = fma_rn(pv, rt, acc2[c]);
                    acc2[W + c] = add_rn(acc2[W + c], pv);
                }
            }
        }
    }
    if constexpr (EMBED) block_vec_sum<2 * W>(acc2, sm, part + (size_t)blockIdx.x * 2 * W);
}

// out[k] += sum_b part[b][k] (fixed block order), scattered by `map`:
// 0 layer block (dW -> dWs / dWm, db), 1 read-out tail (dwo, domega_j, loss),
// 2 embedding (de, db0)
__global__ void k_lm_reduce(const float *part, int nblocks, int K, int map, int l, float *grad, float *loss) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int b = 0; b < nblocks; ++b) s = add_rn(s, part[(size_t)b * K + k]);
        if (map == 0) {
            if (k < W * 2 * W) {
                const int m = k / (2 * W), c = k % (2 * W);
                float *dst = (c < W) ? grad + OFF_WS + l * W * W + m * W + c : grad + OFF_WM + l * W * W + m * W + (c - W);
                *dst = add_rn(*dst, s);
            } else {
                grad[OFF_B + l * W + (k - W * 2 * W)] = add_rn(grad[OFF_B + l * W + (k - W * 2 * W)], s);
            }
        } else if (map == 1) {
            if (k < W) grad[OFF_WO + k] = add_rn(grad[OFF_WO + k], s);
            else if (k == W) grad[OFF_OJ] = add_rn(grad[OFF_OJ], s);
            else *loss = add_rn(*loss, s);
        } else {
            if (k < W) grad[OFF_E + k] = add_rn(grad[OFF_E + k], s);
            else grad[OFF_B0 + (k - W)] = add_rn(grad[OFF_B0 + (k - W)], s);
        }
    }
}

// t = u - r (the residual of the net's output, u = A^ z)
__global__ void __launch_bounds__(kBlock) k_lm_sub(const float *u, const float *r, float *t, int n) {
    pdl_enter();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) t[i] = sub_rn(u[i], r[i]);
}

// 2 / (||e||^2 P) for the loss mean over P samples
__global__ void __launch_bounds__(kBlock) k_lm_coef(const float *e, int n, int P, float *coef, GridRed<float> gr) {
    float acc[1] = {0.0f};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        acc[0] = fma_rn(e[i], e[i], acc[0]);
    grid_reduce<float, 1>(acc, 1, false, gr, [&](float *res) { *coef = div_rn(2.0f, mul_rn(res[0], (float)P)); });
}

__global__ void k_lm_adam(float *theta, float *m, float *v, const float *grad, int np, float lr, float b1, float b2,
                          float eps, int step) {
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < np; k += gridDim.x * blockDim.x) {
        const float gk = grad[k];
        m[k] = fma_rn(b1, m[k], mul_rn(1.0f - b1, gk));
        v[k] = fma_rn(b2, v[k], mul_rn(1.0f - b2, mul_rn(gk, gk)));
        const float mh = m[k] / c1, vh = v[k] / c2;
        theta[k] = sub_rn(theta[k], mul_rn(lr, mh / (sqrtf(vh) + eps)));
    }
}

// fp16 Richardson vector -> fp32 net input
__global__ void __launch_bounds__(kBlock) k_lm_h2f(const h16 *x, float *y, int n, const int *flags, int check_depth) {
    pdl_enter();
    if (stopped(flags, check_depth)) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = __half2float(x[i]);
}


}  // namespace lm

// ------------------------------------------------------------------ host side
struct LearnedState {
    float *theta = nullptr, *grad = nullptr, *am = nullptr, *av = nullptr;
    b16 *wcat = nullptr, *wcatT = nullptr, *e_bf = nullptr, *wo_bf = nullptr;
    b16 *H[lm::NL + 1] = {}, *G[lm::NL] = {}, *dP[2] = {}, *U = nullptr;
    float *dHs = nullptr, *misc = nullptr, *part = nullptr, *coef = nullptr, *loss = nullptr, *zbuf = nullptr;
    float *r32 = nullptr;
    float *tbuf = nullptr, *vbuf = nullptr;  // residual loss: A^ z - r and A^ (A^ z - r)
    int loss_kind = 0;                       // 0: error loss, 1: residual loss
    int part_blocks = 0;
    bool train_buffers = false;
    int adam_step = 0;
};

namespace {
void *lalloc(Ctx &c, size_t bytes) {
    void *p = pool_alloc(c.dev, bytes, c.zstream);
    if (!p) return nullptr;
    c.allocs.push_back(p);
    c.bytes += (long long)bytes;
    cudaMemsetAsync(p, 0, bytes, c.zstream);
    return p;
}

lm::NetDev netdev(const LearnedState &L) { return lm::NetDev{L.theta, L.wcat, L.wcatT, L.e_bf, L.wo_bf}; }

int lm_grid(const Ctx &c) { return std::max(1, std::min(ceil_div((long long)c.n, 64), c.nsm * 4)); }
}  // namespace

f3r_status learned_enable(Ctx &c, const float *theta_host_or_dev, bool train) {
    if (!c.a16) return F3R_ERR_UNSUPPORTED;  // the net reads the fp16 copy of A^
    if (!c.learned) c.learned = new (std::nothrow) LearnedState;
    LearnedState &L = *c.learned;
    const size_t n = c.n, hw = n * lm::W;
    if (!L.theta) {
        L.theta = (float *)lalloc(c, sizeof(float) * lm::kNP);
        L.grad = (float *)lalloc(c, sizeof(float) * lm::kNP);
        L.am = (float *)lalloc(c, sizeof(float) * lm::kNP);
        L.av = (float *)lalloc(c, sizeof(float) * lm::kNP);
        L.wcat = (b16 *)lalloc(c, sizeof(b16) * lm::NL * lm::W * 2 * lm::W);
        L.wcatT = (b16 *)lalloc(c, sizeof(b16) * lm::NL * lm::W * 2 * lm::W);
        L.e_bf = (b16 *)lalloc(c, sizeof(b16) * lm::W);
        L.wo_bf = (b16 *)lalloc(c, sizeof(b16) * lm::W);
        L.misc = (float *)lalloc(c, sizeof(float) * 4);
        L.coef = (float *)lalloc(c, sizeof(float) * 4);
        L.loss = (float *)lalloc(c, sizeof(float) * 4);
        L.zbuf = (float *)lalloc(c, sizeof(float) * n);
        L.r32 = (float *)lalloc(c, sizeof(float) * n);
        L.H[0] = (b16 *)lalloc(c, sizeof(b16) * hw);
        L.H[1] = (b16 *)lalloc(c, sizeof(b16) * hw);
        L.part_blocks = lm_grid(c);
        L.part = (float *)lalloc(c, sizeof(float) * (size_t)L.part_blocks * lm::kGradLayer);
        if (!L.theta || !L.grad || !L.am || !L.av || !L.wcat || !L.wcatT || !L.e_bf || !L.wo_bf || !L.misc ||
            !L.coef || !L.loss || !L.zbuf || !L.r32 || !L.H[0] || !L.H[1] || !L.part)
            return F3R_ERR_NOMEM;
    }
    if (train && !L.train_buffers) {
        for (int l = 2; l <= lm::NL; ++l) L.H[l] = (b16 *)lalloc(c, sizeof(b16) * hw);
        for (int l = 0; l < lm::NL; ++l) L.G[l] = (b16 *)lalloc(c, sizeof(b16) * hw);
        L.dP[0] = (b16 *)lalloc(c, sizeof(b16) * hw);
        L.dP[1] = (b16 *)lalloc(c, sizeof(b16) * hw);
        L.U = (b16 *)lalloc(c, sizeof(b16) * hw);
        L.dHs = (float *)lalloc(c, sizeof(float) * hw);
        L.tbuf = (float *)lalloc(c, sizeof(float) * n);
        L.vbuf = (float *)lalloc(c, sizeof(float) * n);
        if (!L.tbuf || !L.vbuf) return F3R_ERR_NOMEM;
        for (int l = 2; l <= lm::NL; ++l)
            if (!L.H[l]) return F3R_ERR_NOMEM;
        for (int l = 0; l < lm::NL; ++l)
            if (!L.G[l]) return F3R_ERR_NOMEM;
        if (!L.dP[0] || !L.dP[1] || !L.U || !L.dHs) return F3R_ERR_NOMEM;
        L.train_buffers = true;
    }
    // the buffers are allocated and zeroed in the context's stream; the
    // copies below run in the legacy stream
    if (cudaStreamSynchronize(c.zstream) != cudaSuccess) return F3R_ERR_CUDA;
    if (theta_host_or_dev) {
        cudaMemcpy(L.theta, theta_host_or_dev, sizeof(float) * lm::kNP, cudaMemcpyDefault);
        cudaMemset(L.am, 0, sizeof(float) * lm::kNP);
        cudaMemset(L.av, 0, sizeof(float) * lm::kNP);
        L.adam_step = 0;
    }
    lm::k_lm_prepare<<<1, 256>>>(L.theta, L.wcat, L.wcatT, L.e_bf, L.wo_bf);
    return cudaDeviceSynchronize() == cudaSuccess ? F3R_OK : F3R_ERR_CUDA;
}

// z = M_theta(r) (fp32 device vectors of n), training-mode forward when train
void learned_forward(Ctx &c, const float *r, float *z, bool train, cudaStream_t s) {
    LearnedState &L = *c.learned;
    const Sell S = sell_of(c);
    const float *rs = c.prm.row_scale ? c.rs : nullptr;
    const lm::NetDev net = netdev(L);
    const int g = lm_grid(c);
    launch_pdl(lm::k_lm_scale, dim3(c.G), dim3(kBlock), 0, s, r, c.n, L.misc, GridRed<float>{(float *)c.partials, c.ticket, kMaxDots});
    launch_pdl(lm::k_lm_embed, dim3(std::max(1, std::min(ceil_div((long long)c.n * 4, kBlock), c.nsm * 8))), dim3(kBlock), 0,
               s, r, c.n, (const float *)L.misc, net, L.H[0]);
    c.launches += 2;
    for (int l = 0; l < lm::NL; ++l) {
        const bool last = (l == lm::NL - 1);
        const b16 *hin = train ? L.H[l] : L.H[l & 1];
        b16 *hout = train ? L.H[l + 1] : L.H[(l + 1) & 1];
        if (!last)
            launch_pdl(lm::k_lm_layer<0>, dim3(g), dim3(lm::kLB), 0, s, S, (const h16 *)c.a16, rs, c.n, hin, l, net, hout,
                       train ? L.G[l] : (b16 *)nullptr, (float *)nullptr, r, (const float *)L.misc);
        else if (train)
            launch_pdl(lm::k_lm_layer<2>, dim3(g), dim3(lm::kLB), 0, s, S, (const h16 *)c.a16, rs, c.n, hin, l, net, hout,
                       L.G[l], z, r, (const float *)L.misc);
        else
            launch_pdl(lm::k_lm_layer<1>, dim3(g), dim3(lm::kLB), 0, s, S, (const h16 *)c.a16, rs, c.n, hin, l, net,
                       (b16 *)nullptr, (b16 *)nullptr, z, r, (const float *)L.misc);
        c.launches++;
    }
}

// accumulate the gradient of the mean loss over P samples (R, E: P x n fp32)
f3r_status learned_loss_grad(Ctx &c, const float *R, const float *E, int P, cudaStream_t s) {
    LearnedState &L = *c.learned;
    const Sell S = sell_of(c);
    const float *rs = c.prm.row_scale ? c.rs : nullptr;
    const lm::NetDev net = netdev(L);
    const int g = lm_grid(c);
    const size_t n = c.n;
    cudaMemsetAsync(L.grad, 0, sizeof(float) * lm::kNP, s);
    cudaMemsetAsync(L.loss, 0, sizeof(float), s);
    for (int p = 0; p < P; ++p) {
        const float *r = R + (size_t)p * n, *e = E ? E + (size_t)p * n : nullptr;
        learned_forward(c, r, L.zbuf, true, s);
        const float *gdir = nullptr, *lossv = nullptr;
        if (L.loss_kind == 1) {
            // residual loss: d/dz ||A^ z - r||^2 = 2 A^T (A^ z - r), A^ symmetric
            launch_pdl(lm::k_lm_coef, dim3(c.G), dim3(kBlock), 0, s, r, c.n, P, L.coef,
                       GridRed<float>{(float *)c.partials, c.ticket, kMaxDots});
            if (launch_spmv(c, F3R_F16, F3R_F32, L.zbuf, L.vbuf, s) != F3R_OK) return F3R_ERR_UNSUPPORTED;
            launch_pdl(lm::k_lm_sub, dim3(c.G), dim3(kBlock), 0, s, (const float *)L.vbuf, r, L.tbuf, c.n);
            if (launch_spmv(c, F3R_F16, F3R_F32, L.tbuf, L.vbuf, s) != F3R_OK) return F3R_ERR_UNSUPPORTED;
            gdir = L.vbuf;
            lossv = L.tbuf;
            c.launches += 2;
        } else {
            launch_pdl(lm::k_lm_coef, dim3(c.G), dim3(kBlock), 0, s, e, c.n, P, L.coef,
                       GridRed<float>{(float *)c.partials, c.ticket, kMaxDots});
        }
        launch_pdl(lm::k_lm_out_bwd, dim3(g), dim3(lm::kLB), 0, s, (const float *)L.zbuf, e, r, c.n,
                   (const float *)L.misc, (const float *)L.coef, net, (const b16 *)L.H[lm::NL], L.dP[0], L.part,
                   gdir, lossv);
        lm::k_lm_reduce<<<1, 64, 0, s>>>(L.part, g, lm::W + 2, 1, 0, L.grad, L.loss);
        int cur = 0;
        for (int l = lm::NL - 1; l >= 0; --l) {
            launch_pdl(lm::k_lm_wgrad, dim3(g), dim3(lm::kLB), 0, s, (const b16 *)L.dP[cur], (const b16 *)L.H[l],
                       (const b16 *)L.G[l], c.n, L.part);
            lm::k_lm_reduce<<<ceil_div(lm::kGradLayer, 256), 256, 0, s>>>(L.part, g, lm::kGradLayer, 0, l, L.grad, L.loss);
            launch_pdl(lm::k_lm_bprod, dim3(g), dim3(lm::kLB), 0, s, (const b16 *)L.dP[cur], c.n, l, net, L.dHs, L.U);
            if (l > 0) {
                launch_pdl(lm::k_lm_bspmm<false>, dim3(g), dim3(lm::kLB), 0, s, S, (const h16 *)c.a16, rs, c.n,
                           (const float *)L.dHs, (const b16 *)L.U, (const b16 *)L.H[l], L.dP[cur ^ 1], r,
                           (const float *)L.misc, L.part);
            } else {
                launch_pdl(lm::k_lm_bspmm<true>, dim3(g), dim3(lm::kLB), 0, s, S, (const h16 *)c.a16, rs, c.n,
                           (const float *)L.dHs, (const b16 *)L.U, (const b16 *)L.H[0], L.dP[cur ^ 1], r,
                           (const float *)L.misc, L.part);
                lm::k_lm_reduce<<<1, 64, 0, s>>>(L.part, g, 2 * lm::W, 2, 0, L.grad, L.loss);
            }
            cur ^= 1;
            c.launches += 4;
        }
        c.launches += 4;
    }
    return cudaGetLastError() == cudaSuccess ? F3R_OK : F3R_ERR_CUDA;
}

void learned_adam(Ctx &c, float lr, cudaStream_t s) {
    LearnedState &L = *c.learned;
    L.adam_step++;
    lm::k_lm_adam<<<ceil_div(lm::kNP, 256), 256, 0, s>>>(L.theta, L.am, L.av, L.grad, lm::kNP, lr, 0.9f, 0.999f, 1e-8f,
                                                         L.adam_step);
    lm::k_lm_prepare<<<1, 256, 0, s>>>(L.theta, L.wcat, L.wcatT, L.e_bf, L.wo_bf);
    c.launches += 2;
}

// One Richardson call (Algorithm 1) whose M is the learned net: per step
// k, r_k = fp16(v - A^ z_k) (r_0 = v), u = M_theta(r_k), then the weighted
// update (update calls: w'_k from w = A^ u).  fp16 storage only.
void learned_rich_call(Ctx &c, bool update, int pos, void *out, const void *par_misc, cudaStream_t s) {
    LearnedState &L = *c.learned;
    const Sell S = sell_of(c);
    const float *rs = c.prm.row_scale ? c.rs : nullptr;
    const int cd = c.prm.nlevels - 1, n = c.n, m4 = c.prm.rich_m;
    h16 *zb[2] = {(h16 *)c.rz[0], (h16 *)c.rz[1]};
    for (int k = 0; k < m4; ++k) {
        const bool last = (k == m4 - 1);
        const h16 *zp = (k > 0) ? zb[(k - 1) & 1] : nullptr;
        const h16 *rk = (const h16 *)c.rin;
        if (k > 0) {
            launch_pdl(k_rich_upd_r<h16, h16, float>, dim3(c.Gs), dim3(kBlock), 0, s, sell_of(c), (const h16 *)c.a16, rs,
                       (const h16 *)c.rin, zp, (h16 *)c.rr, (const int *)c.flags, cd, n);
            rk = (const h16 *)c.rr;
            c.launches++;
        }
        launch_pdl(lm::k_lm_h2f, dim3(c.G), dim3(kBlock), 0, s, rk, L.r32, n, (const int *)c.flags, cd);
        learned_forward(c, L.r32, L.zbuf, false, s);
        if (update) {
            launch_pdl(k_rich_upd_w_u, dim3(c.Gs), dim3(kBlock), 0, s, S, (const h16 *)c.a16, rs, rk,
                       (const float *)L.zbuf, (float *)c.omega, (float *)c.wcur, (const long long *)c.c_ntr_base, k, pos,
                       c.prm.c, GridRed<float>{(float *)c.partials, c.ticket, kMaxDots}, (const int *)c.flags, cd, n);
            c.launches++;
        }
        launch_pdl(k_rich_z_u, dim3(c.G), dim3(kBlock), 0, s, (const float *)L.zbuf, zp, zb[k & 1], (float *)out,
                   (const float *)par_misc, (const float *)c.omega, (const float *)c.wcur, k, last ? 1 : 0,
                   update ? 1 : 0, (const int *)c.flags, cd, n, c.counters);
        c.launches += 2;
    }
}

f3r_status learned_set_loss(Ctx &c, int kind) {
    if (!c.learned || (kind != 0 && kind != 1)) return F3R_ERR_ARG;
    c.learned->loss_kind = kind;
    return F3R_OK;
}
int learned_loss_kind(const Ctx &c) { return c.learned ? c.learned->loss_kind : 0; }

float *learned_theta(Ctx &c) { return c.learned ? c.learned->theta : nullptr; }
float *learned_grad(Ctx &c) { return c.learned ? c.learned->grad : nullptr; }
float *learned_loss(Ctx &c) { return c.learned ? c.learned->loss : nullptr; }

void learned_free(Ctx &c) {
    delete c.learned;
    c.learned = nullptr;
}

}  // namespace f3r
