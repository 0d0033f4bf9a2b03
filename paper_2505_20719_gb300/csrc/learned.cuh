// Learned preconditioner M_theta: a 3-layer message-passing network of width
// 32 over the graph of the scaled matrix A^ (project addition).  For a
// residual r with s = 2^ceil(log2 max|r|), r~ = r / s:
//     h0_i = relu(e r~_i + b0)
//     g_i  = sum_{j != i} A^_ij h_j                    (aggregation, CUDA cores)
//     h_i  = relu([h_i | g_i] [Ws | Wm]^T + b),  3 layers (tensor cores)
//     z_i  = s (omega_j r~_i + wo . h_i)
// Weights, activations and messages are stored in bf16, every product is
// accumulated in fp32 (mma.sync m16n8k16 bf16 -> f32 for the per-node
// contractions).  Training keeps fp32 master weights and Adam moments.
#pragma once
#include "kernels.cuh"

namespace f3r {
namespace lm {

constexpr int W = 32;                 // width
constexpr int NL = 3;                 // message-passing layers
constexpr int kLB = 128;              // threads per block (4 warps, 16 nodes each per step)
constexpr int kPadH = 8;              // bf16 padding of shared-memory rows
constexpr int kNP = W + W + NL * W * W * 2 + NL * W + W + 1;  // 6337 parameters
// offsets of the parameter blocks in the flat vector (e, b0, Ws, Wm, b, wo, omega_j)
constexpr int OFF_E = 0, OFF_B0 = W, OFF_WS = 2 * W, OFF_WM = OFF_WS + NL * W * W, OFF_B = OFF_WM + NL * W * W,
              OFF_WO = OFF_B + NL * W, OFF_OJ = OFF_WO + W;
// per-block partial layout of the weight-gradient reductions: per layer
// [32 x 64 dW | 32 db], plus [32 de | 32 db0 | 32 dwo | 1 domega_j]
constexpr int kGradLayer = W * 2 * W + W;
constexpr int kGradTail = 3 * W + 1;

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld32(const b16 *p) { return *reinterpret_cast<const uint32_t *>(p); }
__device__ __forceinline__ uint32_t pack2(b16 lo, b16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// A fragment (16 x 16, row-major) of k-step ks from a shared tile T[16][ldt]
__device__ __forceinline__ void frag_a(uint32_t (&a)[4], const b16 *T, int ldt, int ks, int lane) {
    const int g = lane >> 2, t = lane & 3;
    a[0] = ld32(T + g * ldt + 16 * ks + 2 * t);
    a[1] = ld32(T + (g + 8) * ldt + 16 * ks + 2 * t);
    a[2] = ld32(T + g * ldt + 16 * ks + 8 + 2 * t);
    a[3] = ld32(T + (g + 8) * ldt + 16 * ks + 8 + 2 * t);
}
// B fragment (16 x 8) for output tile nt, k-step ks from Wt[n][ldw] (row n holds B's column n)
__device__ __forceinline__ void frag_b(uint32_t &b0, uint32_t &b1, const b16 *Wt, int ldw, int nt, int ks, int lane) {
    const int g = lane >> 2, t = lane & 3;
    b0 = ld32(Wt + (8 * nt + g) * ldw + 16 * ks + 2 * t);
    b1 = ld32(Wt + (8 * nt + g) * ldw + 16 * ks + 8 + 2 * t);
}

struct NetDev {
    const float *theta;  // fp32 master parameters (flat, kNP)
    const b16 *wcat;     // [NL][W][2W] bf16: row a = [Ws row a | Wm row a]
    const b16 *wcatT;    // [NL][2W][W] bf16: transposed, for the backward product
    const b16 *e_bf, *wo_bf;
};

}  // namespace lm
}  // namespace f3r
