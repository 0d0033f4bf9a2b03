// Shared device helpers of libf3r: typed loads/stores with explicit
// rounding, warp reductions and the deterministic grid reduction.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "f3r.h"

namespace f3r {

constexpr int kBlock = 256;          // threads per block of the vector / SpMV kernels
constexpr int kWarps = kBlock / 32;
constexpr int kSlice = 32;           // rows per SELL slice (Sec. 5.2: chunk size 32)
constexpr int kMaxInnerM = 15;       // inner FGMRES iterations (fits the fused dot registers)
constexpr int kMaxDots = kMaxInnerM + 1;
constexpr int kMaxOuterM = 128;      // outer restart length
constexpr int kMaxStagedBlocksPerSM = 8;  // blocks per SM of a staged kernel at most (partials sized for it)
constexpr int kMaxLongM = 64;        // inner levels beyond kMaxInnerM (chunked CGS2, Table 4's F2)
constexpr int kMaxRich = 8;

typedef __half h16;
typedef __nv_bfloat16 b16;

// ------------------------------------------------------------------ arithmetic
// Explicitly rounded operations, so that the compiler never contracts or
// reorders what the method specifies.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float sqrt_rn(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ double sqrt_rn(double a) { return __dsqrt_rn(a); }

// ------------------------------------------------------------ storage formats
// to_c<TC>(stored value) widens exactly; store<S>(TC) rounds to nearest even.
template <class TC> __device__ __forceinline__ TC to_c(double x) { return (TC)x; }
template <class TC> __device__ __forceinline__ TC to_c(float x) { return (TC)x; }
template <class TC> __device__ __forceinline__ TC to_c(h16 x) { return (TC)__half2float(x); }
template <class TC> __device__ __forceinline__ TC to_c(b16 x) { return (TC)__bfloat162float(x); }

template <class S> struct Store;
template <> struct Store<double> {
    __device__ static __forceinline__ double from(double x) { return x; }
};
template <> struct Store<float> {
    __device__ static __forceinline__ float from(float x) { return x; }
    __device__ static __forceinline__ float from(double x) { return __double2float_rn(x); }
};
template <> struct Store<h16> {
    __device__ static __forceinline__ h16 from(float x) { return __float2half_rn(x); }
    __device__ static __forceinline__ h16 from(double x) { return __double2half(x); }
};
template <> struct Store<b16> {
    __device__ static __forceinline__ b16 from(float x) { return __float2bfloat16_rn(x); }
    __device__ static __forceinline__ b16 from(double x) { return __double2bfloat16(x); }
};

// value rounded to storage format S and widened back to the compute type
template <class S, class TC> __device__ __forceinline__ TC rnd(TC x) {
    return to_c<TC>(Store<S>::from(x));
}

template <class S> struct IsHalfWidth { static constexpr bool value = false; };
template <> struct IsHalfWidth<h16> { static constexpr bool value = true; };
template <> struct IsHalfWidth<b16> { static constexpr bool value = true; };

// 2^-floor(log2 a) for a finite a > 0, else 1 (scaling before a 16-bit cast)
template <class T> __device__ __forceinline__ T pow2_scale_for(T a) {
    if (!(a > (T)0) || !isfinite(a)) return (T)1;
    int e;
    frexp((double)a, &e);  // a = f 2^e, f in [0.5, 1): floor(log2 a) = e - 1
    return (T)ldexp(1.0, 1 - e);
}

// ----------------------------------------------------------------- reductions
template <class T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = add_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
template <class T> __device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Scratch of one deterministic grid reduction: per-block partials and the
// ticket that elects the last block.  `partials` holds gridDim.x * stride.
template <class T> struct GridRed {
    T *partials;
    unsigned *ticket;
    int stride;
};

// Block totals of nd sums (warps summed in order) written to
// part[d * gridDim.x + blockIdx.x]; the next kernel sums them over blocks
// (warp_sum_partials), so no block waits for a last one here.
template <class T, int ND>
__device__ __forceinline__ void block_partials(T (&acc)[ND], int nd, T *part) {
    __shared__ T sm[ND][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        if (d < nd) {
            const T v = warp_sum(acc[d]);
            if (lane == 0) sm[d][warp] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x < nd) {
        const int d = threadIdx.x;
        T s = sm[d][0];
        for (int w = 1; w < nwarps; ++w) s = add_rn(s, sm[d][w]);
        part[(size_t)d * gridDim.x + blockIdx.x] = s;
    }
}

// Deterministic grid-wide reduction of `nd` sums (and optionally one max,
// passed as acc[nd] when with_max) per thread.  Every block writes its
// partials; the last block to arrive (atomic ticket) sums all partials in a
// fixed block order and thread 0 calls fin(result).  Returns true in the
// thread that ran fin.  The order of every addition depends only on the grid
// and block shape, so results are reproducible run to run.
template <class T, int ND, class Fin>
__device__ __forceinline__ void grid_reduce(T (&acc)[ND], int nd, bool with_max, GridRed<T> gr, Fin fin) {
    __shared__ T sm[ND][32];
    __shared__ bool am_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int ntot = nd + (with_max ? 1 : 0);
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        if (d < ntot) {
            T v = (with_max && d == nd) ? warp_max(acc[d]) : warp_sum(acc[d]);
            if (lane == 0) sm[d][warp] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x < ntot) {
        const int d = threadIdx.x;
        T s = sm[d][0];
        for (int w = 1; w < nwarps; ++w) s = (with_max && d == nd) ? fmax(s, sm[d][w]) : add_rn(s, sm[d][w]);
        gr.partials[(size_t)blockIdx.x * gr.stride + d] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = atomicAdd(gr.ticket, 1u);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    T loc[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) loc[d] = (T)0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            if (d < ntot) {
                T p = __ldcg(gr.partials + (size_t)b * gr.stride + d);
                loc[d] = (with_max && d == nd) ? fmax(loc[d], p) : add_rn(loc[d], p);
            }
        }
    }
    __syncthreads();  // every block's sm reuse below is after all reads of sm above
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        if (d < ntot) {
            T v = (with_max && d == nd) ? warp_max(loc[d]) : warp_sum(loc[d]);
            if (lane == 0) sm[d][warp] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        T res[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            if (d < ntot) {
                T s = sm[d][0];
                for (int w = 1; w < nwarps; ++w) s = (with_max && d == nd) ? fmax(s, sm[d][w]) : add_rn(s, sm[d][w]);
                res[d] = s;
            } else {
                res[d] = (T)0;
            }
        }
        fin(res);
        *gr.ticket = 0u;
    }
}

// ------------------------------------------------------------------- matrix
// Sliced ELLPACK with slices of 32 rows (Sec. 5.2), entries of a slice stored
// column-major (entry k of row 32 s + lane at sptr[s] + 32 k + lane), so a
// warp reads 32 consecutive values per step.  Padding entries carry column
// -1 and are skipped.  Rows keep their CSR order, so every row sum
// accumulates in the same order as a CSR traversal.
struct Sell {
    int n;
    int nslices;
    const int *sptr;  // nslices + 1 entry offsets (multiples of 32)
    const int *col;   // column of each entry, -1 for padding
};

// sum_k a_k x_{c_k} over one row with fused multiply-add in CSR order; the
// loads of a group of 4 entries are issued before its multiply-adds
template <class TC, class TA, class GX>
__device__ __forceinline__ TC sell_row(const Sell &S, const TA *__restrict__ val, int s, int lane, GX gx) {
    constexpr int U = 4;
    const int beg = __ldg(S.sptr + s) + lane;
    const int w = (__ldg(S.sptr + s + 1) - __ldg(S.sptr + s)) >> 5;
    TC acc = (TC)0;
    for (int k0 = 0; k0 < w; k0 += U) {
        int c[U];
        TC a[U], xv[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int idx = beg + ((k0 + q) << 5);
            c[q] = (k0 + q < w) ? __ldg(S.col + idx) : -1;
            a[q] = (k0 + q < w) ? to_c<TC>(val[idx]) : (TC)0;
        }
#pragma unroll
        for (int q = 0; q < U; ++q) xv[q] = (c[q] >= 0) ? gx(c[q]) : (TC)0;
#pragma unroll
        for (int q = 0; q < U; ++q)
            if (c[q] >= 0) acc = fma_rn(a[q], xv[q], acc);
    }
    return acc;
}

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// Programmatic dependent launch.  pdl_wait: wait until every prerequisite
// grid has completed and its writes are visible (a kernel launched with the
// programmatic attribute calls it before touching anything an earlier kernel
// writes).  pdl_trigger: let the next kernel in the stream start launching
// (its blocks run their prologue as this grid drains); without it that
// happens when this grid exits.  Both are no-ops without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_enter() { pdl_wait(); }

// programmatic dependent launch, on unless F3R_PDL=0 is set in the environment
bool pdl_enabled();

// launch with the programmatic-stream-serialization attribute
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

}  // namespace f3r

namespace f3r {
// 16-byte packs for vectorised streaming of Krylov vectors (float4 / double2)
template <class T, int N> struct alignas(sizeof(T) * N) Pack {
    T v[N];
};
template <class T> struct PackN {
    static constexpr int N = 16 / sizeof(T);
};
template <class T, int N> __device__ __forceinline__ Pack<T, N> ldp(const T *p) {
    return *reinterpret_cast<const Pack<T, N> *>(p);
}
template <class T, int N> __device__ __forceinline__ void stp(T *p, const Pack<T, N> &x) {
    *reinterpret_cast<Pack<T, N> *>(p) = x;
}
}  // namespace f3r
