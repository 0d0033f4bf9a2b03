// Shared-memory staging of sliced-ELLPACK slices with bulk asynchronous
// copies (TMA, cp.async.bulk) and mbarrier completion.
//
// Each warp walks its slices s = first, first + stride, ... through a ring of
// S shared-memory stages.  Lane 0 issues, per slice, one bulk copy for the
// slice's column indices, one for its values and one per extra row-aligned
// vector segment (e.g. the Krylov basis rows the fused dot products read),
// all completing on the stage's mbarrier.  S slices are in flight per warp,
// which keeps enough bytes moving to cover HBM latency while the lanes
// gather x from L1/L2 and accumulate.
//
// Every wait is bounded: after kSpinLimit failed polls the kernel records
// an error code, waits (bounded again) for its own copies still in flight and
// returns, so a lost completion can never hang the GPU.
#pragma once
#include "common.cuh"

namespace f3r {

constexpr long long kSpinLimit = 1LL << 24;
constexpr int kMaxExtra = kMaxDots + 1;
enum { ERR_STAGE_TIMEOUT = 1 };

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// global -> shared bulk copy; dst, src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait; false after kSpinLimit polls
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (long long it = 0; it < kSpinLimit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Extra row-aligned segments staged with each slice: rows [32 s, 32 s + 32)
// of `count` vectors base + l * ld (element size esize bytes).
struct Extra {
    const void *base = nullptr;
    int count = 0;
    int ld = 0;
    int esize = 4;
};

// Shared-memory layout of one stage for a slice of width w:
//   [col: 32 w int32][val: 32 w TA][extra l: 32 elements each]
template <class TA> struct StageView {
    const int *col;
    const TA *val;
    const char *extra;
    int w;
    int esize;
    template <class T> __device__ const T *ext(int l) const {
        return reinterpret_cast<const T *>(extra + (size_t)l * kSlice * esize);
    }
};

// Per-warp ring of S stages over the warp's slices.  `ring` points to this
// warp's S * stage_bytes of dynamic shared memory, `bars` to its S mbarriers.
// body(s, view) is called by all 32 lanes for every slice in order.
template <class TA, int S, class Body>
__device__ __forceinline__ bool staged_slices(const Sell &A, const TA *__restrict__ val, int first, int stride,
                                              char *ring, int stage_bytes, uint64_t *bars, Extra ex, int *err,
                                              Body body) {
    const int lane = threadIdx.x & 31;
    auto issue = [&](int s, int st) {
        const int b0 = __ldg(A.sptr + s), b1 = __ldg(A.sptr + s + 1);
        const int w = (b1 - b0) >> 5;
        const uint32_t colb = (uint32_t)w * kSlice * 4u;
        const uint32_t valb = (uint32_t)w * kSlice * (uint32_t)sizeof(TA);
        const uint32_t extb = (uint32_t)kSlice * ex.esize;
        const uint32_t bar = smem_u32(bars + st);
        const uint32_t dst = smem_u32(ring + (size_t)st * stage_bytes);
        fence_proxy_async();  // earlier generic reads of this stage before the async refill
        mbar_expect_tx(bar, colb + valb + extb * ex.count);
        if (colb) {
            bulk_g2s(dst, A.col + b0, colb, bar);
            bulk_g2s(dst + colb, val + b0, valb, bar);
        }
        for (int l = 0; l < ex.count; ++l)
            bulk_g2s(dst + colb + valb + l * extb,
                     (const char *)ex.base + ((size_t)l * ex.ld + (size_t)s * kSlice) * ex.esize, extb, bar);
    };
    if (lane == 0) {
        for (int st = 0; st < S; ++st) mbar_init(smem_u32(bars + st), 1);
        fence_mbar_init();
    }
    __syncwarp();
    if (lane == 0)
        for (int st = 0; st < S; ++st) {
            const int s = first + st * stride;
            if (s < A.nslices) issue(s, st);
        }
    __syncwarp();
    bool ok = true;
    int k = 0;
    for (int s = first; s < A.nslices; s += stride, ++k) {
        const int st = k % S;
        const uint32_t parity = (uint32_t)((k / S) & 1);
        if (!mbar_wait(smem_u32(bars + st), parity)) {
            ok = false;
            break;
        }
        const char *base = ring + (size_t)st * stage_bytes;
        const int b0 = __ldg(A.sptr + s), b1 = __ldg(A.sptr + s + 1);
        StageView<TA> v;
        v.w = (b1 - b0) >> 5;
        v.col = reinterpret_cast<const int *>(base);
        v.val = reinterpret_cast<const TA *>(base + (size_t)v.w * kSlice * 4);
        v.extra = base + (size_t)v.w * kSlice * (4 + sizeof(TA));
        v.esize = ex.esize;
        body(s, v);
        __syncwarp();
        const int sn = s + S * stride;
        if (lane == 0 && sn < A.nslices) issue(sn, st);
        __syncwarp();
    }
    if (!ok) {
        // record the failure, then drain this warp's copies still in flight (bounded)
        if (lane == 0) atomicOr(err, ERR_STAGE_TIMEOUT);
        int kk = k;
        for (int s = first + k * stride; s < A.nslices && kk < k + S; s += stride, ++kk)
            mbar_wait(smem_u32(bars + kk % S), (uint32_t)((kk / S) & 1));
    }
    return ok;
}

// stage size in bytes for slices of width up to wmax
__host__ __device__ inline int stage_bytes_for(int wmax, int asize, int n_extra, int esize) {
    const int b = wmax * kSlice * (4 + asize) + n_extra * kSlice * esize;
    return (b + 15) / 16 * 16;
}

}  // namespace f3r
