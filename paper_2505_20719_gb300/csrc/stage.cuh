// Shared-memory staging of sliced-ELLPACK slices with bulk asynchronous
// copies (TMA, cp.async.bulk) and mbarrier completion.
//
// A block walks a contiguous range of tiles (8 consecutive slices = 256
// rows) through a ring of S shared-memory stages.  A producer warp issues,
// per tile, one bulk copy for the tile's column indices, one for its values
// and one per extra row-aligned vector segment (e.g. the Krylov basis rows
// the fused dot products read), all completing on the stage's mbarrier.  S
// tiles are in flight per block, which keeps enough bytes moving to cover HBM
// latency while the consumer warps gather x (largely from L1, since a block's
// tiles are neighbours) and accumulate.
//
// Every wait is bounded: after about two seconds of failed polls the kernel
// records an error code, waits (bounded again) for its own copies still in
// flight and returns, so a lost completion can never hang the GPU.
#pragma once
#include "common.cuh"

namespace f3r {

constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at the 2.07 GHz SM clock
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

// Order every earlier generic-proxy access (including the previous grid's
// writes made visible by griddepcontrol.wait) before later async-proxy (TMA)
// accesses of this thread.
__device__ __forceinline__ void fence_proxy_async_all() { asm volatile("fence.proxy.async;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// raise the barrier's expected transaction bytes without arriving (the
// phase cannot complete before the arrive that follows)
__device__ __forceinline__ void mbar_expect_tx_only(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// global -> shared bulk copy; dst, src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// L2 policy for data read once per pass (the matrix tiles): evicted first, so
// that the vectors the next kernels read (the basis, w, z, x) stay in L2
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// bulk_g2s with an L2 cache policy
__device__ __forceinline__ void bulk_g2s_hint(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar,
                                              uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar), "l"(policy)
        : "memory");
}


// A waiting thread may be suspended for up to kSuspendNs inside one
// try_wait (it resumes as soon as the phase completes), so a warp that waits
// for a stage does not spin through issue slots the working warps need.
constexpr unsigned kSuspendNs = 20000;

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "n"(kSuspendNs)
        : "memory");
    return ok != 0;
}

// Bounded, warp-uniform wait for phase `parity` of a barrier: every lane
// polls (so each lane acquires the completed phase), the warp leaves together
// once all lanes saw it, and gives up after kWaitCycles of lane 0's clock
// (read only once the first poll found the phase incomplete).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
    const long long t0 = __shfl_sync(0xffffffffu, (long long)clock64(), 0);
    for (;;) {
        const bool ok = mbar_try_wait(bar, parity);
        if (__all_sync(0xffffffffu, ok)) return true;
        const long long now = __shfl_sync(0xffffffffu, (long long)clock64(), 0);
        if (now - t0 > kWaitCycles) return false;
    }
}

// Extra row-aligned segments staged with each tile: rows [256 t, 256 t + 256)
// of `count` vectors base + l * ld (element size esize bytes; ld a multiple
// of 256 so that every tile's rows exist).
struct Extra {
    const void *base = nullptr;
    int count = 0;
    int ld = 0;
    int esize = 4;
};

// A tile is kTileSlices slices; consumer warp w takes slices w, w + kWarps, ...
#ifndef F3R_TILE_SLICES
#define F3R_TILE_SLICES 16
#endif
constexpr int kTileSlices = F3R_TILE_SLICES;
constexpr int kTileRows = kTileSlices * kSlice;  // 512 rows per tile
static_assert(kTileSlices % kWarps == 0 && kTileSlices < 32, "whole slices per consumer warp, offsets in one warp");

// Windowed tiles.  The columns the rows of one tile reference, and the
// tile's own rows, are covered by at most kWinRuns runs of consecutive x
// entries that start and end on kWinChunk-entry boundaries; the producer
// bulk-copies those runs of x into the stage after the tile's matrix and
// zeroes the 16 bytes just past them (the zero slot), and the tile's entries
// carry 16-bit indices into that window instead of int32 columns, so the
// consumers gather x from shared memory.  A padding entry (value +0) points
// at the zero slot: it adds +0 * +0 to its row sum, which leaves every sum
// bit for bit as it was (a sum that starts at +0 never becomes -0 under
// round-to-nearest, and x + (+0) = x for every other x), so no entry needs a
// test.  Per tile a record of kWinRec ints: [runs, window entries, 1 if a
// run reaches past the last row of x (else 0), window index of the tile's
// first row, then (first column, entries, window position) per run].
constexpr int kWinChunk = 32;
constexpr int kWinRuns = 9;
constexpr int kWinRec = 32;
constexpr int kWinRecClamp = 2;
constexpr int kWinRecOwn = 3;
constexpr int kWinRecRun = 4;  // run r at kWinRecRun + 3 r
constexpr int kWinMaxEntries = 4096;
constexpr int kWinPadBytes = 16;  // the zero slot after the window
constexpr int kWinStages = 3;     // ring depth of the windowed kernels

struct Window {
    const uint16_t *lcol = nullptr;  // window index of every SELL entry (padding: the zero slot)
    const int *rec = nullptr;        // kWinRec ints per tile
    const void *x = nullptr;         // the gathered vector
    int xsize = 0;                   // its element size (2, 4 or 8 bytes)
    int n = 0;                       // its entries (runs are clamped to them)
};
// stage header: the tile's kTileSlices + 1 slice offsets (int), padded to a
// multiple of 16 bytes, then (windowed tiles) the tile's window record, so the
// bulk copies after it stay aligned
constexpr int kStageOffs = ((kTileSlices + 1) * 4 + 15) / 16 * 16;
constexpr int kStageHdr = kStageOffs + kWinRec * 4;

// What one warp sees of its slice in a staged tile.
template <class TA> struct StageView {
    const int *col;     // 32 w entries, column-major within the slice (plain tiles)
    const uint16_t *lcol;  // the same as window indices (windowed tiles)
    const TA *val;
    const char *extra;  // extra l of the whole tile at extra + l * 256 * esize
    const char *win;    // the tile's x window (windowed tiles)
    int own;            // window index of the tile's first row (windowed tiles)
    int w;
    int esize;
    int row0;           // row of lane 0 inside the tile (32 * warp)
    template <class T> __device__ const T *ext(int l) const {
        return reinterpret_cast<const T *>(extra + (size_t)l * kTileRows * esize) + row0;
    }
    template <class T> __device__ const T *xwin() const { return reinterpret_cast<const T *>(win); }
};

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Warp-specialised ring of S stages over a contiguous range of tiles.  The
// block has kWarps consumer warps and one producer warp (the last).  The
// producer's lane 0 fills stage st with one bulk copy of the tile's column
// indices, one of its values and one per extra vector, completing on
// full[st]; consumer warp w waits on full[st], processes slice w of the tile
// and arrives on empty[st]; the producer refills a stage once all consumers
// released it.  Consumers therefore run up to S - 1 tiles apart without a
// block-wide barrier.  body(s, view) runs on all lanes of the consumer warp
// owning slice s.  Every wait is bounded; a consumer that gives up records
// the error and stops, the producer stops refilling after a failed wait and
// finally waits (bounded) for the copies it issued.
// gate(): evaluated by every thread once the producer has issued the copies
// of the first S tiles (the matrix and the extras, which no kernel still
// running writes): it waits for the prerequisite grids and returns false
// when the kernel has nothing to do; the producer then waits for the copies
// it issued and the call returns false.
// WIN: windowed tiles (16-bit window indices, Window wn).  The x window of a
// tile is written by the grid the gate waits for, so its runs are copied
// only after the gate: the first S tiles' matrix copies raise their stage's
// expected bytes without arriving, and the window copies (plus the arrive)
// follow the gate.  A run ending past the last 16-byte boundary of x is
// copied in bulk up to that boundary and the rest entry by entry by the
// producer lanes before the arrive.
template <class TA, int S, bool EVICT_FIRST = false, bool WIN = false, class Body, class Gate>
__device__ __forceinline__ bool staged_tiles_gated(const Sell &A, const TA *__restrict__ val, int tile_begin,
                                                   int tile_end, char *ring, int stage_bytes, uint64_t *full,
                                                   uint64_t *empty, Extra ex, int *err, Body body, Gate gate,
                                                   Window wn = Window()) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool producer = (warp == kWarps);
    constexpr uint32_t kIdxBytes = WIN ? 2u : 4u;
    // metadata of the next tile the producer issues, loaded one tile ahead so
    // that no global-load latency sits between two tiles' copies: lanes
    // 0..kTileSlices hold its slice offsets, lane q word q of its window record
    int meta_off = 0, meta_rec = 0;
    uint64_t policy = 0;  // L2 policy of the matrix copies (EVICT_FIRST)
    if constexpr (EVICT_FIRST)
        if (producer) policy = l2_evict_first_policy();
    auto prefetch = [&](int t) {
        if (t >= tile_end) return;
        const int s0 = t * kTileSlices;
        meta_off = (lane <= kTileSlices) ? __ldg(A.sptr + min(s0 + lane, min(s0 + kTileSlices, A.nslices))) : 0;
        if constexpr (WIN) meta_rec = __ldg(wn.rec + (size_t)t * kWinRec + lane);
    };
    // run by the whole producer warp: lanes 0..8 write the tile's slice
    // offsets into the stage header (the consumers read them from shared
    // memory instead of global memory), all lanes its window record, then the
    // next tile's metadata is requested; lane 0 issues the bulk copies of the
    // matrix and the extras; with `arrive` false (windowed tiles) it only
    // raises the expected bytes and issue_window arrives
    auto issue = [&](int t, int st, bool arrive) {
        char *sbase = ring + (size_t)st * stage_bytes;
        const int off = meta_off;
        if (lane <= kTileSlices) reinterpret_cast<int *>(sbase)[lane] = off;
        if constexpr (WIN) reinterpret_cast<int *>(sbase + kStageOffs)[lane] = meta_rec;
        prefetch(t + 1);
        const int b0 = __shfl_sync(0xffffffffu, off, 0), b1 = __shfl_sync(0xffffffffu, off, kTileSlices);
        const uint32_t colb = (uint32_t)(b1 - b0) * kIdxBytes;
        const uint32_t valb = (uint32_t)(b1 - b0) * (uint32_t)sizeof(TA);
        const uint32_t extb = (uint32_t)kTileRows * ex.esize;
        const uint32_t bar = smem_u32(full + st);
        const uint32_t dst = smem_u32(sbase + kStageHdr);
        __syncwarp();  // the header before lane 0's arrive (release) on full[st]
        if (lane == 0) {
            if (arrive) mbar_expect_tx(bar, colb + valb + extb * ex.count);
            else mbar_expect_tx_only(bar, colb + valb + extb * ex.count);
        }
        __syncwarp();  // the expected bytes raised before any copy can complete
        // lane 0 copies the indices, lane 1 the values, lane 2 + l extra l
        if (lane >= 2 + ex.count || (lane < 2 && colb == 0)) return;
        fence_proxy_async();  // the consumers' generic reads of this stage before the async refill
        if (lane < 2) {
            const void *src;
            if (lane == 0) {
                if constexpr (WIN) src = wn.lcol + b0;
                else src = A.col + b0;
            } else {
                src = val + b0;
            }
            const uint32_t d = dst + (lane == 0 ? 0u : colb), bytes = lane == 0 ? colb : valb;
            if constexpr (EVICT_FIRST) bulk_g2s_hint(d, src, bytes, bar, policy);
            else bulk_g2s(d, src, bytes, bar);
        } else {
            const int l = lane - 2;
            bulk_g2s(dst + colb + valb + l * extb,
                     (const char *)ex.base + ((size_t)l * ex.ld + (size_t)t * kTileRows) * ex.esize, extb, bar);
        }
    };
    // windowed tiles, after issue(t, st, false) and the gate: the x runs of
    // the tile in stage st (lane r + 1 copies run r), then the arrive on full[st]
    auto issue_window = [&](int st) {
        const char *sbase = ring + (size_t)st * stage_bytes;
        const int *hdr = reinterpret_cast<const int *>(sbase);
        const int *rec = reinterpret_cast<const int *>(sbase + kStageOffs);  // written by issue()
        const int nruns = rec[0], entries = rec[1];
        const int tile_nnz = hdr[kTileSlices] - hdr[0];
        char *wdst = const_cast<char *>(sbase) + kStageHdr + (size_t)tile_nnz * (kIdxBytes + sizeof(TA)) +
                     (size_t)ex.count * kTileRows * ex.esize;
        // lane r owns run r: its first column, length and place in the window
        int c0 = 0, len = 0, pos = 0;
        if (lane < nruns) {
            c0 = rec[kWinRecRun + 3 * lane];
            len = rec[kWinRecRun + 3 * lane + 1];
            pos = rec[kWinRecRun + 3 * lane + 2];
        }
        const uint32_t bar = smem_u32(full + st);
        if (lane == 0)  // the zero slot padding entries read
            *reinterpret_cast<uint4 *>(wdst + (size_t)entries * wn.xsize) = make_uint4(0u, 0u, 0u, 0u);
        uint32_t bytes;
        if (rec[kWinRecClamp] == 0) {  // every run lies inside x: whole runs, known total
            bytes = (uint32_t)len * (uint32_t)wn.xsize;
            __syncwarp();  // the zero slot before lane 0's arrive (release)
            if (lane == 0) mbar_expect_tx(bar, (uint32_t)entries * (uint32_t)wn.xsize);
        } else {
            // runs cut at the end of x: the part of a run inside x that ends on a
            // 16-byte boundary in bulk, the rest entry by entry
            const int have = max(0, min(len, wn.n - c0));
            const int per16 = 16 / wn.xsize;
            int bulk = have;
            if (c0 + have == wn.n) bulk = have / per16 * per16;
            for (int e = bulk; e < have; ++e) {
                const char *src = (const char *)wn.x + (size_t)(c0 + e) * wn.xsize;
                char *d = wdst + (size_t)(pos + e) * wn.xsize;
                if (wn.xsize == 2) *reinterpret_cast<uint16_t *>(d) = *reinterpret_cast<const uint16_t *>(src);
                else if (wn.xsize == 4) *reinterpret_cast<uint32_t *>(d) = *reinterpret_cast<const uint32_t *>(src);
                else *reinterpret_cast<uint64_t *>(d) = *reinterpret_cast<const uint64_t *>(src);
            }
            bytes = (uint32_t)bulk * (uint32_t)wn.xsize;
            uint32_t total = bytes;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
            __syncwarp();  // the entry-by-entry copies before lane 0's arrive (release)
            if (lane == 0) mbar_expect_tx(bar, total);
        }
        __syncwarp();  // the expected bytes raised before any run's copy can complete
        if (bytes) {
            fence_proxy_async();
            bulk_g2s(smem_u32(wdst + (size_t)pos * wn.xsize), (const char *)wn.x + (size_t)c0 * wn.xsize, bytes, bar);
        }
    };
    if (threadIdx.x == 0) {
        for (int st = 0; st < S; ++st) {
            mbar_init(smem_u32(full + st), 1);
            mbar_init(smem_u32(empty + st), kWarps);
        }
        fence_mbar_init();
    }
    __syncthreads();
    bool ok = true;
    if (producer) {
        fence_proxy_async_all();  // the basis rows an earlier kernel wrote, before the first bulk copy
        int k = 0;
        const int pre = min(S, max(0, tile_end - tile_begin));
        prefetch(tile_begin);
        for (; k < pre; ++k) {
            issue(tile_begin + k, k, !WIN);
            __syncwarp();
        }
        if (!gate()) {
            if constexpr (WIN)  // complete the phases the matrix copies were issued under
                if (lane == 0)
                    for (int kk = 0; kk < pre; ++kk) mbar_arrive(smem_u32(full + kk));
            for (int kk = 0; kk < pre; ++kk) mbar_wait(smem_u32(full + kk), 0u);
            return false;
        }
        if constexpr (WIN) {
            fence_proxy_async_all();  // x, written by the grid the gate waited for, before its bulk copies
            for (int kk = 0; kk < pre; ++kk) {
                issue_window(kk);
                __syncwarp();
            }
        }
        for (int t = tile_begin + k; t < tile_end; ++t, ++k) {
            const int st = k % S;
            if (k >= S && !mbar_wait(smem_u32(empty + st), (uint32_t)(((k / S) - 1) & 1))) {
                ok = false;
                break;
            }
            issue(t, st, !WIN);
            __syncwarp();
            if constexpr (WIN) {
                issue_window(st);
                __syncwarp();
            }
        }
        // wait for the copies of the last (up to S) tiles issued, so none lands after exit
        const int issued = k;
        for (int kk = max(0, issued - S); kk < issued; ++kk)
            mbar_wait(smem_u32(full + kk % S), (uint32_t)((kk / S) & 1));
        if (!ok && lane == 0) atomicOr(err, ERR_STAGE_TIMEOUT);
    } else {
        if (!gate()) return false;
        int k = 0;
        for (int t = tile_begin; t < tile_end; ++t, ++k) {
            const int st = k % S;
            if (!mbar_wait(smem_u32(full + st), (uint32_t)((k / S) & 1))) {
                ok = false;
                if (lane == 0) atomicOr(err, ERR_STAGE_TIMEOUT);
                break;
            }
            const char *base = ring + (size_t)st * stage_bytes;
            const int *hdr = reinterpret_cast<const int *>(base);
            const int bt = hdr[0];
            const int tile_nnz = hdr[kTileSlices] - bt;
            const char *body_base = base + kStageHdr;
            StageView<TA> v;
            v.extra = body_base + (size_t)tile_nnz * (kIdxBytes + sizeof(TA));
            v.win = v.extra + (size_t)ex.count * kTileRows * ex.esize;
            if constexpr (WIN) v.own = reinterpret_cast<const int *>(base + kStageOffs)[kWinRecOwn];
            else v.own = 0;
            v.esize = ex.esize;
#pragma unroll
            for (int sl = warp; sl < kTileSlices; sl += kWarps) {
                const int s = t * kTileSlices + sl;
                if (s < A.nslices) {
                    const int b0 = hdr[sl], b1 = hdr[sl + 1];
                    v.w = (b1 - b0) >> 5;
                    v.col = reinterpret_cast<const int *>(body_base) + (b0 - bt);
                    v.lcol = reinterpret_cast<const uint16_t *>(body_base) + (b0 - bt);
                    v.val = reinterpret_cast<const TA *>(body_base + (size_t)tile_nnz * kIdxBytes) + (b0 - bt);
                    v.row0 = sl * kSlice;
                    body(s, v);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(empty + st));
        }
    }
    return ok;
}

// staged_tiles_gated without a gate (the caller waited already)
template <class TA, int S, bool EVICT_FIRST = false, bool WIN = false, class Body>
__device__ __forceinline__ bool staged_tiles(const Sell &A, const TA *__restrict__ val, int tile_begin,
                                             int tile_end, char *ring, int stage_bytes, uint64_t *full,
                                             uint64_t *empty, Extra ex, int *err, Body body,
                                             Window wn = Window()) {
    return staged_tiles_gated<TA, S, EVICT_FIRST, WIN>(A, val, tile_begin, tile_end, ring, stage_bytes, full, empty,
                                                       ex, err, body, [] { return true; }, wn);
}

// stage size in bytes for tiles of slices up to wmax wide; win_entries > 0:
// windowed tiles (2-byte indices) with x windows of up to that many entries
// of xsize bytes
__host__ __device__ inline int stage_bytes_for(int wmax, int asize, int n_extra, int esize, int win_entries = 0,
                                               int xsize = 0) {
    const int isz = win_entries > 0 ? 2 : 4;
    const int b = kStageHdr + kTileSlices * wmax * kSlice * (isz + asize) + n_extra * kTileRows * esize +
                  (win_entries > 0 ? win_entries * xsize + kWinPadBytes : 0);
    return (b + 15) / 16 * 16;
}

}  // namespace f3r
