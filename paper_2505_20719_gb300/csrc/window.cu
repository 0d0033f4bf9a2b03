// Set-up of windowed tiles (stage.cuh): for every tile of 256 rows, the runs
// of x its columns (and its own rows) fall in and each entry's index into
// their concatenation.
//
// One block per tile (grid-stride): the block finds the tile's smallest and
// largest column, marks the kWinChunk-entry chunks its columns and its own
// rows touch in a shared-memory bitmap, counts chunks and run starts / ends
// per bitmap word, scans those counts, writes the tile's record (runs in
// column order, the window position of its first row) and rewrites each
// entry's column c as slot(c / kWinChunk) * kWinChunk + c % kWinChunk, slot =
// the chunk's rank among the marked ones; padding entries get the index just
// past the window (the zero slot the kernels keep there).  A tile whose
// columns span more than kWinSpanChunks chunks, or that needs more than
// kWinRuns runs or kWinMaxEntries window entries, marks the matrix as not
// windowed (the kernels then gather x by int32 column from global memory).
#include <algorithm>
#include <climits>
#include <cstdlib>

#include "ctx.h"
#include "stage.cuh"

namespace f3r {

constexpr int kWinSpanWords = 1024;                  // bitmap words per tile
constexpr int kWinSpanChunks = kWinSpanWords * 32;   // 32768 chunks: columns within 1 M of each other
constexpr int kWinThreads = 256;
constexpr int kWinWordsPerThread = kWinSpanWords / kWinThreads;

// exclusive block scan of one int per thread (kWinThreads threads); returns
// the prefix, *total the sum
__device__ __forceinline__ int block_excl_scan(int v, int *sm /* 32 */, int *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sm[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = (lane < kWinThreads / 32) ? sm[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kWinThreads / 32) sm[lane] = w;  // inclusive per-warp totals
    }
    __syncthreads();
    const int before = (warp > 0 ? sm[warp - 1] : 0) + x - v;
    *total = sm[kWinThreads / 32 - 1];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(kWinThreads) k_tile_window(const int *__restrict__ sptr, const int *__restrict__ col,
                                                             int n, int nslices, int ntiles, uint16_t *lcol,
                                                             int *rec, int *fail, int *maxwin) {
    __shared__ uint32_t bits[kWinSpanWords];
    __shared__ int slot0[kWinSpanWords];   // marked chunks before each word
    __shared__ int start0[kWinSpanWords];  // run starts before each word
    __shared__ int end0[kWinSpanWords];    // run ends before each word
    __shared__ int sm[32];
    __shared__ int red_min[kWinThreads / 32], red_max[kWinThreads / 32];
    __shared__ int runs_c0[kWinRuns], runs_c1[kWinRuns];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int s0 = t * kTileSlices, s1 = min(s0 + kTileSlices, nslices);
        const int e0 = sptr[s0], e1 = sptr[s1];
        const int r0 = t * kTileRows, r1 = min(r0 + kTileRows, n);  // the tile's own rows
        int mn = r0, mx = r1 - 1;
        for (int k = e0 + tid; k < e1; k += kWinThreads) {
            const int c = col[k];
            if (c >= 0) {
                mn = min(mn, c);
                mx = max(mx, c);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if (lane == 0) {
            red_min[warp] = mn;
            red_max[warp] = mx;
        }
        __syncthreads();
        mn = INT_MAX;
        mx = -1;
        for (int w = 0; w < kWinThreads / 32; ++w) {
            mn = min(mn, red_min[w]);
            mx = max(mx, red_max[w]);
        }
        __syncthreads();
        int *r = rec + (size_t)t * kWinRec;
        const int base = mn / kWinChunk;
        const int span = mx / kWinChunk - base + 1;
        if (span > kWinSpanChunks) {
            if (tid == 0) atomicOr(fail, 1);
            continue;
        }
        const int nw = (span + 31) / 32;
        for (int w = tid; w < nw; w += kWinThreads) bits[w] = 0u;
        __syncthreads();
        for (int k = e0 + tid; k < e1; k += kWinThreads) {
            const int c = col[k];
            if (c >= 0) {
                const int q = c / kWinChunk - base;
                atomicOr(&bits[q >> 5], 1u << (q & 31));
            }
        }
        for (int c = r0 + tid * kWinChunk; c < r1; c += kWinThreads * kWinChunk) {
            const int q = c / kWinChunk - base;
            atomicOr(&bits[q >> 5], 1u << (q & 31));
        }
        __syncthreads();
        // per thread: words [4 tid, 4 tid + 4): marked chunks, run starts (a
        // marked chunk after an unmarked one) and run ends (before an unmarked one)
        int cnt_c[kWinWordsPerThread], cnt_s[kWinWordsPerThread], cnt_e[kWinWordsPerThread];
        int tc = 0, ts = 0, te = 0;
#pragma unroll
        for (int q = 0; q < kWinWordsPerThread; ++q) {
            const int w = tid * kWinWordsPerThread + q;
            uint32_t b = 0, st = 0, en = 0;
            if (w < nw) {
                b = bits[w];
                const uint32_t prev_hi = (w > 0) ? (bits[w - 1] >> 31) : 0u;
                const uint32_t next_lo = (w + 1 < nw) ? (bits[w + 1] & 1u) : 0u;
                st = b & ~((b << 1) | prev_hi);
                en = b & ~((b >> 1) | (next_lo << 31));
            }
            cnt_c[q] = __popc(b);
            cnt_s[q] = __popc(st);
            cnt_e[q] = __popc(en);
            tc += cnt_c[q];
            ts += cnt_s[q];
            te += cnt_e[q];
        }
        int chunks, nruns, nends;
        int pc = block_excl_scan(tc, sm, &chunks);
        int ps = block_excl_scan(ts, sm, &nruns);
        int pe = block_excl_scan(te, sm, &nends);
#pragma unroll
        for (int q = 0; q < kWinWordsPerThread; ++q) {
            const int w = tid * kWinWordsPerThread + q;
            if (w < kWinSpanWords) {
                slot0[w] = pc;
                start0[w] = ps;
                end0[w] = pe;
            }
            pc += cnt_c[q];
            ps += cnt_s[q];
            pe += cnt_e[q];
        }
        __syncthreads();
        const int entries = chunks * kWinChunk;
        if (nruns > kWinRuns || nruns != nends || entries > kWinMaxEntries) {
            if (tid == 0) atomicOr(fail, 2);
            continue;
        }
        // run r: its first chunk is the r-th start bit, its last the r-th end bit
        for (int w = tid; w < nw; w += kWinThreads) {
            const uint32_t b = bits[w];
            const uint32_t prev_hi = (w > 0) ? (bits[w - 1] >> 31) : 0u;
            const uint32_t next_lo = (w + 1 < nw) ? (bits[w + 1] & 1u) : 0u;
            uint32_t st = b & ~((b << 1) | prev_hi);
            uint32_t en = b & ~((b >> 1) | (next_lo << 31));
            int rs = start0[w], re = end0[w];
            while (st) {
                const int bit = __ffs(st) - 1;
                runs_c0[rs++] = base + w * 32 + bit;
                st &= st - 1;
            }
            while (en) {
                const int bit = __ffs(en) - 1;
                runs_c1[re++] = base + w * 32 + bit;
                en &= en - 1;
            }
        }
        __syncthreads();
        if (tid == 0) {
            int pos = 0, clamp = 0;
            for (int q = 0; q < nruns; ++q) {
                const int c0 = runs_c0[q] * kWinChunk, len = (runs_c1[q] - runs_c0[q] + 1) * kWinChunk;
                r[kWinRecRun + 3 * q] = c0;
                r[kWinRecRun + 3 * q + 1] = len;
                r[kWinRecRun + 3 * q + 2] = pos;
                pos += len;
                if (c0 + len > n) clamp = 1;
            }
            for (int q = kWinRecRun + 3 * nruns; q < kWinRec; ++q) r[q] = 0;
            r[0] = nruns;
            r[1] = entries;
            r[kWinRecClamp] = clamp;
            atomicMax(maxwin, entries);
        }
        auto index_of = [&](int c) {
            const int q = c / kWinChunk - base;
            const uint32_t b = bits[q >> 5];
            const int slot = slot0[q >> 5] + __popc(b & ((1u << (q & 31)) - 1u));
            return slot * kWinChunk + c % kWinChunk;
        };
        __syncthreads();  // the record's other words before its own-row word
        if (tid == 0) r[kWinRecOwn] = index_of(r0);
        for (int k = e0 + tid; k < e1; k += kWinThreads) {
            const int c = col[k];
            lcol[k] = (uint16_t)(c >= 0 ? index_of(c) : entries);  // padding: the zero slot
        }
        __syncthreads();
    }
}

static void *walloc(Ctx &c, size_t bytes) {
    void *p = pool_alloc(c.dev, bytes ? bytes : 16, c.zstream);
    if (!p) return nullptr;
    c.allocs.push_back(p);
    c.bytes += (long long)bytes;
    return p;
}

f3r_status build_window(Ctx &c, cudaStream_t s) {
    c.win = false;
    c.win_max = 0;
    static const bool off = [] {
        const char *e = getenv("F3R_WINDOW");  // 0: gather x from global memory by int32 column
        return e && e[0] == '0';
    }();
    if (off || !c.staged || c.nslices == 0) return F3R_OK;
    const int ntiles = ceil_div(c.nslices, kTileSlices);
    c.lcol = (uint16_t *)walloc(c, sizeof(uint16_t) * (size_t)c.nsell);
    c.wrec = (int *)walloc(c, sizeof(int) * (size_t)ntiles * kWinRec);
    int *flags = (int *)walloc(c, 2 * sizeof(int));
    if (!c.lcol || !c.wrec || !flags) return F3R_ERR_NOMEM;
    cudaMemsetAsync(flags, 0, 2 * sizeof(int), s);
    const int g = std::max(1, std::min(ntiles, c.nsm * 4));
    k_tile_window<<<g, kWinThreads, 0, s>>>(c.sptr, c.col, c.n, c.nslices, ntiles, c.lcol, c.wrec, flags, flags + 1);
    int h[2] = {1, 0};
    cudaMemcpyAsync(h, flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return F3R_ERR_CUDA;
    c.win = (h[0] == 0);
    c.win_max = c.win ? h[1] : 0;
    return F3R_OK;
}

Window window_of(const Ctx &c, int xsize, int n) {
    Window w;
    if (!c.win) return w;
    w.lcol = c.lcol;
    w.rec = c.wrec;
    w.xsize = xsize;
    w.n = n;
    return w;
}

}  // namespace f3r
