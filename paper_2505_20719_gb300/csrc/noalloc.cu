// Allocation-free residual entry point.
//
// f3r_residual_noalloc computes r = b - A x and the norms ||r||_2, ||b||_2
// for a caller-supplied fp64 CSR matrix.  It is a variant of the outer-level
// residual kernel for callers that must not allocate device memory: its only
// scratch (one pair of partial sums per block and the ticket that elects the
// block finishing the reduction) lives in the file-scope array below, which
// every GPU that loads this library keeps until the process exits.
#include <cuda.h>  // CUcontext and the driver call's signature only; libcuda is reached through the runtime

#include <mutex>

#include "common.cuh"

namespace {

constexpr int kNaBlock = 256;                              // threads per block
constexpr int kNaRowsPerThread = 4;
constexpr int kNaRowsPerBlock = kNaBlock * kNaRowsPerThread;  // 1024 rows per block
constexpr int kNaMaxBlocks = 4096;                          // => n <= 4,194,304
constexpr int kNaTicketBytes = 256;
constexpr size_t kNaScratchBytes = kNaTicketBytes + (size_t)kNaMaxBlocks * 2 * sizeof(double);  // 65,792 B
constexpr int kNaMaxDevices = 64;

// [0, 256): election ticket (must be zero when a call starts)
// [256, ...): per-block partial sums (||r||^2, ||b||^2)
static __device__ __align__(256) unsigned char g_na_scratch[kNaScratchBytes];

__global__ void __launch_bounds__(kNaBlock) k_residual_noalloc(int n, const int *__restrict__ rp,
                                                               const int *__restrict__ ci,
                                                               const double *__restrict__ val,
                                                               const double *__restrict__ b,
                                                               const double *__restrict__ x, double *r,
                                                               double *norms, unsigned char *scratch) {
    unsigned *ticket = reinterpret_cast<unsigned *>(scratch);
    double *part = reinterpret_cast<double *>(scratch + kNaTicketBytes);
    __shared__ double sm[2][kNaBlock / 32];
    __shared__ bool am_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double sr = 0.0, sb = 0.0;
    const int base = blockIdx.x * kNaRowsPerBlock;
    for (int q = 0; q < kNaRowsPerThread; ++q) {
        const int i = base + q * kNaBlock + threadIdx.x;
        if (i < n) {
            double s = 0.0;  // row sum in CSR order with fused multiply-add
            for (int k = rp[i]; k < rp[i + 1]; ++k) s = f3r::fma_rn(val[k], x[ci[k]], s);
            const double bi = b[i];
            const double ri = f3r::sub_rn(bi, s);
            r[i] = ri;
            sr = f3r::fma_rn(ri, ri, sr);
            sb = f3r::fma_rn(bi, bi, sb);
        }
    }
    sr = f3r::warp_sum(sr);
    sb = f3r::warp_sum(sb);
    if (lane == 0) {
        sm[0][warp] = sr;
        sm[1][warp] = sb;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double s = sm[threadIdx.x][0];
        for (int w = 1; w < kNaBlock / 32; ++w) s = f3r::add_rn(s, sm[threadIdx.x][w]);
        part[2 * blockIdx.x + threadIdx.x] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) am_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    // the last block sums all partials in a fixed order
    sr = 0.0;
    sb = 0.0;
    for (int blk = threadIdx.x; blk < (int)gridDim.x; blk += kNaBlock) {
        sr = f3r::add_rn(sr, __ldcg(part + 2 * blk));
        sb = f3r::add_rn(sb, __ldcg(part + 2 * blk + 1));
    }
    __syncthreads();
    sr = f3r::warp_sum(sr);
    sb = f3r::warp_sum(sb);
    if (lane == 0) {
        sm[0][warp] = sr;
        sm[1][warp] = sb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = sm[0][0], c = sm[1][0];
        for (int w = 1; w < kNaBlock / 32; ++w) {
            a = f3r::add_rn(a, sm[0][w]);
            c = f3r::add_rn(c, sm[1][w]);
        }
        norms[0] = f3r::sqrt_rn(a);
        norms[1] = f3r::sqrt_rn(c);
        *ticket = 0u;
    }
}

std::mutex g_na_mutex;
// per device: the scratch array's address in the context it was looked up in
unsigned char *g_na_addr[kNaMaxDevices] = {};
CUcontext g_na_ctx[kNaMaxDevices] = {};

}  // namespace

extern "C" f3r_status f3r_residual_noalloc(int32_t n, const int32_t *rowptr, const int32_t *colidx,
                                           const double *val, const double *b, const double *x, double *r,
                                           double *norms, void *stream) {
    if (n <= 0) return F3R_ERR_ARG;
    if ((long long)n > (long long)kNaMaxBlocks * kNaRowsPerBlock) return F3R_ERR_ARG;  // beyond the scratch
    if (!rowptr || !colidx || !val || !b || !x || !r || !norms) return F3R_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) {
        cudaGetLastError();
        return F3R_ERR_CUDA;
    }
    unsigned char *scratch = nullptr;
    {
        // The array's name is only a host-side stand-in; its device address is
        // looked up once per device and context, with that device current (a
        // cudaDeviceReset ends the context, and the next call looks it up in
        // the new one).
        std::lock_guard<std::mutex> lock(g_na_mutex);
        static CUresult (*ctx_current)(CUcontext *) = nullptr;
        if (!ctx_current) {
            cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
            void *fn = nullptr;
            if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) !=
                    cudaSuccess ||
                q != cudaDriverEntryPointSuccess || !fn) {
                cudaGetLastError();
                return F3R_ERR_CUDA;
            }
            ctx_current = reinterpret_cast<CUresult (*)(CUcontext *)>(fn);
        }
        CUcontext ctx = nullptr;
        if (cudaFree(nullptr) != cudaSuccess || ctx_current(&ctx) != CUDA_SUCCESS || !ctx) {
            cudaGetLastError();
            return F3R_ERR_CUDA;
        }
        if (!g_na_addr[dev] || g_na_ctx[dev] != ctx) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return F3R_ERR_CUDA;
            }
            g_na_addr[dev] = (unsigned char *)p;
            g_na_ctx[dev] = ctx;
        }
        scratch = g_na_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    // the ticket must start at zero (a previous call may have been cut short)
    if (cudaMemsetAsync(scratch, 0, kNaTicketBytes, s) != cudaSuccess) {
        cudaGetLastError();
        return F3R_ERR_CUDA;
    }
    const int grid = (n + kNaRowsPerBlock - 1) / kNaRowsPerBlock;
    k_residual_noalloc<<<grid, kNaBlock, 0, s>>>(n, rowptr, colidx, val, b, x, r, norms, scratch);
    return cudaGetLastError() == cudaSuccess ? F3R_OK : F3R_ERR_CUDA;
}
