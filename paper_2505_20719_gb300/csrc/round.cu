// Stand-alone 16-bit rounding (test entry): the fp32 -> fp16 / bf16
// conversions every kernel of the library uses when it stores a 16-bit value
// (Store<h16>, Store<b16>: round to nearest, ties to even, subnormals kept,
// overflow to infinity), applied to an array so that tests can compare them
// with an independent definition over every fp32 bit pattern.
#include <algorithm>

#include "f3r.h"
#include "common.cuh"

namespace f3r {

template <class S>
__global__ void __launch_bounds__(kBlock) k_round16(const float *__restrict__ x, uint16_t *__restrict__ out,
                                                     long long n) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const S h = Store<S>::from(x[i]);
        out[i] = *reinterpret_cast<const uint16_t *>(&h);
    }
}

}  // namespace f3r

extern "C" f3r_status f3r_round16(int prec, const float *x, uint16_t *out, int64_t n, void *stream) {
    using namespace f3r;
    if ((prec != F3R_F16 && prec != F3R_BF16) || n < 0 || (n > 0 && (!x || !out))) return F3R_ERR_ARG;
    if (n == 0) return F3R_OK;
    int dev = 0, nsm = 1;
    if (cudaGetDevice(&dev) != cudaSuccess) return F3R_ERR_CUDA;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long blocks = std::min<long long>((n + kBlock - 1) / kBlock, (long long)nsm * 16);
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == F3R_F16)
        k_round16<h16><<<(unsigned)blocks, kBlock, 0, s>>>(x, out, (long long)n);
    else
        k_round16<b16><<<(unsigned)blocks, kBlock, 0, s>>>(x, out, (long long)n);
    return cudaGetLastError() == cudaSuccess ? F3R_OK : F3R_ERR_CUDA;
}
