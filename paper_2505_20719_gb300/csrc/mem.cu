// Device memory of the solver contexts: stream-ordered allocations from one
// memory pool per device that keeps the blocks given back to it (release
// threshold at the maximum).  A process that sets up and destroys contexts
// repeatedly then reuses device memory without a cudaMalloc / cudaFree (and
// the device-wide synchronisation of cudaFree) per buffer.  f3r_trim_memory
// returns the unused blocks to the CUDA driver.
#include <cstdint>
#include <map>
#include <mutex>
#include <utility>

#include "ctx.h"

namespace f3r {

namespace {
std::mutex g_pool_mu;
std::map<int, cudaMemPool_t> g_pools;

cudaMemPool_t pool_of(int dev) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(dev);
    if (it != g_pools.end()) return it->second;
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools[dev] = pool;
    return pool;
}
}  // namespace

void *pool_alloc(int dev, size_t bytes, cudaStream_t s) {
    cudaMemPool_t pool = pool_of(dev);
    if (!pool) return nullptr;
    void *p = nullptr;
    if (cudaMallocFromPoolAsync(&p, bytes ? bytes : 16, pool, s) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void pool_free(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

namespace {
std::mutex g_smem_mu;
std::map<std::pair<int, const void *>, int> g_smem;  // limit set per (device, kernel)
}  // namespace

bool ensure_dyn_smem(const void *kern, int bytes) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    std::lock_guard<std::mutex> lk(g_smem_mu);
    int &cur = g_smem[std::make_pair(dev, kern)];
    if (bytes <= cur) return true;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cur = bytes;
    return true;
}

}  // namespace f3r

extern "C" f3r_status f3r_trim_memory(void) {
    std::lock_guard<std::mutex> lk(f3r::g_pool_mu);
    for (auto &kv : f3r::g_pools)
        if (cudaMemPoolTrimTo(kv.second, 0) != cudaSuccess) return F3R_ERR_CUDA;
    return F3R_OK;
}
