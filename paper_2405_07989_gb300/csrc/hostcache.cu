// Host-side caches of launch attributes: occupancy, the dynamic shared-memory
// opt-in of a kernel and the SM count are asked of the runtime once per
// device (and kernel / shape) instead of on every call, which keeps the host
// ahead of the GPU when a call's kernels are short.
#include <cuda_runtime.h>

#include <map>
#include <atomic>
#include <mutex>
#include <tuple>

#include "launch.h"

namespace fsi {

namespace {
std::mutex g_cache_mu;
std::map<std::tuple<int, const void*, int, int>, int> g_occ;
std::map<std::pair<int, const void*>, int> g_optin;
std::map<int, int> g_sms;
}  // namespace

// The opt-in covers the kernel's static shared memory too: static + dynamic
// above 48 KB needs it even when the dynamic part alone is below, so every
// nonzero dynamic size is declared (once per device, kernel and larger size).
cudaError_t smem_optin(const void* kern, int smem)
{
    if (smem <= 0) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_cache_mu);
    int& have = g_optin[{dev, kern}];
    if (have >= smem) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) have = smem;
    return e;
}

cudaError_t occupancy_cached(const void* kern, int threads, int smem, int* nb)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = smem_optin(kern, smem);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_cache_mu);
    const auto key = std::make_tuple(dev, kern, threads, smem);
    auto it = g_occ.find(key);
    if (it != g_occ.end()) {
        *nb = it->second;
        return cudaSuccess;
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, kern, threads, smem);
    if (e == cudaSuccess) g_occ[key] = *nb;
    return e;
}

cudaError_t sm_count_cached(int* sms)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto it = g_sms.find(dev);
    if (it != g_sms.end()) {
        *sms = it->second;
        return cudaSuccess;
    }
    e = cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) g_sms[dev] = *sms;
    return e;
}

// Allocation counters (fs_alloc_counts).
static std::atomic<uint64_t> g_dev_allocs{0}, g_host_allocs{0};

cudaError_t dev_alloc(void** p, size_t bytes)
{
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) g_dev_allocs.fetch_add(1, std::memory_order_relaxed);
    return e;
}

cudaError_t host_alloc(void** p, size_t bytes)
{
    const cudaError_t e = cudaMallocHost(p, bytes);
    if (e == cudaSuccess) g_host_allocs.fetch_add(1, std::memory_order_relaxed);
    return e;
}

}  // namespace fsi

extern "C" void fs_alloc_counts(uint64_t* device_allocs, uint64_t* pinned_host_allocs)
{
    if (device_allocs) *device_allocs = fsi::g_dev_allocs.load(std::memory_order_relaxed);
    if (pinned_host_allocs) *pinned_host_allocs = fsi::g_host_allocs.load(std::memory_order_relaxed);
}
