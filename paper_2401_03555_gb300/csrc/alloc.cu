// alloc.cu -- every device and pinned-host allocation the library makes goes
// through these wrappers. They keep a count of the live bytes per kind (so a
// test can see that a failed call released everything it took) and can make
// the n-th allocation from now fail as if the device were out of memory (so
// a test can drive every entry point through its out-of-memory path on the
// host, without exhausting or faulting a GPU).
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <unordered_map>

#include "../../include/impact.h"
#include "alloc.h"

namespace {

std::atomic<int64_t> g_countdown{0};   // > 0: the allocation that brings it to 0 fails
std::mutex g_mu;
std::unordered_map<void *, std::pair<size_t, bool>> g_live;   // pointer -> (bytes, host)
int64_t g_dev_bytes = 0, g_host_bytes = 0;

bool injected_failure()
{
    int64_t c = g_countdown.load();
    while (c > 0) {
        if (g_countdown.compare_exchange_weak(c, c - 1)) return c == 1;
    }
    return false;
}

void track(void *p, size_t bytes, bool host)
{
    if (!p) return;
    std::lock_guard<std::mutex> lock(g_mu);
    g_live[p] = {bytes, host};
    (host ? g_host_bytes : g_dev_bytes) += (int64_t)bytes;
}

void untrack(void *p)
{
    if (!p) return;
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_live.find(p);
    if (it == g_live.end()) return;
    (it->second.second ? g_host_bytes : g_dev_bytes) -= (int64_t)it->second.first;
    g_live.erase(it);
}

}  // namespace

namespace impact {

cudaError_t dev_malloc_async(void **p, size_t bytes, cudaStream_t st)
{
    *p = nullptr;
    if (injected_failure()) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMallocAsync(p, bytes, st);
    if (e == cudaSuccess) track(*p, bytes, false);
    else *p = nullptr;
    return e;
}

cudaError_t dev_free_async(void *p, cudaStream_t st)
{
    if (!p) return cudaSuccess;
    untrack(p);
    return cudaFreeAsync(p, st);
}

cudaError_t dev_malloc(void **p, size_t bytes)
{
    *p = nullptr;
    if (injected_failure()) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) track(*p, bytes, false);
    else *p = nullptr;
    return e;
}

cudaError_t dev_free(void *p)
{
    if (!p) return cudaSuccess;
    untrack(p);
    return cudaFree(p);
}

cudaError_t host_malloc(void **p, size_t bytes)
{
    *p = nullptr;
    if (injected_failure()) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMallocHost(p, bytes);
    if (e == cudaSuccess) track(*p, bytes, true);
    else *p = nullptr;
    return e;
}

cudaError_t host_free(void *p)
{
    if (!p) return cudaSuccess;
    untrack(p);
    return cudaFreeHost(p);
}

}  // namespace impact

extern "C" {

impact_status impact_debug_fail_alloc(int64_t n)
{
    if (n < 0) return IMPACT_ERR_ARG;
    g_countdown.store(n);
    return IMPACT_OK;
}

impact_status impact_debug_live_bytes(int64_t *device_bytes, int64_t *host_bytes)
{
    std::lock_guard<std::mutex> lock(g_mu);
    if (device_bytes) *device_bytes = g_dev_bytes;
    if (host_bytes) *host_bytes = g_host_bytes;
    return IMPACT_OK;
}

}  // extern "C"
