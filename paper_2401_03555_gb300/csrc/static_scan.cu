// static_scan.cu -- the row-pointer scan for callers that cannot allocate.
//
// impact_scan_rows_static turns per-row pair counts into CSR row pointers in
// place, like the scan of the FP64-plain count pass, but its scratch (one partial sum
// per tile of rows) lives in a fixed file-scope device array instead of
// memory allocated per call. Nothing here calls cudaMalloc, cudaFree or any
// allocating library routine.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "../../include/impact.h"
#include "kernels.h"

namespace {

// One int64 per tile of 4096 rows (the scan's tile), plus the total.
constexpr int64_t kStaticTiles = IMPACT_SCAN_STATIC_MAX_ROWS / 4096;
static __device__ __align__(256) int64_t g_tile_sums[kStaticTiles + 1];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
int64_t *g_dev_ptr[kMaxDevices] = {};

impact_status fail(impact_status s, const std::string &m)
{
    impact::set_last_error(m);
    return s;
}

}  // namespace

extern "C" impact_status impact_scan_rows_static(int64_t *row_ptr, int64_t rows, void *stream)
{
    if (rows < 1 || rows > IMPACT_SCAN_STATIC_MAX_ROWS)
        return fail(IMPACT_ERR_ARG, "rows must be in [1, " +
                                        std::to_string((long long)IMPACT_SCAN_STATIC_MAX_ROWS) +
                                        "] for the allocation-free scan");
    if (!row_ptr) return fail(IMPACT_ERR_ARG, "null row_ptr");
    {   // a host or stale pointer would reach the kernels: refuse it
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, row_ptr) != cudaSuccess) {
            cudaGetLastError();
            return fail(IMPACT_ERR_ARG, "row_ptr must be a device array");
        }
        if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
            return fail(IMPACT_ERR_ARG, "row_ptr must be a device array");
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(IMPACT_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(IMPACT_ERR_ARG, "device index too large");
    int64_t *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_dev_ptr[dev]) {
            // In host code g_tile_sums names a host-side stand-in, not device
            // memory: the device address must be looked up, once per device,
            // with that device current.
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_tile_sums);
            if (e != cudaSuccess)
                return fail(IMPACT_ERR_CUDA, std::string("cudaGetSymbolAddress: ") +
                                                 cudaGetErrorString(e));
            g_dev_ptr[dev] = (int64_t *)p;
        }
        scratch = g_dev_ptr[dev];
    }
    // Every tile sum is written before it is read, so the array needs no
    // clearing between calls.
    e = impact::launch_scan(row_ptr, rows, scratch, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(IMPACT_ERR_CUDA, cudaGetErrorString(e));
    return IMPACT_OK;
}
