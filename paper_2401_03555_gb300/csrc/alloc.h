// alloc.h -- the library's allocation wrappers (alloc.cu): tracked, and able
// to fail on request (impact_debug_fail_alloc); internal.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace impact {

cudaError_t dev_malloc_async(void **p, size_t bytes, cudaStream_t st);
cudaError_t dev_free_async(void *p, cudaStream_t st);
cudaError_t dev_malloc(void **p, size_t bytes);
cudaError_t dev_free(void *p);
cudaError_t host_malloc(void **p, size_t bytes);
cudaError_t host_free(void *p);

template <typename T>
cudaError_t dev_malloc_async(T **p, size_t bytes, cudaStream_t st)
{
    return dev_malloc_async(reinterpret_cast<void **>(p), bytes, st);
}
template <typename T>
cudaError_t dev_malloc(T **p, size_t bytes)
{
    return dev_malloc(reinterpret_cast<void **>(p), bytes);
}
template <typename T>
cudaError_t host_malloc(T **p, size_t bytes)
{
    return host_malloc(reinterpret_cast<void **>(p), bytes);
}

}  // namespace impact
