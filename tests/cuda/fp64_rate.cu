// Throughput of FP64 fused multiply-adds (and, for scale, FP32 ones) on the
// device: many threads, eight independent chains each, no memory traffic in
// the timed loop. Host entry: fp_rate(&fp64_flops, &fp32_flops), FLOP/s.
#include <cuda_runtime.h>

template <typename T>
__global__ void fma_chains(T *out, int iters, T a, T b)
{
    T x0 = (T)threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
    T x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
        x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
        x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
    }
    // keeps the chains live; the sum is never non-zero for the a, b used
    if (x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7 == (T)-1.2345) out[blockIdx.x] = x0;
}

template <typename T>
static double rate(int iters)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8, threads = 256;
    T *out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * blocks) != cudaSuccess) return -1.0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    fma_chains<T><<<blocks, threads>>>(out, iters / 10, (T)0.999, (T)0.001);   // warm-up
    cudaEventRecord(e0);
    fma_chains<T><<<blocks, threads>>>(out, iters, (T)0.999, (T)0.001);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (cudaGetLastError() != cudaSuccess || ms <= 0.0f) return -1.0;
    return 2.0 * 8.0 * (double)iters * blocks * threads / (ms * 1e-3);
}

extern "C" int fp_rate(double *fp64, double *fp32)
{
    *fp64 = rate<double>(20000);
    *fp32 = rate<float>(200000);
    return (*fp64 > 0.0 && *fp32 > 0.0) ? 0 : 1;
}
