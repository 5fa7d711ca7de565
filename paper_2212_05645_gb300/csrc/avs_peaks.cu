// FMA throughput of this GPU in FP32 and FP64, measured with independent
// multiply-add chains per thread (used as the ALU roofline of the step
// kernels; the paper has no counterpart).
#include <cuda_runtime.h>

#include "avs_internal.h"

namespace {

template <typename T>
__global__ void k_fma(int iters, T seed, T* out)
{
    T a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = seed + (T)(threadIdx.x + j);
    const T m = (T)0.999999, c = (T)1e-7;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = a[j] * m + c;
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    if (s == (T)-1) out[0] = s;     // keeps the chains live
}

}  // namespace

// GFLOP/s (2 per FMA) over `reps` timed launches on the current device.
extern "C" avs_status avs_measure_fma_peak(int fp64, int iters, double* gflops)
{
    if (!gflops || iters <= 0) return AVS_EINVAL;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int threads = 256, blocks = nsm * 8;
    void* out = nullptr;
    if (cudaMalloc(&out, 16) != cudaSuccess) return AVS_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {     // first launch warms up
        cudaEventRecord(e0);
        if (fp64) k_fma<double><<<blocks, threads>>>(iters, 1.0, (double*)out);
        else k_fma<float><<<blocks, threads>>>(iters, 1.0f, (float*)out);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (cudaGetLastError() != cudaSuccess) return AVS_ECUDA;
    *gflops = 2.0 * 8.0 * (double)iters * threads * blocks / (ms * 1e-3) / 1e9;
    return AVS_OK;
}
