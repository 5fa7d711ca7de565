// FMA throughput of this GPU in FP32, FP64 and packed FP32 pairs, measured
// with independent multiply-add chains per thread (used as the ALU roofline of
// the step kernels; the paper has no counterpart).
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

// the same chains on FP32 pairs with the packed two-lane FMA
__global__ void k_fma2(int iters, float seed, float* out)
{
    float2 a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = make_float2(seed + (float)(threadIdx.x + j), seed - (float)j);
    const float2 m = make_float2(0.999999f, 0.999998f), c = make_float2(1e-7f, 2e-7f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = __ffma2_rn(a[j], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j].x + a[j].y;
    if (s == -1.f) out[0] = s;
}

}  // namespace

// GFLOP/s (2 per FMA) of the second of two launches on the current device.
// kind: 0 FP32, 1 FP64, 2 FP32 pairs (packed two-lane FMA).
extern "C" avs_status avs_measure_fma_peak(int kind, int iters, double* gflops)
{
    if (!gflops || iters <= 0 || kind < 0 || kind > 2) return AVS_EINVAL;
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
        if (kind == 1) k_fma<double><<<blocks, threads>>>(iters, 1.0, (double*)out);
        else if (kind == 2) k_fma2<<<blocks, threads>>>(iters, 1.0f, (float*)out);
        else k_fma<float><<<blocks, threads>>>(iters, 1.0f, (float*)out);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (cudaGetLastError() != cudaSuccess) return AVS_ECUDA;
    *gflops = (kind == 2 ? 2.0 : 1.0) * 2.0 * 8.0 * (double)iters * threads * blocks / (ms * 1e-3) / 1e9;
    return AVS_OK;
}
