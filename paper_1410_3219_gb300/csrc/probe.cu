// Arithmetic-pipe peaks measured on the device: independent chains of fused
// multiply-adds in FP64 and in FP32, timed with CUDA events.  The sweep's
// FP64 kernels are bound by FP64 issue, so their roofline fraction is read
// against both the peak derived from unit counts and clocks and this
// measured one.
#include <cuda_runtime.h>

#include "../../include/rich.h"
#include "api_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kIters = 2048;
constexpr int kBlock = 256;

template <class T> __global__ void __launch_bounds__(kBlock) k_fma_chains(T seed, T *sink)
{
    T a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) a[c] = seed + (T)(threadIdx.x + c);
    const T b = (T)0.999999, d = (T)1e-7;
    for (int it = 0; it < kIters; it++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) a[c] = fma(a[c], b, d);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += a[c];
    if (s == (T)-1) sink[blockIdx.x] = s;  // never true: keeps the chains live
}

template <class T> int time_chains(int blocks, double *tflops)
{
    T *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    RICH_CUDA_TRY(cudaMalloc(&sink, sizeof(T) * blocks));
    cudaError_t err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    float best = 0.0f;
    for (int rep = 0; rep < 4 && err == cudaSuccess; rep++) {  // the first launch warms up
        cudaEventRecord(e0);
        k_fma_chains<T><<<blocks, kBlock>>>((T)1.0, sink);
        cudaEventRecord(e1);
        err = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (err != cudaSuccess) return rich::set_error(RICH_ECUDA, cudaGetErrorString(err));
    const double flops = 2.0 * kChains * kIters * (double)kBlock * blocks;
    *tflops = flops / (best * 1e-3) / 1e12;
    return RICH_OK;
}

}  // namespace

extern "C" int rich_probe_pipe_peaks(double *fp64_tflops, double *fp32_tflops)
{
    if (!fp64_tflops || !fp32_tflops) return rich::set_error(RICH_EINVAL, "NULL output");
    int dev = 0, sms = 0;
    RICH_CUDA_TRY(cudaGetDevice(&dev));
    RICH_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int rc = time_chains<double>(sms * 8, fp64_tflops);
    if (rc != RICH_OK) return rc;
    // FP32 runs 64x faster: more blocks so the launch lasts long enough to time
    return time_chains<float>(sms * 256, fp32_tflops);
}
