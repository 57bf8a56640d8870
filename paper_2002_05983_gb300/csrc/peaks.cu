// Measured device peaks for the roofline R(t) = min(P_fp32 / F, BW * t / (2 s)):
// the FP32 fused multiply-add throughput of the CUDA cores (independent FMA
// chains in every thread, far more warps than the FMA pipes need) and the
// HBM bandwidth seen by a plain 16-byte copy kernel over buffers larger than
// L2.  Both are timed with CUDA events after a warm-up launch.
#include <cstdint>

#include <cuda_runtime.h>

#include "stencil.h"

namespace {

constexpr int kChains = 8;    // independent FMA chains per thread
constexpr int kUnroll = 16;   // FMAs per chain per loop iteration

__global__ void __launch_bounds__(1024) fma_peak_kernel(float *sink, int iters, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = 1.0f + static_cast<float>(threadIdx.x * kChains + i) * 1e-7f;
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int i = 0; i < kChains; ++i) x[i] = __fmaf_rn(x[i], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    if (s == -1.0f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;   // never true; keeps the chains live
}

__global__ void __launch_bounds__(256) copy_peak_kernel(const float4 *__restrict__ src, float4 *__restrict__ dst,
                                                        int64_t n)
{
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = src[i];
}

int fail(cudaError_t e)
{
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? STENCIL_ERR_OOM : STENCIL_ERR_CUDA;
}

}  // namespace

extern "C" int stencil_measure_peaks(void *stream, stencil_peaks *out)
{
    if (!out) return STENCIL_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0, khz = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
    if (e != cudaSuccess) return fail(e);
    const size_t bytes = size_t(1) << 30;   // per buffer: far above the L2 size
    float *sink = nullptr, *a = nullptr, *b = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float fma_ms = 0.f, copy_ms = 1e30f;
    const int threads = 1024, blocks = sms * 2, iters = 8192;
    const int64_t n4 = static_cast<int64_t>(bytes / sizeof(float4));
    e = cudaMalloc(&sink, sizeof(float) * threads * blocks);
    if (e == cudaSuccess) e = cudaMalloc(&a, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&b, bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(a, 0, bytes, st);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        fma_peak_kernel<<<blocks, threads, 0, st>>>(sink, iters / 8, 0.9999999f, 1e-7f);   // warm-up
        cudaEventRecord(e0, st);
        fma_peak_kernel<<<blocks, threads, 0, st>>>(sink, iters, 0.9999999f, 1e-7f);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&fma_ms, e0, e1);
    }
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // first launch warms up; best of the rest
        cudaEventRecord(e0, st);
        copy_peak_kernel<<<sms * 8, 256, 0, st>>>(reinterpret_cast<const float4 *>(a), reinterpret_cast<float4 *>(b), n4);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && e == cudaSuccess) copy_ms = ms < copy_ms ? ms : copy_ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    cudaFree(a);
    cudaFree(b);
    if (e != cudaSuccess) return fail(e);
    const double fmas = static_cast<double>(blocks) * threads * iters * kUnroll * kChains;
    out->fp32_flops = 2.0 * fmas / (fma_ms * 1e-3);
    out->copy_bytes_per_s = 2.0 * static_cast<double>(bytes) / (copy_ms * 1e-3);
    out->sms = sms;
    out->sm_clock_khz = khz;
    return STENCIL_OK;
}
