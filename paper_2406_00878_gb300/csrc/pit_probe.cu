// pit_probe.cu -- pit_probe_fma_peak: the FP64 (or FP32) fused multiply-add rate this
// GPU sustains, measured in the calling process.
//
// The level-chain kernels of this library do FP64 arithmetic on data held in shared
// memory, so their roofline is the FP64 pipe, not HBM. GB300 runs FP64 at a small
// fraction of its FP32 rate, and the nominal figure depends on the clock the part
// holds under load, so the benchmark measures the rate it compares against: every
// thread of a full-occupancy grid runs eight independent FMA chains (enough
// independent work to keep the pipe busy through its latency), timed with CUDA
// events, best of several launches.
#include <cuda_runtime.h>

#include <algorithm>

#include "pit.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_probe_kernel(T* out, int iters, T b, T c) {
    T a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (T)((threadIdx.x + k) & 15) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);  // bounded: fixed point c / (1 - b)
    }
    T s = a[0];
#pragma unroll
    for (int k = 1; k < kChains; ++k) s += a[k];
    out[(size_t)blockIdx.x * kThreads + threadIdx.x] = s;
}

template <typename T>
pit_status run_probe(cudaStream_t st, int iters, double* tflops) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PIT_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PIT_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fma_probe_kernel<T>, kThreads, 0) != cudaSuccess)
        return PIT_ECUDA;
    const int blocks = sms * std::max(per, 1);
    T* out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * (size_t)blocks * kThreads) != cudaSuccess) return PIT_ENOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    pit_status s = PIT_OK;
    double best = 0.0;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) s = PIT_ECUDA;
    // one warm-up launch, then the best of five
    for (int rep = 0; rep < 6 && s == PIT_OK; ++rep) {
        if (cudaEventRecord(e0, st) != cudaSuccess) s = PIT_ECUDA;
        fma_probe_kernel<T><<<blocks, kThreads, 0, st>>>(out, iters, (T)0.9999, (T)1e-4);
        if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess)
            s = PIT_ECUDA;
        float ms = 0.f;
        if (s == PIT_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) s = PIT_ECUDA;
        if (s == PIT_OK && rep > 0 && ms > 0.f) {
            const double flops = 2.0 * kChains * (double)iters * blocks * kThreads;
            best = std::max(best, flops / (ms * 1e-3) / 1e12);
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (s == PIT_OK) *tflops = best;
    return s;
}

}  // namespace

extern "C" pit_status pit_probe_fma_peak(int precision, void* stream, double* tflops) {
    if (!tflops || (precision != 0 && precision != 1)) return PIT_EINVAL;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    // ~40 ms per launch at GB300's rates (FP32 runs 64x the FP64 rate)
    return precision == 0 ? run_probe<double>(st, 8192, tflops) : run_probe<float>(st, 8192 * 48, tflops);
}
