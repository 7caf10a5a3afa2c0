// Arithmetic peaks of the GPU the library runs on, measured: the FP64 and FP32 FMA rates that
// bound the SIMT contractions (FP64 grids, the batched FP32 instances) and the FP64 Fourier
// passes. Each thread runs independent FMA chains in registers; the rate is 2 flops per FMA
// over the CUDA-event time of the launch.
#include <cuda_runtime.h>

#include "../../include/adr.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_loop_kernel(int iters, T seed, T* sink) {
    T acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = seed + T(threadIdx.x + c);
    const T m = T(0.999999), a = T(1e-7);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], m, a);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    if (s == T(-1.2345)) *sink = s;   // never true for these inputs; keeps the chains live
}

template <typename T>
adr_status measure(int iters, double* tflops) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ADR_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return ADR_ERR_CUDA;
    T* sink = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    adr_status out = ADR_OK;
    if (cudaMalloc(&sink, sizeof(T)) != cudaSuccess) return ADR_ERR_ALLOC;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess)
        out = ADR_ERR_CUDA;
    const unsigned blocks = unsigned(sms) * 8u;
    if (out == ADR_OK) {
        fma_loop_kernel<T><<<blocks, kThreads, 0, st>>>(iters / 8 + 1, T(0.5), sink);   // warm-up
        cudaEventRecord(e0, st);
        fma_loop_kernel<T><<<blocks, kThreads, 0, st>>>(iters, T(0.5), sink);
        cudaEventRecord(e1, st);
        float ms = 0.f;
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f) {
            out = ADR_ERR_CUDA;
        } else {
            const double fmas = double(blocks) * kThreads * double(iters) * 16.0 * kChains;
            *tflops = 2.0 * fmas / (double(ms) * 1e-3) / 1e12;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(sink);
    return out;
}

}  // namespace

extern "C" adr_status adr_measure_peak(int kind, int iters, double* tflops) {
    if (!tflops || iters < 1 || iters > (1 << 20)) return ADR_ERR_ARG;
    if (kind == ADR_PEAK_FP64_FMA) return measure<double>(iters, tflops);
    if (kind == ADR_PEAK_FP32_FMA) return measure<float>(iters, tflops);
    return ADR_ERR_ARG;
}
