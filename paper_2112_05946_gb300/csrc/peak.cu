// FMA throughput of the GPU's FP64 and FP32 pipes: the compute denominators of the stage
// kernels' roofline.  Not part of the scheme.  Every thread runs kChains independent chains
// x <- x * a + b (one fused multiply-add each) for `iters` rounds of kUnroll steps, so that
// the pipe never waits on a dependency; a grid of 8 CTAs of 256 threads per SM keeps every
// scheduler fed.  The result of the chains is written only if it equals a value it cannot
// reach, so the compiler keeps the arithmetic and nothing is stored.
#include <cuda_runtime.h>

#include "frsg_peak.h"

namespace {

constexpr int kChains = 16;
constexpr int kUnroll = 8;

template <typename T>
__global__ void fma_chains(T* sink, int iters, T a, T b) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
        }
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == T(-12345.678)) sink[blockIdx.x] = s;
}

template <typename T>
int measure(int iters, int reps, double* tflops) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    const int blocks = sms * 8, threads = 256;
    T* sink = nullptr;
    if (cudaMalloc(&sink, sizeof(T) * blocks) != cudaSuccess) return 1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const T a = T(0.999999), b = T(1e-6);
    fma_chains<T><<<blocks, threads>>>(sink, iters, a, b);   // warm-up
    float best = 1e30f;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0);
        fma_chains<T><<<blocks, threads>>>(sink, iters, a, b);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (err != cudaSuccess) return 1;
    const double flops = 2.0 * kChains * kUnroll * (double)iters * blocks * threads;
    *tflops = flops / (best * 1e-3) / 1e12;
    return 0;
}

}  // namespace

extern "C" int frsg_peak_fma(int fp64, int iters, int reps, double* tflops) {
    if (!tflops || iters < 1 || reps < 1) return 1;
    return fp64 ? measure<double>(iters, reps, tflops) : measure<float>(iters, reps, tflops);
}
