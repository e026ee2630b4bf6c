// Measured FMA throughput of the CUDA cores (the ALU peak the FP64 and FP32
// stencil paths are compared against).  Every thread runs 8 independent FMA
// chains for `iters` rounds on values the compiler cannot fold, and writes
// their sum so that nothing is eliminated; the grid fills every SM several
// times over.  FLOP = 2 * 8 * iters * threads, timed with CUDA events after a
// warm-up launch.
#include "mpmc.h"

#include <cuda_runtime.h>

namespace {

template <class T>
__global__ void __launch_bounds__(256) k_fma_peak(int iters, T b, T c, T* out) {
    T a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = (T)(threadIdx.x + i) * (T)1e-3;
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = fma(a[i], b, c);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += a[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T>
int run(double* tflops) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return MPMC_ECUDA;
    const int blocks = sms * 16, threads = 256, iters = sizeof(T) == 8 ? 2048 : 16384;
    T* out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * (size_t)blocks * threads) != cudaSuccess) {
        (void)cudaGetLastError();
        return MPMC_ENOMEM;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const T b = (T)0.999999, c = (T)1e-7;
    k_fma_peak<T><<<blocks, threads>>>(iters, b, c, out);   // warm-up
    cudaEventRecord(e0);
    k_fma_peak<T><<<blocks, threads>>>(iters, b, c, out);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess || !(ms > 0)) return MPMC_ECUDA;
    *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (ms * 1e-3) / 1e12;
    return MPMC_OK;
}

}  // namespace

extern "C" int mpmc_fma_peak(int precision, double* tflops) {
    if (!tflops) return MPMC_EINVAL;
    if (precision == MPMC_FP64) return run<double>(tflops);
    if (precision == MPMC_FP32) return run<float>(tflops);
    return MPMC_ENOTSUP;
}
