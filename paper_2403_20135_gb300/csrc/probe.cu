// FP64 fused multiply-add rate of the current GPU: the denominator the FP64
// transform kernels are measured against (their contractions and FFT
// butterflies run on the FP64 pipe).  Every SM runs blocks of independent
// FMA chains long enough that the pipe, not the issue of the loop, bounds
// the rate.  Nothing here changes a GPU setting; clocks are whatever the GPU
// runs at.

#include <cuda_runtime.h>

#include "../../include/sdc.h"

namespace {

constexpr int kChains = 8;          // independent FMA chains per thread (covers the FP64 pipe latency)
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_dfma_rate(int iters, double x, double y, double *sink) {
    double a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = 1.0 + 1e-3 * (threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], x, y);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    // never true for the values the host passes; keeps the chains live
    if (s == -1.0) sink[0] = s;
}

}  // namespace

extern "C" int sdc_fp64_fma_rate(int iters, int repeats, void *cuda_stream, double *sink, double *tflops) {
    if (!sink || !tflops || iters < 1 || repeats < 1) return SDC_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SDC_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SDC_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dfma_rate, kThreads, 0) != cudaSuccess)
        return SDC_ECUDA;
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return SDC_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return SDC_ECUDA;
    }
    const double x = 0.999999, y = 1e-6;           // a -> a x + y stays near 1: no overflow, no subnormals
    k_dfma_rate<<<blocks, kThreads, 0, st>>>(iters, x, y, sink);   // warm-up
    cudaEventRecord(e0, st);
    for (int r = 0; r < repeats; ++r) k_dfma_rate<<<blocks, kThreads, 0, st>>>(iters, x, y, sink);
    cudaEventRecord(e1, st);
    int status = SDC_OK;
    float ms = 0.0f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
        cudaPeekAtLastError() != cudaSuccess || !(ms > 0.0f)) {
        status = SDC_ECUDA;
    } else {
        const double flops = 2.0 * kChains * (double)iters * kThreads * (double)blocks * repeats;
        *tflops = flops / (ms * 1e-3) / 1e12;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return status;
}
