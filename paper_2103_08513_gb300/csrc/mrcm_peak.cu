// FP64 throughput measurement: the denominator of the FP64 roofline fractions
// the benchmark reports (the FP64 pipe bounds the refinement residual and the
// interface factorisation).  No counterpart in the paper.
//
// Method: every thread of a grid of 8 CTAs x 256 threads per SM runs eight
// independent dependent chains x <- fma(x, a, b); enough warps per SM and
// independent chains per warp keep the FP64 unit busy, so the measured rate is
// its issue limit.  Timed with CUDA events on the caller's stream; the best of
// three launches (after one warm-up) is reported.
#include <cuda_runtime.h>

#include "../../include/mrcm.h"

namespace {

__device__ double g_peak_sink;

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_fp64_fma(int iters, double a, double b) {
    double x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 1e-3 * (threadIdx.x + 1) + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == -1.0) g_peak_sink = s;               // never true; keeps the chains live
}

}  // namespace

extern "C" mrcm_status mrcm_measure_fp64_peak(void* stream, double* tflops) {
    if (!tflops) return MRCM_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MRCM_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MRCM_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const int iters = 4096, grid = sms * 8;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return MRCM_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return MRCM_ERR_CUDA; }
    float best = 0.0f;
    bool ok = true;
    for (int rep = 0; rep < 4 && ok; ++rep) {
        cudaEventRecord(e0, st);
        k_fp64_fma<<<grid, kThreads, 0, st>>>(iters, 0.9999999, 1e-7);
        cudaEventRecord(e1, st);
        ok = cudaEventSynchronize(e1) == cudaSuccess;
        float ms = 0.0f;
        if (ok) ok = cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
        if (ok && rep > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok || cudaGetLastError() != cudaSuccess || best <= 0.0f) return MRCM_ERR_CUDA;
    const double flops = 2.0 * (double)grid * kThreads * kChains * iters;
    *tflops = flops / (best * 1e-3) / 1e12;
    return MRCM_OK;
}
