// measure.cu -- the float64 arithmetic rate of the GPU, for stating the float64
// path against the roof that binds it (the float64 Born iteration is bound by
// the FP64 pipes of this part, not by HBM).
//
// Each thread runs eight independent chains of fused multiply-adds in double
// precision (one FMA = 2 floating-point operations); the grid fills every SM
// with 16 blocks of 256 threads.  Not on the solver's path.
#include <cuda_runtime.h>

#include "cbs.h"

namespace {

__global__ void k_fp64_fma_chains(double* out, int iters)
{
    double a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = 1e-3 * (threadIdx.x + j);
    const double b = 0.9999999, c = 1e-7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = fma(a[j], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    if (s == -1.0) out[0] = s;  // never true; keeps the chains live
}

}  // namespace

extern "C" cbs_status cbs_fp64_rate(double* tflops)
{
    if (!tflops) return CBS_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CBS_ECUDA;
    double* out = nullptr;
    if (cudaMalloc(&out, sizeof(double)) != cudaSuccess) return CBS_ENOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const int blocks = sms * 16, threads = 256, iters = 1 << 14;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        k_fp64_fma_chains<<<blocks, threads>>>(out, iters);  // warm-up
        cudaEventRecord(e0);
        k_fp64_fma_chains<<<blocks, threads>>>(out, iters);
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
    }
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess || ms <= 0.0f) return CBS_ECUDA;
    const double flops = 2.0 * 8.0 * iters * (double)blocks * threads;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return CBS_OK;
}
