// FP32 fused multiply-add throughput probe.  The per-atom kernels are bound by the FP32
// CUDA-core pipe, so their roofline denominator is this probe's measured rate on the GPU
// that runs them (not a figure derived from unit counts and the maximum clock).
//
// Every thread runs CHAINS independent dependent-FMA chains; CHAINS x (warps per
// scheduler) covers the FMA latency, so the pipe is the only limit.  The result feeds a
// store guarded by a runtime flag the compiler cannot see through, which keeps the
// chains live without writing anything in practice.
#include <cuda_runtime.h>
#include <stdint.h>

#include "nep_gb300.h"

namespace {
constexpr int CHAINS = 8;
constexpr int THREADS = 256;
constexpr int UNROLL = 16;

__global__ void __launch_bounds__(THREADS) k_fma_probe(int64_t iters, float b, float c, int flag, float *sink) {
    float a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = (float)threadIdx.x * 1e-3f + (float)k;
    for (int64_t it = 0; it < iters; it += UNROLL) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
#pragma unroll
            for (int k = 0; k < CHAINS; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k];
    if (flag) sink[0] = s;
}
}  // namespace

extern "C" int nep_fp32_fma_probe(void *cuda_stream, int blocks, int64_t iters, float *sink_dev, double *flops) {
    if (blocks < 1 || iters < UNROLL || iters % UNROLL != 0 || !sink_dev || !flops) return NEP_EINVAL;
    k_fma_probe<<<blocks, THREADS, 0, (cudaStream_t)cuda_stream>>>(iters, 0.999f, 1e-3f, 0, sink_dev);
    if (cudaGetLastError() != cudaSuccess) return NEP_ECUDA;
    *flops = 2.0 * CHAINS * (double)iters * (double)blocks * THREADS;
    return NEP_OK;
}
