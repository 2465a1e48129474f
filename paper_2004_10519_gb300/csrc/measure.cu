// Measurement hook: FP32 (non-tensor) FMA throughput of the current device,
// the compute ceiling against which the stencil kernels' FLOP rates are
// quoted.  Declared in the Python binding, not in the public header.
#include "internal.h"

#include <algorithm>

namespace {

constexpr int CHAINS = 8;   // independent FMA chains per thread (hide the pipe latency)

__global__ void __launch_bounds__(256) ffma_kernel(float *out, int iters, float a, float b)
{
    float x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; c++) x[c] = 1e-3f * (threadIdx.x + c);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < CHAINS; c++) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CHAINS; c++) s += x[c];
    if (s == 1234.5f) out[blockIdx.x] = s;   // keeps the chains live; never true for a, b below
}

}  // namespace

// TFLOP/s of fused multiply-adds (2 FLOP each) over all SMs, best of 3 runs
extern "C" int prop_fp32_peak(double *tflops)
{
    if (!tflops) return PROP_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PROP_ECUDA;
    const int blocks = sms * 8, threads = 256, iters = 1 << 15;
    float *out = nullptr;
    if (int rc = wp_malloc(nullptr, (void **)&out, sizeof(float) * blocks, "FP32 peak measurement")) return rc;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 0.0;
    ffma_kernel<<<blocks, threads>>>(out, iters / 8, 0.999f, 1e-4f);   // warm-up (clocks up)
    for (int r = 0; r < 3; r++) {
        cudaEventRecord(e0);
        ffma_kernel<<<blocks, threads>>>(out, iters, 0.999f, 1e-4f);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double flops = 2.0 * CHAINS * (double)iters * blocks * threads;
        if (ms > 0.f) best = std::max(best, flops / (ms * 1e-3) / 1e12);
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return PROP_ECUDA;
    *tflops = best;
    return PROP_OK;
}
