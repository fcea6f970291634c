// FP32 FMA throughput probe: the denominator of the pair stage's roofline.
// Every thread runs kChains independent FMA chains (enough to cover the FMA
// latency at full occupancy) for a fixed number of steps; the grid fills every
// SM several times over.  One FMA counts as two flops.
#include <cstdio>

#include "internal.h"

namespace g3 {
namespace {

constexpr int kChains = 8;
constexpr int kSteps = 4096;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_fma_probe(float* out, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int s = 0; s < kSteps; ++s) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float t = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) t += x[c];
    if (t == 1234.5f) out[blockIdx.x * blockDim.x + threadIdx.x] = t;  // keeps the chains live
}

}  // namespace
}  // namespace g3

extern "C" int g3pcf_fp32_peak(double* tflops, void* stream) {
    using namespace g3;
    if (!tflops) return G3PCF_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return G3PCF_ERR_CUDA;
    const int blocks = nsm * 8 * 4;
    float* out = nullptr;
    if (cudaMalloc(&out, sizeof(float) * blocks * kThreads) != cudaSuccess) return G3PCF_ERR_ALLOC;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int r = 0; r < 6; ++r) {
        cudaEventRecord(e0, st);
        k_fma_probe<<<blocks, kThreads, 0, st>>>(out, 0.999f, 1e-4f);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0 && ms < best) best = ms;  // first launch is warm-up
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return G3PCF_ERR_CUDA;
    const double flops = 2.0 * kChains * (double)kSteps * blocks * kThreads;
    *tflops = flops / (best * 1e-3) / 1e12;
    return G3PCF_OK;
}
