// diag.cu -- measurement helper: the FP32 FMA throughput of the device, the roofline
// denominator of the ACE contraction (plain FP32 arithmetic, no tensor cores).
#include <cuda_runtime.h>

#include "ap.h"

namespace {

constexpr int kChains = 16;     // independent FMA chains per thread (hide the FMA latency)
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_fma_peak(float* out, int iters, float a, float b) {
    float acc[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc[k] = fmaf(acc[k], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += acc[k];
    if (s == 1.2345678f) out[blockIdx.x] = s;   // keeps the chains live; never true in practice
}

}  // namespace

extern "C" ap_status ap_probe_fp32_peak(int iters, double* tflops, double* ms_out) {
    if (!tflops || iters < 1 || iters > (1 << 20)) return AP_ERR_ARG;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return AP_ERR_CUDA;
    const int blocks = nsm * 8;      // 8 blocks x 256 threads = 64 warps per SM
    float* out = nullptr;
    if (cudaMalloc((void**)&out, sizeof(float) * blocks) != cudaSuccess) return AP_ERR_OOM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma_peak<<<blocks, kThreads>>>(out, iters / 4 + 1, 0.999f, 1e-4f);      // warm-up
    cudaEventRecord(e0);
    k_fma_peak<<<blocks, kThreads>>>(out, iters, 0.999f, 1e-4f);
    cudaEventRecord(e1);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return AP_ERR_CUDA;
    const double flops = 2.0 * kChains * (double)iters * blocks * kThreads;
    *tflops = flops / (ms * 1e-3) / 1e12;
    if (ms_out) *ms_out = ms;
    return AP_OK;
}
