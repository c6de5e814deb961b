// Measured FP32 FMA throughput of the device: the ALU roofline against which the trajectory
// kernels (FP32 arithmetic, no dense contraction) are reported.  Every thread runs kChains
// independent chains of fused multiply-adds, enough to cover the FMA latency with a few warps
// per scheduler; the grid fills every SM with kCtasPerSm CTAs.  The chains' values stay
// bounded (|a| < 1) and feed a store that never happens but that the compiler cannot rule
// out, so no FMA is removed.
#include <cuda_runtime.h>

#include <string>

#include "spasm.h"

namespace {

constexpr int kChains = 16;
constexpr int kThreads = 256;
constexpr int kCtasPerSm = 8;
constexpr int kUnroll = 8;

__global__ void __launch_bounds__(kThreads) k_fma_peak(float* __restrict__ sink, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = (float)threadIdx.x * 1e-3f + (float)i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int i = 0; i < kChains; ++i) x[i] = fmaf(x[i], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    if (s == -1.2345e-30f) sink[blockIdx.x] = s;
}

struct Events {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Events() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

}  // namespace

extern "C" spasm_status spasm_fp32_fma_peak(double target_ms, double* tflops, double* ms, double* flop) {
    if (!tflops || !(target_ms > 0.0) || target_ms > 10000.0) return SPASM_ERR_INVALID;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SPASM_ERR_CUDA;
    const int grid = sms * kCtasPerSm;
    float* sink = nullptr;
    if (cudaMalloc(reinterpret_cast<void**>(&sink), sizeof(float) * grid) != cudaSuccess) return SPASM_ERR_NOMEM;
    Events ev;
    cudaError_t e = cudaEventCreate(&ev.a);
    if (e == cudaSuccess) e = cudaEventCreate(&ev.b);
    // calibrate: a short run, then one sized to about target_ms (at least 64 iterations)
    int iters = 64;
    float t = 0.f;
    for (int pass = 0; pass < 3 && e == cudaSuccess; ++pass) {
        cudaEventRecord(ev.a, 0);
        k_fma_peak<<<grid, kThreads>>>(sink, iters, 0.9999999f, 1e-7f);
        cudaEventRecord(ev.b, 0);
        e = cudaEventSynchronize(ev.b);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ev.a, ev.b);
        if (e != cudaSuccess || pass == 2) break;
        const double scale = t > 0.f ? target_ms / t : 100.0;
        const double next = (double)iters * (scale > 1000.0 ? 1000.0 : scale);
        iters = next < 64.0 ? 64 : (next > 2e8 ? 200000000 : (int)next);
    }
    cudaFree(sink);
    if (e != cudaSuccess) return SPASM_ERR_CUDA;
    const double f = 2.0 * kChains * kUnroll * (double)iters * (double)kThreads * (double)grid;
    *tflops = f / ((double)t * 1e-3) / 1e12;
    if (ms) *ms = t;
    if (flop) *flop = f;
    return SPASM_OK;
}
