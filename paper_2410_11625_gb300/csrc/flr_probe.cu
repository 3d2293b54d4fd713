// flr_probe.cu -- measured FP32 FMA throughput of the current GPU (instrumentation; the
// paper has no counterpart).  The per-pixel FLR path is bound by the FP32 ALUs, so its
// roofline needs the rate those ALUs actually reach on this part at the clock it holds.
//
// Each thread runs 8 independent chains x <- fma(x, a, b) (a, b kernel arguments, so
// nothing folds), 16 warps per SM, 4 CTAs of 256 threads per SM: enough independent
// instructions per scheduler to hide the FMA latency.  One FMA = 2 flops.
#include <cuda_runtime.h>

#include "flr.h"

namespace {

constexpr int kProbeThreads = 256, kChains = 8;

__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(float *out, int iters, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = (float)(threadIdx.x + j) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k)
#pragma unroll
            for (int j = 0; j < kChains; ++j) x[j] = fmaf(x[j], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += x[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int flr_fp32_fma_peak(int iters, double *tflops, double *ms)
{
    if (iters <= 0 || !tflops || !ms) return FLR_ERR_ARG;
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FLR_ERR_CUDA;
    const int blocks = 4 * n_sm;
    float *out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int status = FLR_OK;
    if (cudaMalloc(&out, sizeof(float) * blocks * kProbeThreads) != cudaSuccess) return FLR_ERR_NOMEM;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        status = FLR_ERR_CUDA;
    } else {
        float best = -1.f;
        for (int rep = 0; rep < 4 && status == FLR_OK; ++rep) {  // the first run warms the clocks up
            cudaEventRecord(e0, st);
            fma_probe_kernel<<<blocks, kProbeThreads, 0, st>>>(out, iters, 0.9999999f, 1e-7f);
            cudaEventRecord(e1, st);
            float t = 0.f;
            if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
                status = FLR_ERR_CUDA;
            else if (rep > 0 && (best < 0.f || t < best))
                best = t;
        }
        if (status == FLR_OK) {
            const double flops = 2.0 * blocks * kProbeThreads * kChains * 16.0 * (double)iters;
            *ms = best;
            *tflops = flops / (best * 1e-3) / 1e12;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(out);
    return status;
}
