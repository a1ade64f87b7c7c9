// FP32 FMA throughput of the device: the denominator of the plane kernel's
// roofline (an ALU-bound kernel).  Every thread runs eight independent FFMA
// chains over its registers; the grid fills every SM with 2048 threads, so
// the FMA pipes, not latency, set the rate.  Timed with CUDA events after a
// warm-up launch; the best of several launches is reported.
#include <cuda_runtime.h>

#include "../../include/mb.h"
#include "../../include/mb_testing.h"

namespace mb {

constexpr int kProbeChains = 8;
constexpr int kProbeUnroll = 16;

__global__ void __launch_bounds__(256) fma_probe_kernel(float b, float c, int iters, float *sink) {
    float a[kProbeChains];
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) a[i] = (float)(threadIdx.x + i) * 1e-3f;
    for (int it = 0; it < iters; it += kProbeUnroll) {
#pragma unroll
        for (int u = 0; u < kProbeUnroll; ++u)
#pragma unroll
            for (int i = 0; i < kProbeChains; ++i) a[i] = fmaf(a[i], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) s += a[i];
    if (s == 1234.5678f) sink[blockIdx.x] = s;   // keeps the chains live; never true for the inputs used
}

}  // namespace mb

extern "C" int mb_probe_fp32_fma(int device, int reps, double *tflops, double *ms) {
    if (reps < 1 || reps > 100 || device < 0) return MB_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return MB_ECUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return MB_ECUDA;
    const int threads = 256, blocks = sms * 8, iters = 1 << 15;
    float *sink = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = MB_OK;
    if (cudaMalloc(&sink, sizeof(float) * blocks) != cudaSuccess) return MB_ENOMEM;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        rc = MB_ECUDA;
    double best = 1e300;
    for (int r = -1; r < reps && rc == MB_OK; ++r) {     // r = -1: warm-up
        cudaEventRecord(e0, s);
        mb::fma_probe_kernel<<<blocks, threads, 0, s>>>(0.999f, 1e-4f, iters, sink);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            rc = MB_ECUDA;
            break;
        }
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (r >= 0 && t < best) best = t;
    }
    if (rc == MB_OK) {
        const double flops = 2.0 * mb::kProbeChains * (double)iters * threads * blocks;
        if (ms) *ms = best;
        if (tflops) *tflops = flops / (best * 1e-3) / 1e12;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(sink);
    return rc;
}
