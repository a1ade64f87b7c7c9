// FMA throughput of the device in FP32 and FP64: the denominators of the
// rooflines of the ALU-bound kernels (the FP32 plane kernel; the FP64
// density kernel of the self-consistent loop).  Every thread runs eight
// independent FMA chains over its registers; the grid fills every SM with
// 2048 threads, so the FMA pipes, not latency, set the rate.  Timed with
// CUDA events after a warm-up launch; the best of several launches is
// reported.
#include <cuda_runtime.h>

#include "../../include/mb.h"
#include "../../include/mb_testing.h"

namespace mb {

constexpr int kProbeChains = 8;
constexpr int kProbeUnroll = 16;

template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(T b, T c, int iters, T *sink) {
    T a[kProbeChains];
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) a[i] = (T)(threadIdx.x + i) * (T)1e-3;
    for (int it = 0; it < iters; it += kProbeUnroll) {
#pragma unroll
        for (int u = 0; u < kProbeUnroll; ++u)
#pragma unroll
            for (int i = 0; i < kProbeChains; ++i) a[i] = fma(a[i], b, c);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < kProbeChains; ++i) s += a[i];
    if (s == (T)1234.5678) sink[blockIdx.x] = s;   // keeps the chains live; never true for the inputs used
}

template <typename T>
static int probe(int device, int reps, int iters, double *tflops, double *ms) {
    if (reps < 1 || reps > 100 || device < 0) return MB_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return MB_ECUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return MB_ECUDA;
    const int threads = 256, blocks = sms * 8;
    T *sink = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = MB_OK;
    if (cudaMalloc(&sink, sizeof(T) * blocks) != cudaSuccess) return MB_ENOMEM;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        rc = MB_ECUDA;
    double best = 1e300;
    for (int r = -1; r < reps && rc == MB_OK; ++r) {     // r = -1: warm-up
        cudaEventRecord(e0, s);
        fma_probe_kernel<T><<<blocks, threads, 0, s>>>((T)0.999, (T)1e-4, iters, sink);
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
        const double flops = 2.0 * kProbeChains * (double)iters * threads * blocks;
        if (ms) *ms = best;
        if (tflops) *tflops = flops / (best * 1e-3) / 1e12;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(sink);
    return rc;
}

}  // namespace mb

extern "C" int mb_probe_fp32_fma(int device, int reps, double *tflops, double *ms) {
    return mb::probe<float>(device, reps, 1 << 15, tflops, ms);
}

extern "C" int mb_probe_fp64_fma(int device, int reps, double *tflops, double *ms) {
    return mb::probe<double>(device, reps, 1 << 11, tflops, ms);
}
