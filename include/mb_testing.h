/* mb_testing.h -- self-test entry points of libmbgb300 (not part of the
 * numerical method; the paper has no counterpart).  They let a test check a
 * building block of the library on its own. */
#ifndef MB_TESTING_H
#define MB_TESTING_H
#ifdef __cplusplus
extern "C" {
#endif

/* D = A * Bt^T on the tensor cores (tcgen05, BF16 operands, FP32
 * accumulation in tensor memory).  A: device M x K BF16 row-major, Bt:
 * device N x K BF16 row-major, D: device M x N float row-major.  Allocates a
 * 4-byte status word; returns MB_ETIMEOUT if a bounded device wait expired. */
int mb_debug_gemm_bf16(const void *A, const void *Bt, float *D, int M, int N, int K, void *stream);

/* G = A^H B on the tensor cores (tcgen05, TF32 operands split as hi + lo for
 * FP32 accuracy, FP32 accumulation in tensor memory, chunks reduced in
 * FP64): the eigensolver's Gram building block.  V: device FP32 complex
 * (interleaved), ma + mb vectors of n elements stored one after another, the
 * ma vectors of A first; nsplit chunks of the vector length (1..4096).  G:
 * host, ma x mb complex (interleaved doubles), row i = A_i.  Requires
 * 1 <= ma <= 64 and 1 <= mb <= 64.  Allocates and frees its own device
 * buffers; returns MB_EINVAL for bad sizes, MB_ETIMEOUT if a bounded device
 * wait expired. */
int mb_debug_gram_tc32(const void *V, long long n, int ma, int mb, int nsplit, double *G, void *stream);

/* C = A Y with the eigensolver's float-float rotation kernel (FP64 vectors,
 * products and sums in pairs of FP32 numbers).  A: device FP64 complex
 * (interleaved), ma vectors of n elements one after another; Y: host ma x mc
 * complex (interleaved doubles), row i = the coefficients of A_i; C: device,
 * mc vectors of n elements, overwritten.  1 <= ma <= 112, 1 <= mc <= 128.
 * Allocates and frees its own device buffers; MB_EINVAL for bad sizes. */
int mb_debug_combine_ff(const void *A, const double *Y, long long n, int ma, int mc, void *C, void *stream);

/* FP32 fused multiply-add throughput of `device` in TFLOP/s (2 flops per
 * FFMA): eight independent FFMA chains per thread, 2048 threads on every SM,
 * timed with CUDA events; the best of `reps` (1..100) launches after one
 * warm-up launch.  The denominator of the roofline of an FP32-ALU-bound
 * kernel.  Runs at whatever clocks the device is at (it changes no setting).
 * Allocates a small sink buffer; MB_EINVAL for bad arguments, MB_ECUDA if a
 * CUDA call fails.  Outputs may be NULL. */
int mb_probe_fp32_fma(int device, int reps, double *tflops, double *ms);

/* The same probe with FP64 FMA chains (fewer iterations: GB300's FP64 rate
 * is a small fraction of its FP32 rate). */
int mb_probe_fp64_fma(int device, int reps, double *tflops, double *ms);

#ifdef __cplusplus
}
#endif
#endif
