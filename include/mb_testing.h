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

#ifdef __cplusplus
}
#endif
#endif
