// BF16 tensor-core GEMM on sm_103a (tcgen05 + TMEM), FP32 accumulation.
//
//   D[M x N] = A[M x K] * Bt[N x K]^T        (both operands K-major)
//
// One CTA of 128 threads computes a 128-row tile of D for one N tile
// (16 <= N_tile <= 256, a multiple of 16) with the accumulator in tensor
// memory.  Per K chunk of 64 the CTA stages A and B into shared memory in the
// canonical K-major layout without swizzle (8 x 16-byte core matrices:
// element (r, k) at (r/8)*SBO + (k/8)*LBO + (r%8)*16 + (k%8)*2), one elected
// thread issues four tcgen05.mma (K = 16 each) and commits them to an
// mbarrier that the CTA waits on (bounded) before the next chunk overwrites
// the operands.  The epilogue reads the accumulator with tcgen05.ld: warp w
// owns TMEM lanes (= rows) 32w .. 32w+31.
//
// Operand producers are functors so that callers stage from their own data
// (FP32 complex coefficient rows converted to BF16 for the projector
// contractions, plain BF16 arrays for the self-test).
#include <cuda_bf16.h>

#include "apply_common.cuh"
#include "mb_internal.h"

#include "tc_gemm.cuh"

namespace mb {
namespace tc {

// ---- self-test kernel: plain BF16 operands (A row-major M x K, Bt N x K)
__global__ void __launch_bounds__(128) gemm_bf16_kernel(const __nv_bfloat16 *A, const __nv_bfloat16 *Bt, float *D,
                                                        int M, int N, int K, int ntile, int *err) {
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * ntile;
    auto la = [&](int r, int k) -> __nv_bfloat162 {
        __nv_bfloat162 v;
        v.x = (r < M && k < K) ? A[(size_t)r * K + k] : __float2bfloat16(0.f);
        v.y = (r < M && k + 1 < K) ? A[(size_t)r * K + k + 1] : __float2bfloat16(0.f);
        return v;
    };
    auto lb = [&](int r, int k) -> __nv_bfloat162 {
        __nv_bfloat162 v;
        v.x = (r < N && k < K) ? Bt[(size_t)r * K + k] : __float2bfloat16(0.f);
        v.y = (r < N && k + 1 < K) ? Bt[(size_t)r * K + k + 1] : __float2bfloat16(0.f);
        return v;
    };
    auto st = [&](int r, int c, float x) { D[(size_t)r * N + c] = x; };
    gemm_tile(M, N, K, m0, n0, ntile, la, lb, st, err);
}

size_t smem_bytes(int ntile) { return (size_t)(128 + ntile) * 64 * 2 + 1024; }

// ---- Kleinman-Bylander contractions on the tensor cores (MB_BF16 applies)
//
// Complex products become real ones on interleaved (re, im) rows.
//  projection       W[m][p] = sum_G X[m][G] conj(q_p(G)):  A = X rows (K = 2 ng),
//                   Bt0[2p + c][2G + c'] = real 2x2 block of conj(q_p(G))
//  back-projection  Y[m][G] += sum_p C[m][p] q_p(G):       A = C rows (K = 2 nterm),
//                   Bt1[2G + c][2p + c'] = real 2x2 block of q_p(G)
// with m = (band, j).  Both B matrices are BF16 tables built once per k-point.
struct ProjArgs {
    const __nv_bfloat16 *B;   // all k: per k at bofs[k]
    int mode, nb, nbands, nterm;
    int *err;
    KDesc d[kMaxK];
    int bofs[kMaxK];          // element offset of this k-point's B table
    int bld[kMaxK];           // its row length (K of the GEMM, padded to 16)
};

__global__ void __launch_bounds__(128) proj_tc_kernel(const __grid_constant__ ProjArgs a, int ntile) {
    const int ks = blockIdx.z;
    const KDesc &d = a.d[ks];
    const int M = a.nbands * a.nb;
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * ntile;
    const int N = a.mode == 0 ? 2 * a.nterm : 2 * d.ng;
    if (n0 >= N) return;
    const int K = a.mode == 0 ? 2 * d.ng : 2 * a.nterm;
    const int lda = a.mode == 0 ? d.ldg : a.nterm;          // complex elements per A row
    const float2 *Ar = reinterpret_cast<const float2 *>(a.mode == 0 ? d.X : d.C);
    const __nv_bfloat16 *B = a.B + a.bofs[ks];
    const int ldb = a.bld[ks];
    auto la = [&](int r, int k) -> __nv_bfloat162 {    // k even: (re, im) of element k/2
        float2 v = (r < M && k < K) ? Ar[(size_t)r * lda + k / 2] : make_float2(0.f, 0.f);
        return __floats2bfloat162_rn(v.x, v.y);
    };
    auto lb = [&](int r, int k) -> __nv_bfloat162 {
        if (r >= N || k >= K) return __floats2bfloat162_rn(0.f, 0.f);
        return *reinterpret_cast<const __nv_bfloat162 *>(B + (size_t)r * ldb + k);
    };
    float *out = reinterpret_cast<float *>(a.mode == 0 ? d.W : d.Y);
    const int ldo = a.mode == 0 ? 2 * a.nterm : 2 * d.ldg;
    auto st = [&](int r, int c, float x) {
        if (a.mode == 0) out[(size_t)r * ldo + c] = x;
        else out[(size_t)r * ldo + c] += x;
    };
    gemm_tile(M, N, K, m0, n0, ntile, la, lb, st, a.err);
}

}  // namespace tc
}  // namespace mb

namespace mb {

// host: the BF16 B tables of every k-point (uploaded once per handle)
int upload_proj_tables(mb_handle *h) {
    if (h->nterm == 0) return MB_OK;
    const int NP = h->nterm;
    std::vector<__nv_bfloat16> all;
    h->pb0_ofs.assign(h->kp.size(), 0);
    h->pb1_ofs.assign(h->kp.size(), 0);
    h->pb0_ld.assign(h->kp.size(), 0);
    h->pb1_ld.assign(h->kp.size(), 0);
    for (size_t ik = 0; ik < h->kp.size(); ++ik) {
        const KPoint &kp = h->kp[ik];
        const int K0 = (2 * kp.ng + 15) / 16 * 16, K1 = (2 * NP + 15) / 16 * 16;
        // projection: rows 2p + c, columns 2G + c'; conj(q) = (qr, -qi)
        h->pb0_ofs[ik] = (int)all.size();
        h->pb0_ld[ik] = K0;
        std::vector<__nv_bfloat16> b0((size_t)2 * NP * K0, __float2bfloat16(0.f));
        for (int p = 0; p < NP; ++p)
            for (int g = 0; g < kp.ng; ++g) {
                const cdouble q = kp.qproj[(size_t)p * kp.ldg + g];
                const float qr = (float)q.real(), qi = (float)q.imag();
                // re row:  xr*qr + xi*qi ;  im row: -xr*qi + xi*qr
                b0[(size_t)(2 * p) * K0 + 2 * g] = __float2bfloat16(qr);
                b0[(size_t)(2 * p) * K0 + 2 * g + 1] = __float2bfloat16(qi);
                b0[(size_t)(2 * p + 1) * K0 + 2 * g] = __float2bfloat16(-qi);
                b0[(size_t)(2 * p + 1) * K0 + 2 * g + 1] = __float2bfloat16(qr);
            }
        all.insert(all.end(), b0.begin(), b0.end());
        // back-projection: rows 2G + c, columns 2p + c'
        h->pb1_ofs[ik] = (int)all.size();
        h->pb1_ld[ik] = K1;
        std::vector<__nv_bfloat16> b1((size_t)2 * kp.ldg * K1, __float2bfloat16(0.f));
        for (int g = 0; g < kp.ng; ++g)
            for (int p = 0; p < NP; ++p) {
                const cdouble q = kp.qproj[(size_t)p * kp.ldg + g];
                const float qr = (float)q.real(), qi = (float)q.imag();
                // re: cr*qr - ci*qi ;  im: cr*qi + ci*qr
                b1[(size_t)(2 * g) * K1 + 2 * p] = __float2bfloat16(qr);
                b1[(size_t)(2 * g) * K1 + 2 * p + 1] = __float2bfloat16(-qi);
                b1[(size_t)(2 * g + 1) * K1 + 2 * p] = __float2bfloat16(qi);
                b1[(size_t)(2 * g + 1) * K1 + 2 * p + 1] = __float2bfloat16(qr);
            }
        all.insert(all.end(), b1.begin(), b1.end());
    }
    // uploaded on the handle's stream (upload_tables waits for it before returning)
    return dev_upload(h, &h->d_projB, all.data(), all.size() * sizeof(__nv_bfloat16));
}

// one projector contraction for a group of k-points (mode 0 or 1)
cudaError_t proj_tc_launch(mb_handle *h, int mode, int nsel, const int *iks, const KDesc *desc, int nbands,
                           cudaStream_t s) {
    tc::ProjArgs a;
    a.B = reinterpret_cast<const __nv_bfloat16 *>(h->d_projB);
    a.mode = mode;
    a.nb = h->nb;
    a.nbands = nbands;
    a.nterm = h->nterm;
    a.err = reinterpret_cast<int *>(h->d_tcerr);
    int maxN = 0;
    for (int i = 0; i < nsel; ++i) {
        a.d[i] = desc[i];
        a.bofs[i] = mode == 0 ? h->pb0_ofs[iks[i]] : h->pb1_ofs[iks[i]];
        a.bld[i] = mode == 0 ? h->pb0_ld[iks[i]] : h->pb1_ld[iks[i]];
        maxN = std::max(maxN, mode == 0 ? 2 * h->nterm : 2 * h->kp[iks[i]].ng);
    }
    const int ntile = maxN <= 256 ? (maxN + 15) / 16 * 16 : 256;
    const dim3 grid((nbands * h->nb + 127) / 128, (maxN + ntile - 1) / ntile, nsel);
    const size_t smem = tc::smem_bytes(ntile);
    cudaError_t e = smem_limit_once((const void *)tc::proj_tc_kernel, h->device, h->smem_optin);
    if (e != cudaSuccess) return e;
    tc::proj_tc_kernel<<<grid, 128, smem, s>>>(a, ntile);
    return cudaGetLastError();
}

}  // namespace mb

using namespace mb;

extern "C" int mb_debug_gemm_bf16(const void *A, const void *Bt, float *D, int M, int N, int K, void *stream) {
    if (!A || !Bt || !D || M < 1 || N < 1 || K < 1) return MB_EINVAL;
    int ntile = N <= 256 ? (N + 15) / 16 * 16 : 128;
    const dim3 grid((M + 127) / 128, (N + ntile - 1) / ntile);
    int *err = nullptr;
    if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) return MB_ENOMEM;
    cudaMemsetAsync(err, 0, sizeof(int), (cudaStream_t)stream);
    const size_t smem = tc::smem_bytes(ntile);
    cudaFuncSetAttribute(tc::gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    tc::gemm_bf16_kernel<<<grid, 128, smem, (cudaStream_t)stream>>>(
        reinterpret_cast<const __nv_bfloat16 *>(A), reinterpret_cast<const __nv_bfloat16 *>(Bt), D, M, N, K, ntile,
        err);
    cudaError_t e = cudaGetLastError();
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(err);
    if (e != cudaSuccess) return MB_ECUDA;
    return herr ? MB_ETIMEOUT : MB_OK;
}
