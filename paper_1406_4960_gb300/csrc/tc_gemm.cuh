// tcgen05 BF16 GEMM tile (device code shared by the projector contractions
// and the self-test); see tc_gemm.cu for the description.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

namespace mb {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;          // descriptor version for tcgen05
    return d;                        // base offset 0, no swizzle
}

// kind::f16 instruction descriptor: D F32, A BF16, B BF16, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded wait for the given phase: at most `limit` polls and one second;
// false when either limit was reached
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t phase, long long limit) {
    const uint32_t a = smem_u32(bar);
    const uint64_t start = global_ns();
    for (long long it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(phase));
        if (done) return true;
        if (global_ns() - start > 1000000000ull) return false;
    }
    return false;
}

template <class LoadA, class LoadB, class Store>
__device__ void gemm_tile(int M, int N, int K, int m0, int n0, int ntile, LoadA loadA, LoadB loadB, Store store,
                          int *err) {
    constexpr int BK = 64;
    constexpr int LBO = 128;                 // next core matrix along K
    constexpr int SBO = (BK / 8) * 128;      // next 8 rows
    extern __shared__ __align__(1024) unsigned char sm[];
    __nv_bfloat16 *As = reinterpret_cast<__nv_bfloat16 *>(sm);            // 128 x BK
    __nv_bfloat16 *Bs = As + 128 * BK;                                     // ntile x BK
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int failed;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int ncols = 32;
    while (ncols < ntile) ncols <<= 1;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mbar_init(&mbar, 1);
        failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = idesc_bf16(128, ntile);
    uint32_t phase = 0;
    const int nk16 = (K + 15) / 16;
    for (int k0 = 0; k0 < K; k0 += BK) {
        // stage A (128 x BK) and B (ntile x BK); zero outside the matrices
        for (int e = tid; e < 128 * (BK / 2); e += blockDim.x) {
            const int r = e / (BK / 2), kp = e % (BK / 2);
            const int k = 2 * kp;
            __nv_bfloat162 v = loadA(m0 + r, k0 + k);
            const int off = (r / 8) * SBO + (k / 8) * LBO + (r % 8) * 16 + (k % 8) * 2;
            *reinterpret_cast<__nv_bfloat162 *>(reinterpret_cast<unsigned char *>(As) + off) = v;
        }
        for (int e = tid; e < ntile * (BK / 2); e += blockDim.x) {
            const int r = e / (BK / 2), kp = e % (BK / 2);
            const int k = 2 * kp;
            __nv_bfloat162 v = loadB(n0 + r, k0 + k);
            const int off = (r / 8) * SBO + (k / 8) * LBO + (r % 8) * 16 + (k % 8) * 2;
            *reinterpret_cast<__nv_bfloat162 *>(reinterpret_cast<unsigned char *>(Bs) + off) = v;
        }
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) {
            const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
            for (int kk = 0; kk < BK / 16; ++kk) {
                const int kstep = k0 / 16 + kk;
                if (kstep >= nk16) break;
                const uint64_t ad = smem_desc(a0 + kk * 2 * LBO, LBO, SBO);
                const uint64_t bd = smem_desc(b0 + kk * 2 * LBO, LBO, SBO);
                const uint32_t acc = (kstep > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&mbar)));
        }
        if (!mbar_wait(&mbar, phase, 1ll << 24)) {
            if (tid == 0) {
                failed = 1;
                atomicExch(err, 1);
            }
        }
        phase ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;");
        __syncthreads();
        if (failed) break;
    }
    if (!failed) {
        // epilogue: warp w reads rows 32w + lane, 8 columns per tcgen05.ld
        const int row = m0 + 32 * warp + lane;
        for (int c0 = 0; c0 < ntile; c0 += 8) {
            uint32_t v[8];
            const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                           "=r"(v[7])
                         : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (row < M)
                for (int j = 0; j < 8; ++j)
                    if (n0 + c0 + j < N) store(row, n0 + c0 + j, __uint_as_float(v[j]));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

}  // namespace tc
}  // namespace mb
