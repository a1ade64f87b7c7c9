// S X and S^-1 X for blocks of trial vectors (§II.B.1, Eqs. (7)-(8): S is
// G-diagonal and banded in j; S^-1 through the banded Cholesky factor
// S = L L^T of the G-independent S_z).
//
// S X: one CTA owns a (k-point, band, 32-column, RT-row) tile.  The tile's
// RT + 2 (kappa - 1) rows of X arrive in shared memory by TMA bulk copies
// (one row of 32 columns per copy, issued by the lanes of one warp and counted
// on one mbarrier), together with its RT padded band rows, so every byte of
// the tile is in flight from HBM at once.  Each of the NS threads of a column
// then forms RT / NS consecutive outputs from a sliding window; the row loop
// is unrolled, so the window slides by renaming, and a band row is read as
// 16-byte shared-memory loads (the same address across the warp).
//
// S^-1 X: one CTA owns a (k-point, band, block of CW disc columns) tile: the
// tile's nb rows of X arrive in shared memory by TMA bulk copies (one row of
// CW columns per copy, issued by the lanes of one warp and counted on one
// mbarrier), so the whole tile is in flight from HBM together.  Each thread
// then runs the forward and backward banded triangular solves of its column
// out of shared memory and writes Y directly (consecutive threads,
// consecutive columns: coalesced stores).
//
// Every k-point and band of a batch is one launch.
#include <algorithm>
#include <cstdint>

#include "apply_common.cuh"
#include "mb_internal.h"
#include "tc_gemm.cuh"

namespace mb {

struct BandK {
    const void *X;
    void *Y;
    int ng, ldg;
};

template <typename R> struct BandArgs {
    const R *coef;    // S: Sband padded to [nb][band_pad(K)]; S^-1: L with reciprocal diagonal [nb][K]
    int *err;         // set when the copies' bounded wait expired
    int nb;
    BandK d[kMaxK];
};

// one padded band row as 16-byte loads
template <typename R, int WP> __device__ __forceinline__ void band_row(const R *p, R (&c)[WP]) {
    if constexpr (sizeof(R) == 4) {
#pragma unroll
        for (int q = 0; q < WP / 4; ++q) {
            const float4 v = reinterpret_cast<const float4 *>(p)[q];
            c[4 * q] = v.x, c[4 * q + 1] = v.y, c[4 * q + 2] = v.z, c[4 * q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < WP / 2; ++q) {
            const double2 v = reinterpret_cast<const double2 *>(p)[q];
            c[2 * q] = v.x, c[2 * q + 1] = v.y;
        }
    }
}

// S X for one (k-point, band, 32-column, RT-row) tile, NS threads per column.
template <typename R, int KK, int NS, int RT>
__global__ void __launch_bounds__(32 * NS, sizeof(R) == 4 ? 16 : 8)
    band_S_kernel(const __grid_constant__ BandArgs<R> a) {
    typedef typename V2<R>::T R2;
    constexpr int H = KK - 1, W = 2 * KK - 1, WP = band_pad(KK), RS = RT / NS;
    static_assert(RT % NS == 0, "whole row runs per thread");
    extern __shared__ __align__(128) unsigned char bsm[];
    __shared__ uint64_t bar;
    const BandK &d = a.d[blockIdx.z];
    const int g0 = blockIdx.x * 32;
    if (g0 >= d.ldg) return;                     // the batch's widest k-point sizes the grid
    const int nb = a.nb, ldg = d.ldg;            // ldg and g0 are multiples of 32: whole 32-column rows
    const int ntile = (nb + RT - 1) / RT;
    const int b = blockIdx.y / ntile, tile = blockIdx.y % ntile;
    const int r0 = tile * RT, r1 = min(nb, r0 + RT);                  // output rows
    const int x0 = max(0, r0 - H), x1 = min(nb, r1 + H), nx = x1 - x0;   // rows read
    R2 *buf = reinterpret_cast<R2 *>(bsm);       // [RT + 2H][32]: row x0 + i at i
    R *cf = reinterpret_cast<R *>(buf + (size_t)(RT + 2 * H) * 32);   // [RT][WP]
    const R2 *X = reinterpret_cast<const R2 *>(d.X) + ((size_t)b * nb + x0) * ldg + g0;
    constexpr uint32_t bytes = 32 * sizeof(R2);
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        // warp 0: the byte count first, then the row copies spread over the lanes
        if (threadIdx.x == 0)
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(&bar)),
                         "r"(bytes * (uint32_t)nx)
                         : "memory");
        __syncwarp();
        for (int j = threadIdx.x; j < nx; j += 32)
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    tc::smem_u32(buf + (size_t)j * 32)),
                "l"(X + (size_t)j * ldg), "r"(bytes), "r"(tc::smem_u32(&bar))
                : "memory");
    }
    {   // the tile's band rows (16-byte copies) while the rows are in flight
        const float4 *src = reinterpret_cast<const float4 *>(a.coef + (size_t)r0 * WP);
        float4 *dst = reinterpret_cast<float4 *>(cf);
        const int n16 = (int)((size_t)(r1 - r0) * WP * sizeof(R) / 16);
        for (int e = threadIdx.x; e < n16; e += 32 * NS) dst[e] = __ldg(src + e);
    }
    __syncthreads();
    if (!tc::mbar_wait(&bar, 0, 1ll << 24)) {    // every row of the tile is in shared memory
        if (threadIdx.x == 0) atomicExch(a.err, 1);
        return;
    }
    const int c = threadIdx.x % 32, seg = threadIdx.x / 32;
    const int ja = r0 + seg * RS;                // this thread's rows: ja .. ja + RS - 1 (those < r1)
    R2 *y = reinterpret_cast<R2 *>(d.Y) + (size_t)b * nb * ldg + g0 + c;
    if (g0 + c >= d.ng) {                        // padding columns are written as zero
#pragma unroll
        for (int r = 0; r < RS; ++r)
            if (ja + r < r1) y[(size_t)(ja + r) * ldg] = czero<R2>();
        return;
    }
    const R2 *x = buf + c - (size_t)x0 * 32;     // x[row * 32]: rows x0 .. x1 - 1 of the column
    auto xrow = [&](int row) { return (row >= x0 && row < x1) ? x[(size_t)row * 32] : czero<R2>(); };
    R2 win[W];                                   // win[i] = X[j - H + i]
#pragma unroll
    for (int i = 0; i + 1 < W; ++i) win[i + 1] = xrow(ja - H + i);
#pragma unroll
    for (int r = 0; r < RS; ++r) {
        const int j = ja + r;
#pragma unroll
        for (int i = 0; i + 1 < W; ++i) win[i] = win[i + 1];
        win[W - 1] = xrow(j + H);
        if (j < r1) {
            R cj[WP];
            band_row<R, WP>(cf + (size_t)(j - r0) * WP, cj);
            R2 v = czero<R2>();
#pragma unroll
            for (int i = 0; i < W; ++i) rfma(v, cj[i], win[i]);
            y[(size_t)j * ldg] = v;
        }
    }
}

// S^-1 X for one (k-point, band, CW-column) tile: L y = x (forward), then
// L^T z = y (backward), L[j][j-dd] at coef[j K + dd] with 1 / L[j][j] at
// dd = 0; the whole column in shared memory, y overwriting x there.
template <typename R, int KK, int CW>
__global__ void __launch_bounds__(CW) band_Sinv_kernel(const __grid_constant__ BandArgs<R> a) {
    typedef typename V2<R>::T R2;
    extern __shared__ __align__(128) unsigned char bsm[];
    __shared__ uint64_t bar;
    const BandK &d = a.d[blockIdx.z];
    const int g0 = blockIdx.x * CW;
    if (g0 >= d.ldg) return;                     // the batch's widest k-point sizes the grid
    const int nb = a.nb, ldg = d.ldg, ncol = min(CW, ldg - g0);
    const int b = blockIdx.y;
    R2 *buf = reinterpret_cast<R2 *>(bsm);       // [nb][CW]
    R *cf = reinterpret_cast<R *>(buf + (size_t)nb * CW);
    const R2 *X = reinterpret_cast<const R2 *>(d.X) + (size_t)b * nb * ldg + g0;
    R2 *Y = reinterpret_cast<R2 *>(d.Y) + (size_t)b * nb * ldg + g0;
    const uint32_t bytes = (uint32_t)(ncol * sizeof(R2));   // ldg and g0 are multiples of 32 columns
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        // warp 0: the byte count first, then the row copies spread over the lanes
        if (threadIdx.x == 0)
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(&bar)),
                         "r"(bytes * (uint32_t)nb)
                         : "memory");
        __syncwarp();
        for (int j = threadIdx.x; j < nb; j += 32)
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    tc::smem_u32(buf + (size_t)j * CW)),
                "l"(X + (size_t)j * ldg), "r"(bytes), "r"(tc::smem_u32(&bar))
                : "memory");
    }
    // the factor's coefficients while the rows are in flight
    for (int e = threadIdx.x; e < nb * KK; e += CW) cf[e] = a.coef[e];
    __syncthreads();
    if (!tc::mbar_wait(&bar, 0, 1ll << 24)) {    // every row of the tile is in shared memory
        if (threadIdx.x == 0) atomicExch(a.err, 1);
        return;
    }
    const int c = threadIdx.x;
    if (c >= ncol) return;
    const int g = g0 + c;
    R2 *y = Y + c;
    if (g >= d.ng) {                             // padding columns are written as zero
        for (int j = 0; j < nb; ++j) y[(size_t)j * ldg] = czero<R2>();
        return;
    }
    R2 *xw = buf + c;
    R2 w[KK - 1];                                // w[dd-1] = y[j - dd]
#pragma unroll
    for (int i = 0; i < KK - 1; ++i) w[i] = czero<R2>();
    for (int j = 0; j < nb; ++j) {
        const R *lj = cf + (size_t)j * KK;
        R2 s = xw[(size_t)j * CW];
        // oldest term first: only the last FMA waits on y[j-1]
#pragma unroll
        for (int dd = KK - 1; dd >= 1; --dd) rfma(s, -lj[dd], w[dd - 1]);   // w = 0 before row 0
        const R2 yj = rscale(lj[0], s);
        xw[(size_t)j * CW] = yj;
#pragma unroll
        for (int i = KK - 2; i > 0; --i) w[i] = w[i - 1];
        w[0] = yj;
    }
#pragma unroll
    for (int i = 0; i < KK - 1; ++i) w[i] = czero<R2>();
    for (int j = nb - 1; j >= 0; --j) {
        R2 s = xw[(size_t)j * CW];
#pragma unroll
        for (int dd = KK - 1; dd >= 1; --dd)
            if (j + dd < nb) rfma(s, -cf[(size_t)(j + dd) * KK + dd], w[dd - 1]);
        const R2 zj = rscale(cf[(size_t)j * KK], s);
        y[(size_t)j * ldg] = zj;
#pragma unroll
        for (int i = KK - 2; i > 0; --i) w[i] = w[i - 1];
        w[0] = zj;
    }
}

constexpr int kBandCW = 32;        // columns per S^-1 tile (FP32 and FP64)
constexpr int kBandRT = 32;        // output rows per S tile
constexpr int kBandNS = 2;         // threads per column of an S tile

// Shared memory of one S^-1 tile, or 0 when it does not fit.
static size_t sinv_smem(const mb_handle *h, size_t c2) {
    const size_t bytes = (size_t)h->nb * kBandCW * c2 + (size_t)h->nb * h->order * (c2 / 2);
    return bytes <= (size_t)h->smem_optin ? bytes : 0;
}

bool banded_block_supported(const mb_handle *h, int prec, bool inv) {
    if (!inv) return h->order >= 3 && h->order <= 8;
    const size_t c2 = prec == MB_FP64 ? 16 : 8;
    return h->order == 6 && sinv_smem(h, c2) > 0 && h->nb >= 4;
}

template <typename R>
static void band_args(const mb_handle *h, bool inv, int nsel, const int *iks, const void *const *X,
                      void *const *Y, BandArgs<R> &a, int &maxldg) {
    const DevTables &t = sizeof(R) == 4 ? h->t32 : h->t64;
    a.coef = reinterpret_cast<const R *>(inv ? t.Lrecip : t.SbandP);
    a.err = reinterpret_cast<int *>(h->d_tcerr);
    a.nb = h->nb;
    maxldg = 0;
    for (int i = 0; i < nsel; ++i) {
        const KPoint &kp = h->kp[iks[i]];
        a.d[i].X = X[i];
        a.d[i].Y = Y[i];
        a.d[i].ng = kp.ng;
        a.d[i].ldg = kp.ldg;
        maxldg = std::max(maxldg, kp.ldg);
    }
}

template <typename R>
static int launch_S(mb_handle *h, int nsel, const int *iks, const void *const *X, void *const *Y, int nbands,
                    cudaStream_t s) {
    BandArgs<R> a;
    int maxldg;
    band_args<R>(h, false, nsel, iks, X, Y, a, maxldg);
    const int K = h->order;
    const size_t smem = (size_t)(kBandRT + 2 * (K - 1)) * 32 * sizeof(typename V2<R>::T) +
                        (size_t)kBandRT * band_pad(K) * sizeof(R);
    const int ntile = (h->nb + kBandRT - 1) / kBandRT;
    const dim3 grid((maxldg + 31) / 32, nbands * ntile, nsel);
    cudaEvent_t ev;
    prof_begin(h, s, KN_BANDED, &ev);
    switch (K) {
#define MB_BAND_S(KK) \
    case KK: band_S_kernel<R, KK, kBandNS, kBandRT><<<grid, 32 * kBandNS, smem, s>>>(a); break;
        MB_BAND_S(3) MB_BAND_S(4) MB_BAND_S(5) MB_BAND_S(6) MB_BAND_S(7) MB_BAND_S(8)
#undef MB_BAND_S
    }
    prof_end(h, s, KN_BANDED, ev);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MB_OK : cuda_fail(h, e);
}

template <typename R>
static int launch_Sinv(mb_handle *h, int nsel, const int *iks, const void *const *X, void *const *Y, int nbands,
                       cudaStream_t s) {
    BandArgs<R> a;
    int maxldg;
    band_args<R>(h, true, nsel, iks, X, Y, a, maxldg);
    const size_t smem = sinv_smem(h, sizeof(typename V2<R>::T));
    const void *fn = (const void *)band_Sinv_kernel<R, 6, kBandCW>;
    cudaError_t e = smem_limit_once(fn, h->device, h->smem_optin);
    if (e != cudaSuccess) return cuda_fail(h, e);
    const dim3 grid((maxldg + kBandCW - 1) / kBandCW, nbands, nsel);
    cudaEvent_t ev;
    prof_begin(h, s, KN_BANDED, &ev);
    band_Sinv_kernel<R, 6, kBandCW><<<grid, kBandCW, smem, s>>>(a);
    prof_end(h, s, KN_BANDED, ev);
    e = cudaGetLastError();
    return e == cudaSuccess ? MB_OK : cuda_fail(h, e);
}

int banded_block_apply(mb_handle *h, bool inv, int nsel, const int *iks, const void *const *X, void *const *Y,
                       int nbands, int prec, cudaStream_t s) {
    for (int i0 = 0; i0 < nsel; i0 += kMaxK) {
        const int n = std::min(kMaxK, nsel - i0);
        int rc;
        if (prec == MB_FP64)
            rc = inv ? launch_Sinv<double>(h, n, iks + i0, X + i0, Y + i0, nbands, s)
                     : launch_S<double>(h, n, iks + i0, X + i0, Y + i0, nbands, s);
        else
            rc = inv ? launch_Sinv<float>(h, n, iks + i0, X + i0, Y + i0, nbands, s)
                     : launch_S<float>(h, n, iks + i0, X + i0, Y + i0, nbands, s);
        if (rc) return rc;
    }
    return MB_OK;
}

}  // namespace mb
