// S X and S^-1 X for blocks of trial vectors (§II.B.1, Eqs. (7)-(8): S is
// G-diagonal and banded in j; S^-1 through the banded Cholesky factor
// S = L L^T of the G-independent S_z).
//
// One CTA owns a (k-point, band, block of CW disc columns) tile: the tile's nb
// rows of X arrive in shared memory by TMA bulk copies (one row of CW columns
// per copy, all issued at once by one thread and counted on one mbarrier), so
// the whole tile is in flight from HBM together.  Each thread then runs its
// column out of shared memory -- the 2 kappa - 1 diagonals of S, or the
// forward and backward banded triangular solves -- and writes Y directly
// (consecutive threads, consecutive columns: coalesced stores).  Every
// k-point and band of a batch is one launch.
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
    const R *coef;    // S: Sband [nb][2K-1]; S^-1: L with reciprocal diagonal [nb][K]
    int *err;         // set when the copies' bounded wait expired
    int nb;
    BandK d[kMaxK];
};

// NS: threads per column -- S splits each column's rows into NS segments
// (no recurrence), S^-1 keeps one thread per column (NS = 1).
// RT: rows of X per CTA for S (0: all; S^-1 needs all rows of a column):
// the tile holds rows [r0 - (K-1), r1 + K-1) of its RT output rows.
template <typename R, bool INV, int KK, int CW, int NS, int RT>
__global__ void __launch_bounds__(CW * NS) banded_block_kernel(const __grid_constant__ BandArgs<R> a) {
    typedef typename V2<R>::T R2;
    constexpr int W = 2 * KK - 1, NC = INV ? KK : W;
    extern __shared__ __align__(128) unsigned char bsm[];
    __shared__ uint64_t bar;
    const BandK &d = a.d[blockIdx.z];
    const int g0 = blockIdx.x * CW;
    if (g0 >= d.ldg) return;                     // the batch's widest k-point sizes the grid
    const int nb = a.nb, ldg = d.ldg, ncol = min(CW, ldg - g0);
    const int ntile = RT ? (nb + RT - 1) / RT : 1;
    const int b = blockIdx.y / ntile, tile = blockIdx.y % ntile;
    const int r0 = RT ? tile * RT : 0, r1 = RT ? min(nb, r0 + RT) : nb;          // output rows
    const int x0 = RT ? max(0, r0 - (KK - 1)) : 0, x1 = RT ? min(nb, r1 + KK - 1) : nb;   // rows read
    const int nx = x1 - x0;
    R2 *buf = reinterpret_cast<R2 *>(bsm);       // [nx][CW]: row x0 + i at i
    R *cf = reinterpret_cast<R *>(buf + (size_t)(RT ? RT + 2 * (KK - 1) : nb) * CW);
    const R2 *X = reinterpret_cast<const R2 *>(d.X) + ((size_t)b * nb + x0) * ldg + g0;
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
                         "r"(bytes * (uint32_t)nx)
                         : "memory");
        __syncwarp();
        for (int j = threadIdx.x; j < nx; j += 32)
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    tc::smem_u32(buf + (size_t)j * CW)),
                "l"(X + (size_t)j * ldg), "r"(bytes), "r"(tc::smem_u32(&bar))
                : "memory");
    }
    // band coefficients of the output rows while the rows are in flight
    for (int e = threadIdx.x; e < (r1 - r0) * NC; e += CW * NS) cf[e] = a.coef[(size_t)r0 * NC + e];
    __syncthreads();
    if (!tc::mbar_wait(&bar, 0, 1ll << 24)) {    // every row of the tile is in shared memory
        if (threadIdx.x == 0) atomicExch(a.err, 1);
        return;
    }
    const int c = threadIdx.x % CW, seg = threadIdx.x / CW;
    if (c >= ncol) return;
    const int g = g0 + c;
    R2 *y = Y + c;
    const int ja = r0 + (seg * (r1 - r0)) / NS, jb = r0 + ((seg + 1) * (r1 - r0)) / NS;   // this thread's rows
    if (g >= d.ng) {                             // padding columns are written as zero
        for (int j = ja; j < jb; ++j) y[(size_t)j * ldg] = czero<R2>();
        return;
    }
    const R2 *x = buf + c - (size_t)x0 * CW;      // x[row * CW]: row of the whole column
    if constexpr (!INV) {
        // Y[j] = sum_{o=-(K-1)}^{K-1} S[j][j+o] X[j+o]: a window of 2K-1 rows in registers
        R2 win[W];
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const int row = ja + i - (KK - 1);
            win[i] = (row >= 0 && row < nb) ? x[(size_t)row * CW] : czero<R2>();
        }
        for (int j = ja; j < jb; ++j) {
            const R *sj = cf + (size_t)(j - r0) * W;
            R2 v = czero<R2>();
#pragma unroll
            for (int i = 0; i < W; ++i) rfma(v, sj[i], win[i]);
            y[(size_t)j * ldg] = v;
#pragma unroll
            for (int i = 0; i + 1 < W; ++i) win[i] = win[i + 1];
            const int nx = j + KK;
            win[W - 1] = nx < nb ? x[(size_t)nx * CW] : czero<R2>();
        }
    } else {
        // L y = x (forward), then L^T z = y (backward); L[j][j-dd] at cf[j K + dd],
        // 1 / L[j][j] at dd = 0.  y overwrites x in shared memory.
        R2 *xw = buf + c;
        R2 w[KK - 1];                            // w[dd-1] = y[j - dd]
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
}

// Shared memory of one tile, or 0 when the tile does not fit.
constexpr int kBandRowTile = 32;   // output rows per S tile

static size_t band_smem(const mb_handle *h, size_t c2, int cw, bool inv) {
    const int K = h->order, nc = inv ? K : 2 * K - 1;
    const int rows = inv ? h->nb : kBandRowTile + 2 * (K - 1), crow = inv ? h->nb : kBandRowTile;
    const size_t bytes = (size_t)rows * cw * c2 + (size_t)crow * nc * (c2 / 2);
    return bytes <= (size_t)h->smem_optin ? bytes : 0;
}

bool banded_block_supported(const mb_handle *h, int prec, bool inv) {
    if (h->order != 6) return false;
    const size_t c2 = prec == MB_FP64 ? 16 : 8;
    return band_smem(h, c2, 32, inv) > 0 && h->nb >= 4;
}

template <typename R, bool INV>
static int launch_band(mb_handle *h, int nsel, const int *iks, const void *const *X, void *const *Y, int nbands,
                       cudaStream_t s) {
    constexpr int CW = 32;   // columns per tile (FP32 and FP64)
    const DevTables &t = sizeof(R) == 4 ? h->t32 : h->t64;
    BandArgs<R> a;
    a.coef = reinterpret_cast<const R *>(INV ? t.Lrecip : t.Sband);
    a.err = reinterpret_cast<int *>(h->d_tcerr);
    a.nb = h->nb;
    int maxldg = 0;
    for (int i = 0; i < nsel; ++i) {
        const KPoint &kp = h->kp[iks[i]];
        a.d[i].X = X[i];
        a.d[i].Y = Y[i];
        a.d[i].ng = kp.ng;
        a.d[i].ldg = kp.ldg;
        maxldg = std::max(maxldg, kp.ldg);
    }
    const size_t smem = band_smem(h, sizeof(typename V2<R>::T), CW, INV);
    constexpr int NS = INV ? 1 : 2, RT = INV ? 0 : kBandRowTile;
    const void *fn = (const void *)banded_block_kernel<R, INV, 6, CW, NS, RT>;
    cudaError_t e = smem_limit_once(fn, h->device, h->smem_optin);
    if (e != cudaSuccess) return cuda_fail(h, e);
    const int ntile = RT ? (h->nb + RT - 1) / RT : 1;
    const dim3 grid((maxldg + CW - 1) / CW, nbands * ntile, nsel);
    cudaEvent_t ev;
    prof_begin(h, s, KN_BANDED, &ev);
    banded_block_kernel<R, INV, 6, CW, NS, RT><<<grid, CW * NS, smem, s>>>(a);
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
            rc = inv ? launch_band<double, true>(h, n, iks + i0, X + i0, Y + i0, nbands, s)
                     : launch_band<double, false>(h, n, iks + i0, X + i0, Y + i0, nbands, s);
        else
            rc = inv ? launch_band<float, true>(h, n, iks + i0, X + i0, Y + i0, nbands, s)
                     : launch_band<float, false>(h, n, iks + i0, X + i0, Y + i0, nbands, s);
        if (rc) return rc;
    }
    return MB_OK;
}

}  // namespace mb
