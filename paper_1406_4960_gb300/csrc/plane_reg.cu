// Local-potential plane kernel with register-resident FFT lines.
//
// Same computation as the radix-2 plane kernel in apply.cu (B-spline
// evaluation on the Gauss planes, inverse 2D FFT, product with
// w_q V(r, z_q) / (N1 N2), forward 2D FFT, adjoint B-spline sum), organised
// for throughput:
//  * every 1D transform of N <= 64 points runs inside one thread's registers
//    (radix-2, bit reversal by register renaming, trivial twiddles folded at
//    compile time, six fused multiply-adds per butterfly with a nontrivial
//    twiddle), so a plane crosses shared memory three times per direction
//    instead of once per butterfly stage;
//  * planes are stored with rows padded to N2 + 1 so that row-wise and
//    column-wise line loads are both free of bank conflicts;
//  * the inverse column transform, the potential product and the forward
//    column transform are fused in registers;
//  * rows of the grid that hold no point of the cutoff disc are skipped in
//    both row passes (their inverse input and their forward output are not
//    needed);
//  * a CTA serves `bt` bands of one k-point over a run of knot intervals and
//    keeps their kappa output rows in a shared-memory ring, exactly like the
//    radix-2 kernel (same boundary-row protocol and scratch layout).
#include <cstdio>

#include "apply_common.cuh"
#include "mb_internal.h"

namespace mb {

// Twiddles of the in-register transforms, in the scaled form of the radix-2
// butterfly with fused multiply-adds (Linzer & Feig, 1993): the twiddle
// w = cos a + i sin a of angle a = 2 pi k / 64 is stored as w = c (1 + i r)
// with (c, r) = (cos a, tan a) where |cos a| >= |sin a|, else as
// w = c (r + i) with (c, r) = (sin a, cot a).  Then a +- w b costs two fused
// multiply-adds for t = b (1 + i r) (or b (r + i)) and four for a +- c t:
// six per butterfly instead of eight for a complex product and two complex
// additions, with |r| <= 1 so that no term is amplified.
__constant__ float2 c_tsf[64];
__constant__ double2 c_tsd[64];

constexpr bool tw_tan_form(int k) { return (k % 32) <= 8 || (k % 32) >= 24; }

void upload_fft_twiddles() {
    float2 tf[64];
    double2 td[64];
    for (int k = 0; k < 64; ++k) {
        const double a = 2.0 * 3.14159265358979323846 * k / 64.0;
        const double c = std::cos(a), s = std::sin(a);
        td[k] = tw_tan_form(k) ? make_double2(c, s / c) : make_double2(s, c / s);
        tf[k] = make_float2((float)td[k].x, (float)td[k].y);
    }
    cudaMemcpyToSymbol(c_tsf, tf, sizeof(tf));
    cudaMemcpyToSymbol(c_tsd, td, sizeof(td));
}

template <typename C> __device__ __forceinline__ C ctws(int k);
template <> __device__ __forceinline__ float2 ctws<float2>(int k) { return c_tsf[k]; }
template <> __device__ __forceinline__ double2 ctws<double2>(int k) { return c_tsd[k]; }

__device__ __forceinline__ float fmar(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmar(double a, double b, double c) { return fma(a, b, c); }

constexpr int brev_c(int x, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((x >> b) & 1) << (bits - 1 - b);
    return r;
}
constexpr int ilog2_c(int n) { return n <= 1 ? 0 : 1 + ilog2_c(n / 2); }

// (a, b) <- (a + w b, a - w b), w = exp(sign 2 pi i tk / N), sign = + for the
// inverse transform (the forward twiddle is the conjugate: r and, in the
// cot form, c change sign)
template <int N, bool INV, typename C>
__device__ __forceinline__ void bfly(C &a, C &b, int tk) {
    const C u = a;
    if (tk == 0) {
        a = u + b;
        b = u - b;
        return;
    }
    if (4 * tk == N) {
        const C wb = INV ? mk(-b.y, b.x) : mk(b.y, -b.x);
        a = u + wb;
        b = u - wb;
        return;
    }
    const int k = tk * (64 / N);
    const C q = ctws<C>(k);
    auto c = q.x, r = q.y;
    const bool tan_form = tw_tan_form(k);
    if (!INV) {
        r = -r;
        if (!tan_form) c = -c;
    }
    C t;
    if (tan_form) {
        t.x = fmar(-r, b.y, b.x);
        t.y = fmar(r, b.x, b.y);
    } else {
        t.x = fmar(r, b.x, -b.y);
        t.y = fmar(r, b.y, b.x);
    }
    a.x = fmar(c, t.x, u.x);
    a.y = fmar(c, t.y, u.y);
    b.x = fmar(-c, t.x, u.x);
    b.y = fmar(-c, t.y, u.y);
}

// true when every input index that reaches positions [p, p + len) of the
// bit-reversed array is >= nin (those positions hold zeros until the stage
// that merges them with a lower block)
constexpr bool zero_block(int p, int len, int bits, int nin) {
    for (int i = p; i < p + len; ++i)
        if (brev_c(i, bits) < nin) return false;
    return true;
}
// bit q: the lower half of butterfly group q of the stage of half-width
// `half` is all zeros
constexpr unsigned long long stage_zero_mask(int n, int half, int bits, int nin) {
    unsigned long long m = 0;
    for (int g = 0; g < n; g += 2 * half)
        if (nin < n && zero_block(g + half, half, bits, nin)) m |= 1ull << (g / (2 * half));
    return m;
}

template <int N, bool INV, int NIN, int HALF, typename C>
__device__ __forceinline__ void fft_stages(C (&x)[N]) {
    constexpr unsigned long long zm = stage_zero_mask(N, HALF, ilog2_c(N), NIN);
#pragma unroll
    for (int g = 0; g < N; g += 2 * HALF) {
#pragma unroll
        for (int j = 0; j < HALF; ++j) {
            if ((zm >> (g / (2 * HALF))) & 1) x[g + j + HALF] = x[g + j];
            else bfly<N, INV>(x[g + j], x[g + j + HALF], j * (N / (2 * HALF)));
        }
    }
    if constexpr (2 * HALF < N) fft_stages<N, INV, NIN, 2 * HALF>(x);
}

// in-register radix-2 FFT of N points (natural order in and out); inputs
// NIN .. N-1 are known to be zero, and the butterflies whose lower operand
// is still all zeros become copies (a + w 0 = a - w 0 = a)
template <int N, bool INV, int NIN = N, typename C>
__device__ __forceinline__ void fft_reg(C (&x)[N]) {
    constexpr int L = ilog2_c(N);
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const int j = brev_c(i, L);
        if (j > i) {
            C t = x[i];
            x[i] = x[j];
            x[j] = t;
        }
    }
    fft_stages<N, INV, NIN, 1>(x);
}

// CTA shape: FP32 planes of 16 columns, and 32 x 32 FP32 planes, use 192
// threads (a 12-plane group of 16 columns, or a 6-plane group of 32 columns,
// is then one fused column line per thread), everything else 256.  Those FP32
// grids and all others of at most 512 points run three CTAs per SM, the
// remaining FP32 grids with both sides <= 32 two (the host plan sizes shared
// memory for that); the register budget follows.
template <typename R, int N1, int N2> struct PlaneShape {
    static constexpr int threads = (sizeof(R) == 4 && (N2 == 16 || (N1 == 32 && N2 == 32))) ? 192 : 256;
    static constexpr int ctas = (sizeof(R) == 4 && (N1 * N2 <= 512 || (N1 == 32 && N2 == 32))) ? 3
                              : (N1 <= 32 && N2 <= 32 && sizeof(R) == 4) ? 2 : 1;
};

// KK: the B-spline order when it is known at compile time (6, every cell
// here), else 0 (read from the arguments, at most 8)
template <typename R, int N1, int N2, int KK>
__global__ void __launch_bounds__(PlaneShape<R, N1, N2>::threads, PlaneShape<R, N1, N2>::ctas)
    plane_reg_kernel(const __grid_constant__ PlaneArgs<R> a) {
    typedef typename V2<R>::T C;
    constexpr int LDP = N2 + 1;
    constexpr int PS = N1 * LDP;
    constexpr int NN = N1 * N2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *planes = reinterpret_cast<C *>(smem_raw);
    C *acc = planes + (size_t)a.np * PS;
    constexpr int KM = KK ? KK : 8;       // register extent of the kappa-wide windows
    const int K = KK ? KK : a.order, P = a.nquad, nb = a.nb;

    const int nbt = (a.nbands + a.bt - 1) / a.bt;
    const int item = blockIdx.x;
    const int c = item % a.nchunks;
    const int kb = item / a.nchunks;
    const int bt = kb % nbt;
    const int ks = kb / nbt;
    const KDesc &d = a.d[ks];
    const int ldg = d.ldg, ng = d.ng;
    const int b0 = bt * a.bt;
    const int nbb = min(a.bt, a.nbands - b0);
    const int *goff = a.goff + d.kofs;
    const int *rows = a.rows + d.rows_ofs;
    const int nrows = d.nrows;
    const int t0 = chunk_begin(c, a.nint, a.nchunks), t1 = chunk_begin(c + 1, a.nint, a.nchunks);
    const int nplanes = nbb * P;          // (band, Gauss point) planes per interval
    const size_t band_stride = (size_t)nb * ldg;
    const size_t part_stride = (size_t)(a.nchunks - 1) * 2 * (K - 1) * ldg;

    for (int i = threadIdx.x; i < nbb * K * ldg; i += blockDim.x) acc[i] = czero<C>();
    __syncthreads();

    auto write_row = [&](int j) {
        int lo = max(0, j - K + 2), hi = min(a.nint - 1, j + 1);
        for (int bb = 0; bb < nbb; ++bb) {
            C *slot = acc + ((size_t)bb * K + (j % K)) * ldg;
            C *dst;
            const int b = b0 + bb;
            C *part = reinterpret_cast<C *>(d.part) + (size_t)b * part_stride;
            if (lo >= t0 && hi <= t1 - 1)
                dst = reinterpret_cast<C *>(d.Y) + (size_t)b * band_stride + (size_t)j * ldg;
            else if (lo < t0)
                dst = part + ((size_t)((c - 1) * 2 + 1) * (K - 1) + (j - (t0 - 1))) * ldg;
            else
                dst = part + ((size_t)(c * 2 + 0) * (K - 1) + (j - (t1 - 1))) * ldg;
            for (int g = threadIdx.x; g < ldg; g += blockDim.x) {
                dst[g] = g < ng ? slot[g] : czero<C>();
                slot[g] = czero<C>();
            }
        }
    };

    // per-group plane metadata: band and Gauss point of each plane, and its B values
    int *pl_b = reinterpret_cast<int *>(acc + (size_t)a.bt * K * a.ldg_max);
    int *pl_s = pl_b + a.np;
    R *bqs = reinterpret_cast<R *>(pl_b + 2 * a.np);   // np x 8; pl_b is 8-byte aligned and 2 np ints are 8 np bytes
    const unsigned rmagic = d.rows_magic;

    for (int t = t0; t < t1; ++t) {
        const int slot0 = (t - 1 + K) % K;      // ring slot of row t-1
        for (int p0 = 0; p0 < nplanes; p0 += a.np) {
            const int npl = min(a.np, nplanes - p0);
            if (threadIdx.x < npl) {
                const int p = p0 + threadIdx.x, bb = p / P, s = p - bb * P;
                pl_b[threadIdx.x] = bb;
                pl_s[threadIdx.x] = s;
#pragma unroll
                for (int m = 0; m < 8; ++m) bqs[threadIdx.x * 8 + m] = m < K ? a.Bq[(size_t)(t * P + s) * K + m] : R(0);
            }
            // zero the planes of the group (16-byte stores)
            {
                float4 *z = reinterpret_cast<float4 *>(planes);
                const int n16 = (int)((size_t)npl * PS * sizeof(C) / 16);
                for (int e = threadIdx.x; e < n16; e += blockDim.x) z[e] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            __syncthreads();
            // (a) B-spline evaluation of every plane of the group
            for (int g = threadIdx.x; g < ng; g += blockDim.x) {
                const int o = goff[g];
                const int op = o + o / N2;           // padded offset
                int cur_b = -1;
                C x[KM];
                for (int pl = 0; pl < npl; ++pl) {
                    const int bb = pl_b[pl];
                    if (bb != cur_b) {
                        cur_b = bb;
                        const C *X = reinterpret_cast<const C *>(d.X) + (size_t)(b0 + bb) * band_stride;
#pragma unroll
                        for (int m = 0; m < KM; ++m) {
                            int j = t + m - 1;
                            x[m] = ((KK || m < K) && j >= 0 && j < nb) ? X[(size_t)j * ldg + g] : czero<C>();
                        }
                    }
                    C psi = czero<C>();
#pragma unroll
                    for (int m = 0; m < KM; ++m)
                        if (KK || m < K) rfma(psi, bqs[pl * 8 + m], x[m]);
                    planes[(size_t)pl * PS + op] = psi;
                }
            }
            __syncthreads();
            // (b1) inverse transform of the occupied rows
            for (int e = threadIdx.x; e < npl * nrows; e += blockDim.x) {
                const int pl = __umulhi((unsigned)e, rmagic);
                const int r = rows[e - pl * nrows];
                C *line = planes + (size_t)pl * PS + r * LDP;
                C v[N2];
#pragma unroll
                for (int i = 0; i < N2; ++i) v[i] = line[i];
                fft_reg<N2, true>(v);
#pragma unroll
                for (int i = 0; i < N2; ++i) line[i] = v[i];
            }
            __syncthreads();
            // (b2, c, d1) column: inverse transform, w_q V / (N1 N2), forward transform
            for (int e = threadIdx.x; e < npl * N2; e += blockDim.x) {
                const int pl = e / N2, col = e % N2;
                C *line = planes + (size_t)pl * PS + col;
                const R *V = a.Vn + (size_t)(t * P + pl_s[pl]) * NN + col;
                C v[N1];
#pragma unroll
                for (int i = 0; i < N1; ++i) v[i] = line[i * LDP];
                fft_reg<N1, true>(v);
#pragma unroll
                for (int i = 0; i < N1; ++i) v[i] = rscale(__ldg(V + i * N2), v[i]);
                fft_reg<N1, false>(v);
#pragma unroll
                for (int i = 0; i < N1; ++i) line[i * LDP] = v[i];
            }
            __syncthreads();
            // (d2) forward transform of the rows that hold disc points
            for (int e = threadIdx.x; e < npl * nrows; e += blockDim.x) {
                const int pl = __umulhi((unsigned)e, rmagic);
                const int r = rows[e - pl * nrows];
                C *line = planes + (size_t)pl * PS + r * LDP;
                C v[N2];
#pragma unroll
                for (int i = 0; i < N2; ++i) v[i] = line[i];
                fft_reg<N2, false>(v);
#pragma unroll
                for (int i = 0; i < N2; ++i) line[i] = v[i];
            }
            __syncthreads();
            // (e) adjoint B-spline sum into the ring
            for (int g = threadIdx.x; g < ng; g += blockDim.x) {
                const int o = goff[g];
                const int op = o + o / N2;
                C sum[KM];
#pragma unroll
                for (int m = 0; m < KM; ++m) sum[m] = czero<C>();
                int cur = pl_b[0];
                auto flush = [&](int bb) {
#pragma unroll
                    for (int m = 0; m < KM; ++m) {
                        const int j = t + m - 1;
                        if ((KK || m < K) && j >= 0 && j < nb) {
                            int sl = slot0 + m;
                            if (sl >= K) sl -= K;
                            acc[((size_t)bb * K + sl) * ldg + g] += sum[m];
                        }
                        sum[m] = czero<C>();
                    }
                };
                for (int pl = 0; pl < npl; ++pl) {
                    const int bb = pl_b[pl];
                    if (bb != cur) {
                        flush(cur);
                        cur = bb;
                    }
                    const C v = planes[(size_t)pl * PS + op];
#pragma unroll
                    for (int m = 0; m < KM; ++m)
                        if (KK || m < K) rfma(sum[m], bqs[pl * 8 + m], v);
                }
                flush(cur);
            }
            __syncthreads();
        }
        if (t - 1 >= 0) write_row(t - 1);
        __syncthreads();
    }
    for (int j = max(0, t1 - 1); j <= t1 + K - 3 && j < nb; ++j) {
        write_row(j);
        __syncthreads();
    }
}

// grids of 16, 32 or 64 points per side (FP64: up to 32) and B-splines of
// order 6; everything else takes the radix-2 kernel
template <typename R> bool plane_reg_supported(int n1, int n2, int order) {
    const int lim = sizeof(R) == 4 ? 64 : 32;
    auto ok = [&](int n) { return n == 16 || n == 32 || n == 64; };
    return ok(n1) && ok(n2) && n1 <= lim && n2 <= lim && order == 6;
}

template <typename R, int N1, int N2, int KK>
static cudaError_t launch_k(const PlaneArgs<R> &a, unsigned grid, size_t smem, cudaStream_t s) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaError_t e = smem_limit_once((const void *)plane_reg_kernel<R, N1, N2, KK>, dev, optin);
    if (e != cudaSuccess) return e;
    if (smem > (size_t)optin) return cudaErrorInvalidValue;
    plane_reg_kernel<R, N1, N2, KK><<<grid, PlaneShape<R, N1, N2>::threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename R, int N1, int N2>
static cudaError_t launch_one(const PlaneArgs<R> &a, unsigned grid, size_t smem, cudaStream_t s) {
    if (a.order != 6) return cudaErrorInvalidValue;
    return launch_k<R, N1, N2, 6>(a, grid, smem, s);
}

template <typename R>
cudaError_t plane_reg_launch(const PlaneArgs<R> &a, unsigned grid, size_t smem, cudaStream_t s) {
#define MB_PR_CASE(A, B) \
    if (a.n1 == A && a.n2 == B) return launch_one<R, A, B>(a, grid, smem, s);
    if (sizeof(R) == 4) {
        MB_PR_CASE(16, 16) MB_PR_CASE(16, 32) MB_PR_CASE(16, 64)
        MB_PR_CASE(32, 16) MB_PR_CASE(32, 32) MB_PR_CASE(32, 64)
        MB_PR_CASE(64, 16) MB_PR_CASE(64, 32) MB_PR_CASE(64, 64)
    }
    return cudaErrorInvalidValue;
#undef MB_PR_CASE
}

template <>
cudaError_t plane_reg_launch<double>(const PlaneArgs<double> &a, unsigned grid, size_t smem, cudaStream_t s) {
    if (a.n1 == 16 && a.n2 == 16) return launch_one<double, 16, 16>(a, grid, smem, s);
    if (a.n1 == 16 && a.n2 == 32) return launch_one<double, 16, 32>(a, grid, smem, s);
    if (a.n1 == 32 && a.n2 == 16) return launch_one<double, 32, 16>(a, grid, smem, s);
    if (a.n1 == 32 && a.n2 == 32) return launch_one<double, 32, 32>(a, grid, smem, s);
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// FP32 compact-plane kernel.  The same computation as plane_reg_kernel for
// B-splines of order 6 with 6 Gauss points per knot interval, reorganised
// around three facts of the method:
//  * The disc's grid rows form one run of n1 values, n1min .. n1min + nocc - 1.
//    Storing row n1 at compact row n1 - n1min is a cyclic shift of the
//    frequency index along the first grid axis.  The column pass (inverse
//    transform, product with the real potential, forward transform) is a
//    circular convolution with V^ along that axis, so it commutes with the
//    shift: the column transforms run on the compact rows (the rest are zero
//    on input and not needed on output), and no plane ever holds an empty row.
//    A whole interval of planes (6 Gauss points x bands) then fits in shared
//    memory even on 64 x 64 grids.
//  * Every thread owns fixed columns g (= G of the disc) for the whole run of
//    intervals: it keeps the kappa-row window of X for its columns in
//    registers (one new row per interval, loaded one interval ahead), and it
//    alone touches its columns of the output-row ring, so finished rows are
//    written as soon as the adjoint sum completes them, with no extra pass.
//  * The potential is stored per column (i1 fastest), so a column task reads
//    its N1 values with 128-bit loads issued before its inverse transform.
// Phases per interval: B-spline evaluation -> inverse row transforms of the
// occupied rows -> fused column pass -> forward row transforms -> adjoint sum
// (and zeroing of the occupied rows' disc-free positions), four barriers.
// XM: where the kappa-row window of X lives -- 0: read from global memory
// each interval; 1: registers; 2: per-thread slots in shared memory (row j in
// slot j mod kappa), the new row loaded one interval ahead.
template <int N1, int N2, int NOCC, int BT, int T, int GPT, int CTAS, int XM, bool VPRE>
__device__ __forceinline__ void plane32_item(const PlaneArgs<float> &a, const int item) {
    constexpr int K = 6, P = 6, KP = K * P;
    constexpr int LDP = N2 + 1, PS = NOCC * LDP, NPL = BT * P;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *planes = reinterpret_cast<float2 *>(smem_raw);
    const int lda = a.ldg_max;                 // row stride of the output-row ring
    float2 *acc = planes + NPL * PS;           // [BT][K][lda]
    float2 *xs = acc + (size_t)BT * K * lda;   // XM = 2: [K][BT][GPT][T] window slots
    float *bqs = reinterpret_cast<float *>(xs + (XM == 2 ? K * BT * GPT * T : 0));   // B values of the run
    constexpr bool XREG = XM == 1;

    const int nbt = (a.nbands + BT - 1) / BT;
    const int c = item % a.nchunks;
    const int kb = item / a.nchunks;
    const int btile = kb % nbt, ks = kb / nbt;
    const KDesc &d = a.d[ks];
    const int ldg = d.ldg, ng = d.ng, nb = a.nb, nint = a.nint, nocc = d.nocc;
    const int b0 = btile * BT, nbb = min(BT, a.nbands - b0), npl = nbb * P;
    const int ps = nocc * LDP;                 // plane stride: row nocc of a plane is row 0 of the next
    const int t0 = chunk_begin(c, nint, a.nchunks), t1 = chunk_begin(c + 1, nint, a.nchunks);
    const size_t band_stride = (size_t)nb * ldg;
    const size_t part_stride = (size_t)(a.nchunks - 1) * 2 * (K - 1) * ldg;
    const float2 *X = reinterpret_cast<const float2 *>(d.X) + (size_t)b0 * band_stride;
    float2 *Y = reinterpret_cast<float2 *>(d.Y) + (size_t)b0 * band_stride;
    float2 *part = reinterpret_cast<float2 *>(d.part) + (size_t)b0 * part_stride;
    const int tid = threadIdx.x;

    int cp[GPT];                               // compact-plane offset of each owned column (-1: padding)
#pragma unroll
    for (int i = 0; i < GPT; ++i) {
        const int g = tid + i * T;
        cp[i] = g < ng ? __ldg(a.cpos + d.kofs + g) : -1;
    }
    {
        for (int e = tid; e < NPL * PS; e += T) planes[e] = make_float2(0.f, 0.f);
        for (int e = tid; e < (t1 - t0) * KP; e += T) bqs[e] = __ldg(a.Bq + (size_t)t0 * KP + e);
    }
#pragma unroll
    for (int i = 0; i < GPT; ++i) {
        const int g = tid + i * T;
        if (g < ldg)
#pragma unroll
            for (int r = 0; r < BT * K; ++r) acc[(size_t)r * lda + g] = make_float2(0.f, 0.f);
    }
    auto xval = [&](int b, int j, int i) -> float2 {
        const int g = tid + i * T;
        return (b < nbb && j >= 0 && j < nb && g < ng) ? __ldg(X + (size_t)b * band_stride + (size_t)j * ldg + g)
                                                       : make_float2(0.f, 0.f);
    };
    // destination of output row j (band 0; band b at + b * stride): Y for rows
    // that only this run touches, else the boundary scratch, whose two sides
    // the epilogue adds in a fixed order
    auto row_dst = [&](int j, size_t &stride) -> float2 * {
        const int lo = max(0, j - K + 2), hi = min(nint - 1, j + 1);
        if (lo >= t0 && hi <= t1 - 1) {
            stride = band_stride;
            return Y + (size_t)j * ldg;
        }
        stride = part_stride;
        if (lo < t0) return part + ((size_t)((c - 1) * 2 + 1) * (K - 1) + (j - (t0 - 1))) * ldg;
        return part + ((size_t)(c * 2 + 0) * (K - 1) + (j - (t1 - 1))) * ldg;
    };

    float2 xw[XREG ? BT : 1][XREG ? GPT : 1][K];   // xw[b][i][m] = X[t + m - 1] at column i
    auto xslot = [&](int j, int b, int i) -> float2 & { return xs[((((j + K) % K) * BT + b) * GPT + i) * T + tid]; };
    if constexpr (XM != 0) {
#pragma unroll
        for (int b = 0; b < BT; ++b)
#pragma unroll
            for (int i = 0; i < GPT; ++i)
#pragma unroll
                for (int m = 0; m < K; ++m) {
                    if constexpr (XREG) xw[b][i][m] = xval(b, t0 + m - 1, i);
                    else xslot(t0 + m - 1, b, i) = xval(b, t0 + m - 1, i);
                }
    }
    __syncthreads();

    for (int t = t0; t < t1; ++t) {
        const float2 *bq2 = reinterpret_cast<const float2 *>(bqs + (t - t0) * KP);   // this interval's B values
        float2 xn[XM ? BT : 1][XM ? GPT : 1];
        // (a) psi_q(G) = sum_m B_{t+m}(z_q) X[t+m-1][G] for the interval's planes
        {
            float2 x[BT][GPT][K];
#pragma unroll
            for (int b = 0; b < BT; ++b)
#pragma unroll
                for (int i = 0; i < GPT; ++i)
#pragma unroll
                    for (int m = 0; m < K; ++m) {
                        if constexpr (XREG) x[b][i][m] = xw[b][i][m];
                        else if constexpr (XM == 2) x[b][i][m] = xslot(t + m - 1, b, i);
                        else x[b][i][m] = xval(b, t + m - 1, i);
                    }
            if constexpr (XM != 0) {
                // the next interval's new row, in flight during this interval's transforms
#pragma unroll
                for (int b = 0; b < BT; ++b)
#pragma unroll
                    for (int i = 0; i < GPT; ++i) xn[b][i] = xval(b, t + K - 1, i);
            }
#pragma unroll
            for (int s = 0; s < P; ++s) {
                float bq[K];                       // B_{t+m}(z_q) of Gauss point s
#pragma unroll
                for (int m = 0; m < K; m += 2) {
                    const float2 v = bq2[(s * K + m) / 2];
                    bq[m] = v.x;
                    bq[m + 1] = v.y;
                }
#pragma unroll
                for (int i = 0; i < GPT; ++i) {
                    if (cp[i] < 0) continue;
#pragma unroll
                    for (int b = 0; b < BT; ++b) {
                        if (b >= nbb) break;
                        float2 psi = make_float2(0.f, 0.f);
#pragma unroll
                        for (int m = 0; m < K; ++m) rfma(psi, bq[m], x[b][i][m]);
                        planes[(b * P + s) * ps + cp[i]] = psi;
                    }
                }
            }
        }
        __syncthreads();
        // (b1) inverse transforms of the occupied rows
        for (int e = tid; e < npl * nocc; e += T) {
            float2 *line = planes + e * LDP;      // plane e / nocc, row e % nocc
            float2 v[N2];
#pragma unroll
            for (int i = 0; i < N2; ++i) v[i] = line[i];
            fft_reg<N2, true>(v);
#pragma unroll
            for (int i = 0; i < N2; ++i) line[i] = v[i];
        }
        __syncthreads();
        // (b2, c, d1) columns on the compact rows: inverse transform, w_q V / (N1 N2), forward transform
        for (int e = tid; e < npl * N2; e += T) {
            const int pl = e / N2, col = e % N2;
            const int s = pl % P;
            float2 *line = planes + pl * ps + col;
            const float4 *Vc = reinterpret_cast<const float4 *>(a.Vt + ((size_t)(t * P + s) * N2 + col) * N1);
            float vv[N1];
            if constexpr (VPRE) {
#pragma unroll
                for (int q = 0; q < N1 / 4; ++q) {
                    const float4 w = __ldg(Vc + q);
                    vv[4 * q] = w.x;
                    vv[4 * q + 1] = w.y;
                    vv[4 * q + 2] = w.z;
                    vv[4 * q + 3] = w.w;
                }
            }
            float2 v[N1];
#pragma unroll
            for (int i = 0; i < N1; ++i) v[i] = (i < NOCC && i < nocc) ? line[i * LDP] : make_float2(0.f, 0.f);
            fft_reg<N1, true, (NOCC < N1 ? NOCC : N1)>(v);
            if constexpr (VPRE) {
#pragma unroll
                for (int i = 0; i < N1; ++i) v[i] = rscale(vv[i], v[i]);
            } else {
#pragma unroll
                for (int q = 0; q < N1 / 4; ++q) {
                    const float4 w = __ldg(Vc + q);
                    v[4 * q] = rscale(w.x, v[4 * q]);
                    v[4 * q + 1] = rscale(w.y, v[4 * q + 1]);
                    v[4 * q + 2] = rscale(w.z, v[4 * q + 2]);
                    v[4 * q + 3] = rscale(w.w, v[4 * q + 3]);
                }
            }
            fft_reg<N1, false>(v);
#pragma unroll
            for (int i = 0; i < NOCC; ++i)
                if (i < nocc) line[i * LDP] = v[i];
        }
        __syncthreads();
        // (d2) forward transforms of the occupied rows
        for (int e = tid; e < npl * nocc; e += T) {
            float2 *line = planes + e * LDP;      // plane e / nocc, row e % nocc
            float2 v[N2];
#pragma unroll
            for (int i = 0; i < N2; ++i) v[i] = line[i];
            fft_reg<N2, false>(v);
#pragma unroll
            for (int i = 0; i < N2; ++i) line[i] = v[i];
        }
        __syncthreads();
        // (e) adjoint sum of the owned columns into the ring; row t-1 is then
        // complete and leaves the ring
        {
            const int slot0 = (t - 1 + K) % K;      // ring slot of row t-1
            size_t dstride = 0;
            float2 *dst = t >= 1 ? row_dst(t - 1, dstride) : nullptr;
#pragma unroll
            for (int i = 0; i < GPT; ++i) {
                const int g = tid + i * T;
                if (g >= ldg) continue;
#pragma unroll
                for (int b = 0; b < BT; ++b) {
                    if (b >= nbb) break;
                    float2 cm[K];
#pragma unroll
                    for (int m = 0; m < K; ++m) cm[m] = make_float2(0.f, 0.f);
                    if (cp[i] >= 0) {
#pragma unroll
                        for (int s = 0; s < P; ++s) {
                            const float2 phi = planes[(b * P + s) * ps + cp[i]];
#pragma unroll
                            for (int m = 0; m < K; m += 2) {
                                const float2 v = bq2[(s * K + m) / 2];
                                rfma(cm[m], v.x, phi);
                                rfma(cm[m + 1], v.y, phi);
                            }
                        }
                    }
                    float2 *ab = acc + (size_t)b * K * lda + g;
                    {
                        float2 *sl = ab + (size_t)slot0 * lda;
                        if (dst) dst[(size_t)b * dstride + g] = *sl + cm[0];
                        *sl = make_float2(0.f, 0.f);
                    }
#pragma unroll
                    for (int m = 1; m < K; ++m) {
                        if (t + m - 1 < nb) {
                            int sl = slot0 + m;
                            if (sl >= K) sl -= K;
                            ab[(size_t)sl * lda] += cm[m];
                        }
                    }
                }
            }
            // the occupied rows' disc-free positions start the next interval at zero
            for (int e = tid; e < d.nz; e += T) {
                const int pos = __ldg(a.zpos + d.zofs + e);
                for (int pl = 0; pl < npl; ++pl) planes[pl * ps + pos] = make_float2(0.f, 0.f);
            }
            if constexpr (XREG) {
#pragma unroll
                for (int b = 0; b < BT; ++b)
#pragma unroll
                    for (int i = 0; i < GPT; ++i) {
#pragma unroll
                        for (int m = 0; m + 1 < K; ++m) xw[b][i][m] = xw[b][i][m + 1];
                        xw[b][i][K - 1] = xn[b][i];
                    }
            } else if constexpr (XM == 2) {
                // row t+K-1 takes the slot of row t-1, which no later interval reads
#pragma unroll
                for (int b = 0; b < BT; ++b)
#pragma unroll
                    for (int i = 0; i < GPT; ++i) xslot(t + K - 1, b, i) = xn[b][i];
            }
        }
    }
    // rows t1-1 .. t1+K-3 are complete once the run ends
    for (int m = 0; m + 1 < K; ++m) {
        const int j = t1 - 1 + m;
        if (j < 0 || j >= nb) continue;
        size_t dstride = 0;
        float2 *dst = row_dst(j, dstride);
        const int sl = j % K;
#pragma unroll
        for (int i = 0; i < GPT; ++i) {
            const int g = tid + i * T;
            if (g >= ldg) continue;
#pragma unroll
            for (int b = 0; b < BT; ++b)
                if (b < nbb) dst[(size_t)b * dstride + g] = acc[((size_t)b * K + sl) * lda + g];
        }
    }
}

// One launch covers every (k-point, band tile, run of intervals) item of the
// batch.  Static mode: CTA i takes item i.  Persistent mode (a.queue set):
// the grid is one CTA per resident slot, and each CTA takes the next item
// from a device counter until none is left, so items of uneven cost (the
// k-points' discs differ in size) balance over the SMs; the last CTA to
// finish resets the counter pair, which leaves it ready for the next launch
// (and for replays of a captured graph) without a separate memset.
template <int N1, int N2, int NOCC, int BT, int T, int GPT, int CTAS, int XM, bool VPRE>
__global__ void __launch_bounds__(T, CTAS) plane32_kernel(const __grid_constant__ PlaneArgs<float> a) {
    __shared__ int s_item;
    const int nitems = a.nsel * ((a.nbands + BT - 1) / BT) * a.nchunks;
    for (int pass = 0;; ++pass) {
        if (threadIdx.x == 0) s_item = a.queue ? atomicAdd(a.queue, 1) : (pass == 0 ? (int)blockIdx.x : nitems);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= nitems) break;
        plane32_item<N1, N2, NOCC, BT, T, GPT, CTAS, XM, VPRE>(a, item);
        __syncthreads();
    }
    if (a.queue && threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(a.queue + 1, 1) == (int)gridDim.x - 1) {
            atomicExch(a.queue, 0);
            atomicExch(a.queue + 1, 0);
        }
    }
}

// Instances: id, grid, bound on the occupied rows, bands per CTA, threads,
// columns per thread, CTAs per SM, X window (XM), potential loaded ahead of
// the inverse column transform.  The first feasible instance of a grid is the
// default; mb_autotune times all of them.
#define MB_P32_LIST(X)                                   \
    X(0, 16, 16, 10, 2, 96, 1, 4, 1, true)               \
    X(1, 32, 16, 24, 2, 192, 1, 2, 1, true)              \
    X(2, 32, 16, 24, 2, 256, 1, 2, 2, false)             \
    X(3, 32, 16, 24, 2, 192, 1, 2, 2, true)              \
    X(4, 32, 16, 24, 1, 96, 2, 4, 1, true)               \
    X(5, 32, 32, 24, 1, 192, 2, 2, 1, true)              \
    X(6, 32, 32, 24, 2, 384, 1, 1, 1, true)              \
    X(7, 32, 32, 23, 1, 192, 2, 3, 2, false)             \
    X(8, 64, 64, 48, 1, 384, 4, 1, 0, false)             \
    X(9, 64, 64, 48, 1, 256, 6, 1, 0, false)             \
    X(10, 32, 16, 22, 2, 192, 1, 3, 2, false)

int plane32_shapes(int n1, int n2, int order, int nquad, int nocc, int ldg, Plane32Shape *out, int max) {
    int n = 0;
    if (order != 6 || nquad != 6) return 0;
#define MB_P32_SHAPE(ID, A, B, NO, BT, T, GPT, CT, XR, VP)                                          \
    if (n1 == A && n2 == B && nocc <= NO && ldg <= T * GPT && n < max) {                            \
        Plane32Shape &sh = out[n++];                                                                 \
        sh.ok = true;                                                                                \
        sh.id = ID;                                                                                  \
        sh.nocc_max = NO;                                                                            \
        sh.ldg_max = T * GPT;                                                                        \
        sh.bt = BT;                                                                                  \
        sh.threads = T;                                                                              \
        sh.ctas_per_sm = CT;                                                                         \
        sh.smem_fixed = ((size_t)BT * 6 * NO * (B + 1) + (XR == 2 ? 6 * BT * GPT * T : 0)) * sizeof(float2); \
        std::snprintf(sh.name, sizeof(sh.name), "plane32_kernel<%d, %d, %d, %d, %d, %d, %d, %d, %d>", A, B, NO, \
                      BT, T, GPT, CT, XR, VP ? 1 : 0);                                              \
    }
    MB_P32_LIST(MB_P32_SHAPE)
#undef MB_P32_SHAPE
    return n;
}

cudaError_t plane32_launch(const PlaneArgs<float> &a, const Plane32Shape &sh, unsigned grid, size_t smem,
                           cudaStream_t s) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (smem > (size_t)optin) return cudaErrorInvalidValue;
#define MB_P32_LAUNCH(ID, A, B, NO, BT, T, GPT, CT, XR, VP)                                          \
    if (sh.id == ID) {                                                                               \
        if (a.n1 != A || a.n2 != B) return cudaErrorInvalidValue;                                    \
        const void *fn = (const void *)plane32_kernel<A, B, NO, BT, T, GPT, CT, XR, VP>;              \
        cudaError_t e = smem_limit_once(fn, dev, optin);                                             \
        if (e != cudaSuccess) return e;                                                              \
        plane32_kernel<A, B, NO, BT, T, GPT, CT, XR, VP><<<grid, T, smem, s>>>(a);                   \
        return cudaGetLastError();                                                                   \
    }
    MB_P32_LIST(MB_P32_LAUNCH)
#undef MB_P32_LAUNCH
    return cudaErrorInvalidValue;
}

template bool plane_reg_supported<float>(int, int, int);
template bool plane_reg_supported<double>(int, int, int);
template cudaError_t plane_reg_launch<float>(const PlaneArgs<float> &, unsigned, size_t, cudaStream_t);

}  // namespace mb
