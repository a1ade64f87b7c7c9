// Local-potential plane kernel with register-resident FFT lines.
//
// Same computation as the radix-2 plane kernel in apply.cu (B-spline
// evaluation on the Gauss planes, inverse 2D FFT, product with
// w_q V(r, z_q) / (N1 N2), forward 2D FFT, adjoint B-spline sum), organised
// for throughput:
//  * every 1D transform of N <= 64 points runs inside one thread's registers
//    (radix-2, bit reversal by register renaming, trivial twiddles folded at
//    compile time), so a plane crosses shared memory three times per
//    direction instead of once per butterfly stage;
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
#include "apply_common.cuh"
#include "mb_internal.h"

namespace mb {

__constant__ float2 c_twf[64];    // exp(+2 pi i k / 64)
__constant__ double2 c_twd[64];

void upload_fft_twiddles() {
    float2 tf[64];
    double2 td[64];
    for (int k = 0; k < 64; ++k) {
        double a = 2.0 * 3.14159265358979323846 * k / 64.0;
        td[k] = make_double2(std::cos(a), std::sin(a));
        tf[k] = make_float2((float)td[k].x, (float)td[k].y);
    }
    cudaMemcpyToSymbol(c_twf, tf, sizeof(tf));
    cudaMemcpyToSymbol(c_twd, td, sizeof(td));
}

template <typename C> __device__ __forceinline__ C ctw(int k);
template <> __device__ __forceinline__ float2 ctw<float2>(int k) { return c_twf[k]; }
template <> __device__ __forceinline__ double2 ctw<double2>(int k) { return c_twd[k]; }

constexpr int brev_c(int x, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((x >> b) & 1) << (bits - 1 - b);
    return r;
}
constexpr int ilog2_c(int n) { return n <= 1 ? 0 : 1 + ilog2_c(n / 2); }

// b * exp(sign 2 pi i tk / N), sign = + for the inverse transform
template <int N, bool INV, typename C>
__device__ __forceinline__ C twmul(C b, int tk) {
    if (tk == 0) return b;
    if (4 * tk == N) return INV ? mk(-b.y, b.x) : mk(b.y, -b.x);
    C w = ctw<C>(tk * (64 / N));
    if (!INV) w.y = -w.y;
    return cmul(b, w);
}

// in-register radix-2 FFT of N points (natural order in and out)
template <int N, bool INV, typename C>
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
#pragma unroll
    for (int half = 1; half < N; half *= 2) {
#pragma unroll
        for (int g = 0; g < N; g += 2 * half) {
#pragma unroll
            for (int j = 0; j < half; ++j) {
                C b = twmul<N, INV>(x[g + j + half], j * (N / (2 * half)));
                C a = x[g + j];
                x[g + j] = a + b;
                x[g + j + half] = a - b;
            }
        }
    }
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

template bool plane_reg_supported<float>(int, int, int);
template bool plane_reg_supported<double>(int, int, int);
template cudaError_t plane_reg_launch<float>(const PlaneArgs<float> &, unsigned, size_t, cudaStream_t);

}  // namespace mb
