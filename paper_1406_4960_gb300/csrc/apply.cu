// H and S applies of the mixed basis on one GPU (sm_103a).
//
//  plane_kernel   local potential (§II.B.1, Eqs. (12)-(13), (19)-(20)):
//                 B-spline evaluation on the Gauss planes, inverse 2D FFT,
//                 product with w_q V(r, z_q), forward 2D FFT, adjoint
//                 B-spline sum back to coefficients.  One CTA owns a
//                 (k, band, run of knot intervals) and keeps the kappa
//                 output rows that the current interval touches in a ring in
//                 shared memory; rows shared with a neighbouring run go to
//                 scratch and are summed in a fixed order by the epilogue.
//  epilogue       kinetic term Eq. (9) (banded in j, diagonal in G) plus the
//                 boundary-row sums.
//  zgemm          projector contractions of Eq. (17), factorized as
//                 u_p(G, j) = z_p(j) q_p(G): W = X q^H, then
//                 Y += (z E F) q with F_p = sum_j z_p(j) W_p(j).
//  banded_*       S (Eqs. (7)-(8)), S^-1 and the eigensolver's
//                 preconditioner through banded Cholesky factors.
#include <algorithm>
#include <cstring>

#include "apply_common.cuh"
#include "cplx.cuh"
#include "mb_internal.h"

namespace mb {

// ---------------------------------------------------------------------------
// radix-2 FFTs on ns planes of N1 x N2 in shared memory (row-major, i2 fastest)
// Inverse: decimation in frequency, natural in -> bit-reversed out, sign +.
// Forward: decimation in time, bit-reversed in -> natural out, sign -.
template <typename R2, bool INV>
__device__ void fft_axis(R2 *buf, int ns, int N1, int N2, int axis, const R2 *tw, int nmax) {
    const int NN = N1 * N2;
    const int N = axis == 2 ? N2 : N1;
    const int estride = axis == 2 ? 1 : N2;
    const int ntr_plane = axis == 2 ? N1 : N2;
    const int ntr = ns * ntr_plane;
    const int nbf = ntr * (N / 2);
    for (int stage = 0, half = INV ? N / 2 : 1; INV ? half >= 1 : half < N;
         ++stage, half = INV ? half / 2 : half * 2) {
        const int twstep = nmax / (2 * half);
        for (int bi = threadIdx.x; bi < nbf; bi += blockDim.x) {
            int tr = bi / (N / 2);
            int r = bi - tr * (N / 2);
            int plane = tr / ntr_plane;
            int line = tr - plane * ntr_plane;
            int base = plane * NN + (axis == 2 ? line * N2 : line);
            int grp = r / half;
            int j = r - grp * half;
            int i0 = grp * 2 * half + j;
            int i1 = i0 + half;
            R2 w = tw[j * twstep];
            R2 *p0 = buf + base + i0 * estride;
            R2 *p1 = buf + base + i1 * estride;
            R2 a = *p0, b = *p1;
            if (INV) {
                *p0 = a + b;
                *p1 = cmul(a - b, w);
            } else {
                R2 t = cmul_c(b, w);
                *p0 = a + t;
                *p1 = a - t;
            }
        }
        __syncthreads();
    }
}

template <typename R>
__global__ void __launch_bounds__(256) plane_kernel(const __grid_constant__ PlaneArgs<R> a) {
    typedef typename V2<R>::T R2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int NN = a.n1 * a.n2;
    const int K = a.order, P = a.nquad;
    R2 *tw = reinterpret_cast<R2 *>(smem_raw);
    R2 *buf = tw + a.nmax / 2;
    R2 *acc = buf + (size_t)a.np * NN;
    for (int i = threadIdx.x; i < a.nmax / 2; i += blockDim.x) tw[i] = a.tw[i];

    const int item = blockIdx.x;
    const int c = item % a.nchunks;
    const int kb = item / a.nchunks;
    const int b = kb % a.nbands;
    const int ks = kb / a.nbands;
    const KDesc &d = a.d[ks];
    const int ldg = d.ldg, ng = d.ng, nb = a.nb;
    const R2 *X = reinterpret_cast<const R2 *>(d.X) + (size_t)b * nb * ldg;
    R2 *Y = reinterpret_cast<R2 *>(d.Y) + (size_t)b * nb * ldg;
    R2 *part = reinterpret_cast<R2 *>(d.part) + (size_t)b * (a.nchunks - 1) * 2 * (K - 1) * ldg;
    const int *goff = a.goff + d.kofs;
    const int t0 = c * a.chunk, t1 = min(a.nint, t0 + a.chunk);

    for (int i = threadIdx.x; i < K * ldg; i += blockDim.x) acc[i] = czero<R2>();
    __syncthreads();

    auto write_row = [&](int j) {
        R2 *slot = acc + (size_t)(j % K) * ldg;
        int lo = max(0, j - K + 2), hi = min(a.nint - 1, j + 1);
        R2 *dst;
        if (lo >= t0 && hi <= t1 - 1)
            dst = Y + (size_t)j * ldg;
        else if (lo < t0)   // shared with the previous run: right-hand side of boundary c-1
            dst = part + ((size_t)((c - 1) * 2 + 1) * (K - 1) + (j - (t0 - 1))) * ldg;
        else                // shared with the next run: left-hand side of boundary c
            dst = part + ((size_t)(c * 2 + 0) * (K - 1) + (j - (t1 - 1))) * ldg;
        for (int g = threadIdx.x; g < ldg; g += blockDim.x) {
            dst[g] = g < ng ? slot[g] : czero<R2>();
            slot[g] = czero<R2>();
        }
    };

    for (int t = t0; t < t1; ++t) {
        for (int s0 = 0; s0 < P; s0 += a.np) {
            const int ns = min(a.np, P - s0);
            const int q0 = t * P + s0;
            for (int e = threadIdx.x; e < ns * NN; e += blockDim.x) buf[e] = czero<R2>();
            __syncthreads();
            // (a) B-spline evaluation: psi_q(G) = sum_m B_{t+m}(z_q) X[t+m-1][G]
            for (int g = threadIdx.x; g < ng; g += blockDim.x) {
                R2 x[8];
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    int j = t + m - 1;
                    x[m] = (m < K && j >= 0 && j < nb) ? X[(size_t)j * ldg + g] : czero<R2>();
                }
                const int o = goff[g];
                for (int s = 0; s < ns; ++s) {
                    const R *bq = a.Bq + (size_t)(q0 + s) * K;
                    R2 psi = czero<R2>();
#pragma unroll
                    for (int m = 0; m < 8; ++m)
                        if (m < K) rfma(psi, bq[m], x[m]);
                    buf[s * NN + o] = psi;
                }
            }
            __syncthreads();
            // (b) inverse 2D FFT to the real-space plane
            fft_axis<R2, true>(buf, ns, a.n1, a.n2, 2, tw, a.nmax);
            fft_axis<R2, true>(buf, ns, a.n1, a.n2, 1, tw, a.nmax);
            // (c) w_q V(r, z_q) / (N1 N2)
            const R *V = a.V + (size_t)q0 * NN;
            for (int e = threadIdx.x; e < ns * NN; e += blockDim.x) buf[e] = rscale(V[e], buf[e]);
            __syncthreads();
            fft_axis<R2, false>(buf, ns, a.n1, a.n2, 1, tw, a.nmax);
            fft_axis<R2, false>(buf, ns, a.n1, a.n2, 2, tw, a.nmax);
            // (d) adjoint: acc[t+m-1][G] += sum_q B_{t+m}(z_q) phi_q(G)
            for (int g = threadIdx.x; g < ng; g += blockDim.x) {
                const int o = goff[g];
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    int j = t + m - 1;
                    if (m >= K || j < 0 || j >= nb) continue;
                    R2 sum = czero<R2>();
                    for (int s = 0; s < ns; ++s) rfma(sum, a.Bq[(size_t)(q0 + s) * K + m], buf[s * NN + o]);
                    acc[(size_t)(j % K) * ldg + g] += sum;
                }
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

// ---------------------------------------------------------------------------
// epilogue: Y[j] = local(j) + (D/2 + |k+G|^2/2 S) X   (Eq. (9))
template <typename R> struct EpiArgs {
    const R *Sband, *Dband, *q2;
    int order, nb, nbands, nchunks, chunk, nint;
    KDesc d[kMaxK];
};

template <typename R>
__global__ void __launch_bounds__(256) epilogue_kernel(const __grid_constant__ EpiArgs<R> a) {
    typedef typename V2<R>::T R2;
    const int j = blockIdx.x, b = blockIdx.y, ks = blockIdx.z;
    const KDesc &d = a.d[ks];
    const int K = a.order, W = 2 * K - 1, ldg = d.ldg, nb = a.nb;
    const R2 *X = reinterpret_cast<const R2 *>(d.X) + (size_t)b * nb * ldg;
    R2 *Y = reinterpret_cast<R2 *>(d.Y) + (size_t)b * nb * ldg;
    const R2 *part = reinterpret_cast<const R2 *>(d.part) + (size_t)b * (a.nchunks - 1) * 2 * (K - 1) * ldg;
    // boundary c between runs c and c+1 covers rows [t1 - 1, t1 + K - 3], t1 = (c+1)*chunk
    int bc = -1, br = 0;
    for (int c = 0; c + 1 < a.nchunks; ++c) {
        int t1 = (c + 1) * a.chunk;
        if (j >= t1 - 1 && j <= t1 + K - 3) { bc = c; br = j - (t1 - 1); }
    }
    const R *q2 = a.q2 + d.kofs;
    const R *Sr = a.Sband + (size_t)j * W;
    const R *Dr = a.Dband + (size_t)j * W;
    for (int g = threadIdx.x; g < ldg; g += blockDim.x) {
        if (g >= d.ng) { Y[(size_t)j * ldg + g] = czero<R2>(); continue; }
        R2 v;
        if (bc >= 0) {
            const R2 *p0 = part + ((size_t)(bc * 2 + 0) * (K - 1) + br) * ldg;
            const R2 *p1 = part + ((size_t)(bc * 2 + 1) * (K - 1) + br) * ldg;
            v = p0[g] + p1[g];
        } else {
            v = Y[(size_t)j * ldg + g];
        }
        const R hq = R(0.5) * q2[g];
        R2 tx = czero<R2>();
        for (int dd = 0; dd < W; ++dd) {
            int jj = j + dd - (K - 1);
            if (jj < 0 || jj >= nb) continue;
            R coef = R(0.5) * Dr[dd] + hq * Sr[dd];
            rfma(tx, coef, X[(size_t)jj * ldg + g]);
        }
        Y[(size_t)j * ldg + g] = v + tx;
    }
}

// ---------------------------------------------------------------------------
// complex GEMM, batched over k-points:
//   mode 0 (projection):      W[m][n] = sum_k A[m][k] conj(Q[n][k])   A = X rows, Q = q_p(G)
//   mode 1 (back-projection): Y[m][n] += sum_k C[m][k] Q[k][n]        C = coefficients
// m = (band, j) rows; 64x64 output tile, 256 threads, 4x4 outputs each.
template <typename R> struct GemmArgs {
    const typename V2<R>::T *Q;   // q_p(G) table (all k)
    int mode, nb, nbands, nproj;
    KDesc d[kMaxK];
};

template <typename R>
__global__ void __launch_bounds__(256) zgemm_kernel(const __grid_constant__ GemmArgs<R> a) {
    typedef typename V2<R>::T R2;
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ R2 As[BK][BM + 1];
    __shared__ R2 Bs[BK][BN + 1];
    const int ks = blockIdx.z;
    const KDesc &d = a.d[ks];
    const int ldg = d.ldg;
    const int M = a.nbands * a.nb;
    const int N = a.mode == 0 ? a.nproj : d.ng;
    const int KK = a.mode == 0 ? d.ng : a.nproj;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    if (n0 >= N) return;
    const R2 *Q = a.Q + d.qofs;
    const R2 *A = a.mode == 0 ? reinterpret_cast<const R2 *>(d.X) : reinterpret_cast<const R2 *>(d.C);
    const int lda = a.mode == 0 ? ldg : a.nproj;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    R2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jn = 0; jn < 4; ++jn) acc[i][jn] = czero<R2>();
    for (int k0 = 0; k0 < KK; k0 += BK) {
        for (int e = threadIdx.x; e < BM * BK; e += 256) {
            int mm = e / BK, kk = e % BK;
            int gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < M && gk < KK) ? A[(size_t)gm * lda + gk] : czero<R2>();
        }
        for (int e = threadIdx.x; e < BN * BK; e += 256) {
            int nn, kk;
            R2 v = czero<R2>();
            if (a.mode == 0) {   // B[k][n] = conj(Q[n][k])
                nn = e / BK; kk = e % BK;
                int gn = n0 + nn, gk = k0 + kk;
                if (gn < N && gk < KK) { R2 q = Q[(size_t)gn * ldg + gk]; v = mk(q.x, -q.y); }
            } else {             // B[k][n] = Q[k][n]
                kk = e / BN; nn = e % BN;
                int gn = n0 + nn, gk = k0 + kk;
                if (gn < N && gk < KK) v = Q[(size_t)gk * ldg + gn];
            }
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            R2 av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int i = 0; i < 4; ++i) bv[i] = Bs[kk][tx * 4 + i];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int jn = 0; jn < 4; ++jn) cfma(acc[i][jn], av[i], bv[jn]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int gm = m0 + ty * 4 + i;
        if (gm >= M) continue;
#pragma unroll
        for (int jn = 0; jn < 4; ++jn) {
            int gn = n0 + tx * 4 + jn;
            if (gn >= N) continue;
            if (a.mode == 0) {
                reinterpret_cast<R2 *>(d.W)[(size_t)gm * a.nproj + gn] = acc[i][jn];
            } else {
                R2 *y = reinterpret_cast<R2 *>(d.Y) + (size_t)gm * ldg + gn;
                *y = *y + acc[i][jn];
            }
        }
    }
}

// F_p(b) = sum_j z_p(j) W[(b,j)][p];  C[(b,j)][p] = z_p(j) E_p F_p(b)
template <typename R> struct CoefArgs {
    const R *zproj, *E;
    int nb, nbands, nproj;
    KDesc d[kMaxK];
};

template <typename R>
__global__ void coef_kernel(const __grid_constant__ CoefArgs<R> a) {
    typedef typename V2<R>::T R2;
    const int ks = blockIdx.y;
    const KDesc &d = a.d[ks];
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= a.nbands * a.nproj) return;
    const int b = idx / a.nproj, p = idx % a.nproj;
    const R2 *W = reinterpret_cast<const R2 *>(d.W) + (size_t)b * a.nb * a.nproj;
    R2 *C = reinterpret_cast<R2 *>(d.C) + (size_t)b * a.nb * a.nproj;
    const R *z = a.zproj + (size_t)p * a.nb;
    R2 F = czero<R2>();
    for (int j = 0; j < a.nb; ++j) rfma(F, z[j], W[(size_t)j * a.nproj + p]);
    F = rscale(a.E[p], F);
    for (int j = 0; j < a.nb; ++j) C[(size_t)j * a.nproj + p] = rscale(z[j], F);
}

// ---------------------------------------------------------------------------
// banded operators along j, one thread per (band, G) column
template <typename R>
__global__ void banded_S_kernel(const R *Sband, int order, int nb, int ng, int ldg, int nbands,
                                const typename V2<R>::T *X, typename V2<R>::T *Y) {
    typedef typename V2<R>::T R2;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (g >= ldg) return;
    const int K = order, W = 2 * K - 1;
    const R2 *x = X + (size_t)b * nb * ldg;
    R2 *y = Y + (size_t)b * nb * ldg;
    for (int j = 0; j < nb; ++j) {
        R2 s = czero<R2>();
        if (g < ng)
            for (int dd = 0; dd < W; ++dd) {
                int jj = j + dd - (K - 1);
                if (jj >= 0 && jj < nb) rfma(s, Sband[(size_t)j * W + dd], x[(size_t)jj * ldg + g]);
            }
        y[(size_t)j * ldg + g] = s;
    }
}

// L L^T y = x with L[j][j-d] = Lb[(j*K + d)] (per-G factors when gstride > 0)
template <typename R>
__global__ void banded_solve_kernel(const R *Lb, size_t gstride, int order, int nb, int ng, int ldg,
                                    int nbands, const typename V2<R>::T *X, typename V2<R>::T *Y) {
    typedef typename V2<R>::T R2;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (g >= ldg) return;
    const int K = order;
    const R *L = Lb + gstride * g;
    const R2 *x = X + (size_t)b * nb * ldg;
    R2 *y = Y + (size_t)b * nb * ldg;
    if (g >= ng) {
        for (int j = 0; j < nb; ++j) y[(size_t)j * ldg + g] = czero<R2>();
        return;
    }
    for (int j = 0; j < nb; ++j) {
        R2 s = x[(size_t)j * ldg + g];
        for (int dd = 1; dd < K && dd <= j; ++dd) rfma(s, -L[(size_t)j * K + dd], y[(size_t)(j - dd) * ldg + g]);
        y[(size_t)j * ldg + g] = rscale(R(1) / L[(size_t)j * K], s);
    }
    for (int j = nb - 1; j >= 0; --j) {
        R2 s = y[(size_t)j * ldg + g];
        for (int dd = 1; dd < K && j + dd < nb; ++dd)
            rfma(s, -L[(size_t)(j + dd) * K + dd], y[(size_t)(j + dd) * ldg + g]);
        y[(size_t)j * ldg + g] = rscale(R(1) / L[(size_t)j * K], s);
    }
}

// ---------------------------------------------------------------------------
// host side
int cuda_fail(mb_handle *h, cudaError_t e) {
    h->last_cuda_error = cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? MB_ENOMEM : MB_ECUDA;
}

// Launch with accounting: counts the launch and, when profiling, brackets it
// with events on the launch stream.
#define MB_LAUNCH(h, s, kid, ...)                       \
    do {                                                \
        cudaEvent_t ev_;                                \
        prof_begin(h, s, kid, &ev_);                    \
        __VA_ARGS__;                                    \
        prof_end(h, s, kid, ev_);                       \
    } while (0)

#define MB_CUDA(call)                                  \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_fail(h, e_); \
    } while (0)

template <typename R>
static int upload(mb_handle *h, void **dst, const std::vector<double> &src) {
    std::vector<R> tmp(src.begin(), src.end());
    if (*dst) cudaFree(*dst);
    *dst = nullptr;
    if (tmp.empty()) return MB_OK;
    MB_CUDA(cudaMalloc(dst, tmp.size() * sizeof(R)));
    MB_CUDA(cudaMemcpy(*dst, tmp.data(), tmp.size() * sizeof(R), cudaMemcpyHostToDevice));
    return MB_OK;
}

template <typename R>
static int upload_complex(mb_handle *h, void **dst, const std::vector<cdouble> &src) {
    std::vector<R> tmp(2 * src.size());
    for (size_t i = 0; i < src.size(); ++i) {
        tmp[2 * i] = (R)src[i].real();
        tmp[2 * i + 1] = (R)src[i].imag();
    }
    if (*dst) cudaFree(*dst);
    *dst = nullptr;
    if (tmp.empty()) return MB_OK;
    MB_CUDA(cudaMalloc(dst, tmp.size() * sizeof(R)));
    MB_CUDA(cudaMemcpy(*dst, tmp.data(), tmp.size() * sizeof(R), cudaMemcpyHostToDevice));
    return MB_OK;
}

template <typename R>
static int upload_set(mb_handle *h, DevTables &t) {
    int rc;
    if ((rc = upload<R>(h, &t.Bq, h->Bq))) return rc;
    if ((rc = upload<R>(h, &t.Sband, h->Sb))) return rc;
    if ((rc = upload<R>(h, &t.Dband, h->Db))) return rc;
    if ((rc = upload<R>(h, &t.Lband, h->Lb))) return rc;
    {
        std::vector<double> lr(h->Lb);
        for (int j = 0; j < h->nb; ++j) lr[(size_t)j * h->order] = 1.0 / lr[(size_t)j * h->order];
        if ((rc = upload<R>(h, &t.Lrecip, lr))) return rc;
    }
    std::vector<double> q2((size_t)h->total_ldg, 0.0);
    std::vector<cdouble> qp;
    for (size_t ik = 0; ik < h->kp.size(); ++ik) {
        const KPoint &kp = h->kp[ik];
        for (int g = 0; g < kp.ng; ++g) q2[h->kofs[ik] + g] = kp.q2[g];
        qp.insert(qp.end(), kp.qproj.begin(), kp.qproj.end());
    }
    if ((rc = upload<R>(h, &t.q2, q2))) return rc;
    if ((rc = upload_complex<R>(h, &t.qproj, qp))) return rc;
    if ((rc = upload<R>(h, &t.zproj, h->zproj))) return rc;
    if ((rc = upload<R>(h, &t.E, h->Eproj))) return rc;
    const int nmax = std::max(h->n1, h->n2);
    std::vector<cdouble> tw(nmax / 2);
    for (int i = 0; i < nmax / 2; ++i) tw[i] = std::polar(1.0, 2.0 * 3.14159265358979323846 * i / nmax);
    if ((rc = upload_complex<R>(h, &t.tw, tw))) return rc;
    return MB_OK;
}

int upload_potential(mb_handle *h) {
    std::vector<double> vp, vn;
    vtable_permuted(h, vp);
    vtable_natural(h, vn);
    int rc;
    if ((rc = upload<double>(h, &h->t64.V, vp))) return rc;
    if ((rc = upload<float>(h, &h->t32.V, vp))) return rc;
    if ((rc = upload<double>(h, &h->t64.Vn, vn))) return rc;
    if ((rc = upload<float>(h, &h->t32.Vn, vn))) return rc;
    return MB_OK;
}

int upload_tables(mb_handle *h) {
    MB_CUDA(cudaSetDevice(h->device));
    int rc;
    if ((rc = upload_set<double>(h, h->t64))) return rc;
    if ((rc = upload_set<float>(h, h->t32))) return rc;
    if ((rc = upload_potential(h))) return rc;
    std::vector<int> goff((size_t)h->total_ldg, 0);
    for (size_t ik = 0; ik < h->kp.size(); ++ik)
        for (int g = 0; g < h->kp[ik].ng; ++g) goff[h->kofs[ik] + g] = h->kp[ik].goff[g];
    MB_CUDA(cudaMalloc(&h->d_goff, goff.size() * sizeof(int)));
    MB_CUDA(cudaMemcpy(h->d_goff, goff.data(), goff.size() * sizeof(int), cudaMemcpyHostToDevice));
    // grid rows that hold disc points, per k-point
    std::vector<int> rows;
    h->rows_ofs.assign(h->kp.size(), 0);
    h->nrows.assign(h->kp.size(), 0);
    h->rowmask.assign(h->kp.size(), 0ull);
    for (size_t ik = 0; ik < h->kp.size(); ++ik) {
        std::vector<char> used(h->n1, 0);
        for (int g = 0; g < h->kp[ik].ng; ++g) used[h->kp[ik].goff[g] / h->n2] = 1;
        h->rows_ofs[ik] = (int)rows.size();
        for (int r = 0; r < h->n1; ++r)
            if (used[r]) {
                rows.push_back(r);
                if (r < 64) h->rowmask[ik] |= 1ull << r;
            }
        h->nrows[ik] = (int)rows.size() - h->rows_ofs[ik];
    }
    MB_CUDA(cudaMalloc(&h->d_rows, rows.size() * sizeof(int)));
    MB_CUDA(cudaMemcpy(h->d_rows, rows.data(), rows.size() * sizeof(int), cudaMemcpyHostToDevice));
    upload_fft_twiddles();
    MB_CUDA(cudaGetLastError());
    return upload_proj_tables(h);
}

int ensure_precond(mb_handle *h) {
    if (h->pfac_ready) return MB_OK;
    std::vector<double> all;
    for (size_t ik = 0; ik < h->kp.size(); ++ik) {
        std::vector<double> f;
        precond_factors(h, (int)ik, h->precond_shift, f);
        all.insert(all.end(), f.begin(), f.end());
    }
    int rc;
    if ((rc = upload<double>(h, &h->t64.Pfac, all))) return rc;
    if ((rc = upload<float>(h, &h->t32.Pfac, all))) return rc;
    h->pfac_ready = true;
    return MB_OK;
}

static void free_set(DevTables &t) {
    void **ps[] = {&t.Bq, &t.V, &t.Vn, &t.tw, &t.Sband, &t.Dband, &t.Lband, &t.Lrecip, &t.q2, &t.qproj, &t.zproj, &t.E, &t.Pfac};
    for (void **p : ps) {
        if (*p) cudaFree(*p);
        *p = nullptr;
    }
}

void free_tables(mb_handle *h) {
    cudaSetDevice(h->device);
    free_set(h->t64);
    free_set(h->t32);
    if (h->d_goff) cudaFree(h->d_goff);
    h->d_goff = nullptr;
    if (h->d_rows) cudaFree(h->d_rows);
    h->d_rows = nullptr;
    if (h->d_projB) cudaFree(h->d_projB);
    h->d_projB = nullptr;
    if (h->d_tcerr) cudaFree(h->d_tcerr);
    h->d_tcerr = nullptr;
    if (h->scratch.ptr) cudaFree(h->scratch.ptr);
    h->scratch = Scratch();
}

int ensure_scratch(mb_handle *h, size_t bytes) {
    if (bytes <= h->scratch.bytes) return MB_OK;
    if (h->scratch.ptr) {
        MB_CUDA(cudaDeviceSynchronize());
        cudaFree(h->scratch.ptr);
    }
    h->scratch = Scratch();
    MB_CUDA(cudaMalloc(&h->scratch.ptr, bytes));
    h->scratch.bytes = bytes;
    return MB_OK;
}

// Launch plan of the plane kernel for one batched apply.
struct PlanePlan {
    bool reg = false;      // register-FFT kernel (else radix-2 shared-memory kernel)
    int bt = 1;            // bands per CTA
    int np = 1;            // planes in flight
    int chunk = 1, nchunks = 1;
    size_t smem = 0;
};

static PlanePlan plan_plane(const mb_handle *h, int nsel, int nbands, size_t c2, int maxldg, bool reg_ok) {
    PlanePlan p;
    const int K = h->order, P = h->nquad;
    const size_t NN = (size_t)h->n1 * h->n2;
    int ctas_per_sm = 1;
    // defaults, or the shape mb_autotune measured fastest for this batch
    const bool small = h->n1 <= 32 && h->n2 <= 32;
    int bt_max = small ? 2 : 1, waves = 2;
    auto it = h->tuned.find(std::make_tuple(nsel, nbands, c2 == 16 ? 1 : 0));
    if (it != h->tuned.end()) {
        bt_max = it->second.first;
        waves = it->second.second;
    }
    if (reg_ok) {
        const size_t plane_bytes = (size_t)h->n1 * (h->n2 + 1) * c2;
        ctas_per_sm = (small && c2 == 8) ? 2 : 1;     // matches the kernel's launch bounds
        for (int bt = bt_max; bt >= 1 && !p.reg; --bt) {
            size_t budget = (size_t)h->smem_optin / ctas_per_sm - 1024;
            size_t acc = (size_t)bt * K * maxldg * c2;
            if (acc + plane_bytes > budget) continue;
            const size_t meta = 8 + 8 * (2 * sizeof(int) + 8 * c2 / 2);   // per plane, rounded up below
            int np = (int)std::min<size_t>((size_t)bt * P, (budget - acc) / (plane_bytes + meta));
            if (np < 1) continue;
            p.reg = true;
            p.bt = bt;
            p.np = np;
            p.smem = acc + (size_t)np * plane_bytes + ((size_t)(np + 1) * 2 * sizeof(int) + (size_t)np * 8 * (c2 / 2) + 15) / 16 * 16;
        }
    }
    if (!p.reg) {
        ctas_per_sm = 1;
        const int nmax = std::max(h->n1, h->n2);
        const size_t fixed = (nmax / 2 + (size_t)K * maxldg) * c2;
        const size_t budget = (size_t)h->smem_optin;
        p.bt = 1;
        p.np = (int)std::min<size_t>((size_t)P, fixed < budget ? (budget - fixed) / (NN * c2) : 0);
        p.smem = fixed + (size_t)p.np * NN * c2;
    }
    const int pairs = nsel * ((nbands + p.bt - 1) / p.bt);
    const int want = waves * h->num_sms * ctas_per_sm;
    const int target = std::max(1, (want + pairs - 1) / pairs);
    p.chunk = std::max(K, (h->nint + target - 1) / target);
    if (p.chunk >= h->nint) p.chunk = h->nint;
    p.nchunks = (h->nint + p.chunk - 1) / p.chunk;
    return p;
}

static size_t per_k_scratch(const mb_handle *h, int ldg, int nbands, int nchunks, size_t c2) {
    size_t part = (size_t)nbands * std::max(0, nchunks - 1) * 2 * (h->order - 1) * ldg * c2;
    size_t w = (size_t)nbands * h->nb * std::max(1, h->nproj) * c2;
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    return al(part) + 2 * al(w);
}

size_t apply_scratch_bytes(const mb_handle *h, int nsel_max, int nbands, int prec) {
    size_t c2 = prec == MB_FP64 ? 16 : 8;
    int maxldg = 0;
    for (auto &k : h->kp) maxldg = std::max(maxldg, k.ldg);
    int nsel = std::min(nsel_max, kMaxK);
    bool reg = prec == MB_FP64 ? plane_reg_supported<double>(h->n1, h->n2) : plane_reg_supported<float>(h->n1, h->n2);
    PlanePlan p = plan_plane(h, nsel, nbands, c2, maxldg, reg);
    return (size_t)nsel * per_k_scratch(h, maxldg, nbands, p.nchunks, c2);
}

cudaError_t proj_tc_launch(mb_handle *h, int mode, int nsel, const int *iks, const KDesc *desc, int nbands,
                           cudaStream_t s);

template <typename R>
static int apply_H_launch(mb_handle *h, int nsel, const int *iks, const void *const *X, void *const *Y,
                          int nbands, cudaStream_t s, const DevTables &t, char *base, bool tensor = false);

// Scratch bytes one batched apply needs (boundary rows, projector overlaps W
// and coefficients C for every k-point of the group).
template <typename R>
static size_t apply_H_need(const mb_handle *h, int nsel, const int *iks, int nbands) {
    const size_t c2 = sizeof(typename V2<R>::T);
    int maxldg = 0;
    for (int i = 0; i < nsel; ++i) maxldg = std::max(maxldg, h->kp[iks[i]].ldg);
    const PlanePlan plan = plan_plane(h, nsel, nbands, c2, maxldg, plane_reg_supported<R>(h->n1, h->n2));
    return (size_t)nsel * per_k_scratch(h, maxldg, nbands, plan.nchunks, c2);
}

template <typename R>
static int apply_H_group(mb_handle *h, int nsel, const int *iks, const void *const *X, void *const *Y,
                         int nbands, cudaStream_t s, const DevTables &t, bool tensor = false) {
    int rc = ensure_scratch(h, apply_H_need<R>(h, nsel, iks, nbands));
    if (rc) return rc;
    return apply_H_launch<R>(h, nsel, iks, X, Y, nbands, s, t, reinterpret_cast<char *>(h->scratch.ptr), tensor);
}

// Scratch need of a single-k-point apply, and the apply itself on a scratch
// region supplied by the caller of this function (no allocation here).
size_t apply_H_scratch_need(const mb_handle *h, int ik, int nbands, int prec) {
    return prec == MB_FP64 ? apply_H_need<double>(h, 1, &ik, nbands) : apply_H_need<float>(h, 1, &ik, nbands);
}

int apply_H_on_scratch(mb_handle *h, int ik, const void *X, void *Y, int nbands, int prec, cudaStream_t s,
                       void *scratch) {
    const void *xs[1] = {X};
    void *ys[1] = {Y};
    return prec == MB_FP64
               ? apply_H_launch<double>(h, 1, &ik, xs, ys, nbands, s, h->t64, reinterpret_cast<char *>(scratch))
               : apply_H_launch<float>(h, 1, &ik, xs, ys, nbands, s, h->t32, reinterpret_cast<char *>(scratch),
                                       prec == MB_BF16);
}

template <typename R>
static int apply_H_launch(mb_handle *h, int nsel, const int *iks, const void *const *X, void *const *Y,
                          int nbands, cudaStream_t s, const DevTables &t, char *base, bool tensor) {
    typedef typename V2<R>::T R2;
    const size_t c2 = sizeof(R2);
    KDesc desc[kMaxK];
    size_t off = 0;
    int maxldg = 0;
    for (int i = 0; i < nsel; ++i) maxldg = std::max(maxldg, h->kp[iks[i]].ldg);
    const PlanePlan plan = plan_plane(h, nsel, nbands, c2, maxldg, plane_reg_supported<R>(h->n1, h->n2));
    const int chunk = plan.chunk, nchunks = plan.nchunks;
    if (plan.np < 1) return MB_EUNSUPPORTED;
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    for (int i = 0; i < nsel; ++i) {
        const KPoint &kp = h->kp[iks[i]];
        KDesc &d = desc[i];
        d.X = X[i];
        d.Y = Y[i];
        d.ng = kp.ng;
        d.ldg = kp.ldg;
        d.kofs = h->kofs[iks[i]];
        d.qofs = h->qofs[iks[i]];
        d.rows_ofs = h->rows_ofs[iks[i]];
        d.nrows = h->nrows[iks[i]];
        d.rowmask = h->rowmask[iks[i]];
        d.rows_magic = (unsigned)((1ull << 32) / (unsigned)std::max(1, d.nrows) + 1);
        size_t part = (size_t)nbands * std::max(0, nchunks - 1) * 2 * (h->order - 1) * kp.ldg * c2;
        size_t w = (size_t)nbands * h->nb * std::max(1, h->nproj) * c2;
        d.part = base + off;
        off += al(part);
        d.W = base + off;
        off += al(w);
        d.C = base + off;
        off += al(w);
    }
    // projector overlaps first (they read X only)
    if (h->nproj > 0) {
        GemmArgs<R> ga;
        ga.Q = reinterpret_cast<const R2 *>(t.qproj);
        ga.mode = 0;
        ga.nb = h->nb;
        ga.nbands = nbands;
        ga.nproj = h->nproj;
        std::copy(desc, desc + nsel, ga.d);
        dim3 grid((nbands * h->nb + 63) / 64, (h->nproj + 63) / 64, nsel);
        if (tensor) {
            cudaError_t e = cudaSuccess;
            MB_LAUNCH(h, s, KN_PROJ, e = proj_tc_launch(h, 0, nsel, iks, desc, nbands, s));
            MB_CUDA(e);
        } else {
            MB_LAUNCH(h, s, KN_PROJ, zgemm_kernel<R><<<grid, 256, 0, s>>>(ga));
        }
        CoefArgs<R> ca;
        ca.zproj = reinterpret_cast<const R *>(t.zproj);
        ca.E = reinterpret_cast<const R *>(t.E);
        ca.nb = h->nb;
        ca.nbands = nbands;
        ca.nproj = h->nproj;
        std::copy(desc, desc + nsel, ca.d);
        MB_LAUNCH(h, s, KN_COEF, coef_kernel<R><<<dim3((nbands * h->nproj + 127) / 128, nsel), 128, 0, s>>>(ca));
    }
    // local potential through the planes
    PlaneArgs<R> pa;
    pa.Bq = reinterpret_cast<const R *>(t.Bq);
    pa.V = reinterpret_cast<const R *>(t.V);
    pa.Vn = reinterpret_cast<const R *>(t.Vn);
    pa.rows = h->d_rows;
    pa.tw = reinterpret_cast<const R2 *>(t.tw);
    pa.goff = h->d_goff;
    pa.n1 = h->n1;
    pa.n2 = h->n2;
    pa.l1 = h->l1;
    pa.l2 = h->l2;
    pa.nmax = std::max(h->n1, h->n2);
    pa.order = h->order;
    pa.nquad = h->nquad;
    pa.nint = h->nint;
    pa.nb = h->nb;
    pa.nbands = nbands;
    pa.nchunks = nchunks;
    pa.chunk = chunk;
    pa.ldg_max = maxldg;
    pa.nsel = nsel;
    pa.bt = plan.bt;
    pa.np = plan.np;
    std::copy(desc, desc + nsel, pa.d);
    if (plan.reg) {
        const unsigned grid = (unsigned)(nsel * ((nbands + plan.bt - 1) / plan.bt) * nchunks);
        cudaError_t e = cudaSuccess;
        MB_LAUNCH(h, s, KN_PLANE, e = plane_reg_launch<R>(pa, grid, plan.smem, s));
        MB_CUDA(e);
    } else {
        MB_CUDA(smem_limit_once((const void *)plane_kernel<R>, h->device, h->smem_optin));
        MB_LAUNCH(h, s, KN_PLANE, plane_kernel<R><<<nsel * nbands * nchunks, 256, plan.smem, s>>>(pa));
    }
    EpiArgs<R> ea;
    ea.Sband = reinterpret_cast<const R *>(t.Sband);
    ea.Dband = reinterpret_cast<const R *>(t.Dband);
    ea.q2 = reinterpret_cast<const R *>(t.q2);
    ea.order = h->order;
    ea.nb = h->nb;
    ea.nbands = nbands;
    ea.nchunks = nchunks;
    ea.chunk = chunk;
    ea.nint = h->nint;
    std::copy(desc, desc + nsel, ea.d);
    MB_LAUNCH(h, s, KN_EPILOGUE, epilogue_kernel<R><<<dim3(h->nb, nbands, nsel), 256, 0, s>>>(ea));
    if (h->nproj > 0) {
        GemmArgs<R> ga;
        ga.Q = reinterpret_cast<const R2 *>(t.qproj);
        ga.mode = 1;
        ga.nb = h->nb;
        ga.nbands = nbands;
        ga.nproj = h->nproj;
        std::copy(desc, desc + nsel, ga.d);
        dim3 grid((nbands * h->nb + 63) / 64, (maxldg + 63) / 64, nsel);
        if (tensor) {
            cudaError_t e = cudaSuccess;
            MB_LAUNCH(h, s, KN_BACKPROJ, e = proj_tc_launch(h, 1, nsel, iks, desc, nbands, s));
            MB_CUDA(e);
        } else {
            MB_LAUNCH(h, s, KN_BACKPROJ, zgemm_kernel<R><<<grid, 256, 0, s>>>(ga));
        }
    }
    MB_CUDA(cudaGetLastError());
    return MB_OK;
}

int apply_H_batch(mb_handle *h, int nsel, const int *iks, const void *const *X, void *const *Y,
                  int nbands, int prec, cudaStream_t s) {
    if (nsel <= 0 || !iks || !X || !Y) return MB_EINVAL;
    if (nbands <= 0 || nbands > h->max_bands) return MB_EINVAL;
    if (prec != MB_FP64 && prec != MB_FP32 && prec != MB_BF16) return MB_EINVAL;
    for (int i = 0; i < nsel; ++i) {
        if (iks[i] < 0 || iks[i] >= (int)h->kp.size() || !X[i] || !Y[i]) return MB_EINVAL;
        if (X[i] == Y[i]) return MB_EINVAL;
    }
    MB_CUDA(cudaSetDevice(h->device));
    for (int i0 = 0; i0 < nsel; i0 += kMaxK) {
        int n = std::min(kMaxK, nsel - i0);
        int rc = prec == MB_FP64 ? apply_H_group<double>(h, n, iks + i0, X + i0, Y + i0, nbands, s, h->t64)
                                 : apply_H_group<float>(h, n, iks + i0, X + i0, Y + i0, nbands, s, h->t32,
                                                        prec == MB_BF16);
        if (rc) return rc;
    }
    return MB_OK;
}

int apply_banded(mb_handle *h, int which, int ik, const void *X, void *Y, int nbands, int prec,
                 cudaStream_t s) {
    if (ik < 0 || ik >= (int)h->kp.size() || !X || !Y || nbands <= 0) return MB_EINVAL;
    if (prec != MB_FP64 && prec != MB_FP32 && prec != MB_BF16) return MB_EINVAL;
    if (which != BAND_S && X == Y) return MB_EINVAL;
    MB_CUDA(cudaSetDevice(h->device));
    const KPoint &kp = h->kp[ik];
    dim3 grid((kp.ldg + 127) / 128, nbands);
    if (which != BAND_S && which != BAND_SINV) return MB_EINVAL;
    if (prec == MB_FP64) {
        const DevTables &t = h->t64;
        auto x = reinterpret_cast<const double2 *>(X);
        auto y = reinterpret_cast<double2 *>(Y);
        if (which == BAND_S)
            MB_LAUNCH(h, s, KN_BANDED, banded_S_kernel<double><<<grid, 128, 0, s>>>((const double *)t.Sband, h->order, h->nb, kp.ng, kp.ldg, nbands, x, y));
        else
            MB_LAUNCH(h, s, KN_BANDED, banded_solve_kernel<double><<<grid, 128, 0, s>>>((const double *)t.Lband, 0, h->order, h->nb, kp.ng, kp.ldg, nbands, x, y));
    } else {
        const DevTables &t = h->t32;
        auto x = reinterpret_cast<const float2 *>(X);
        auto y = reinterpret_cast<float2 *>(Y);
        if (which == BAND_S)
            MB_LAUNCH(h, s, KN_BANDED, banded_S_kernel<float><<<grid, 128, 0, s>>>((const float *)t.Sband, h->order, h->nb, kp.ng, kp.ldg, nbands, x, y));
        else
            MB_LAUNCH(h, s, KN_BANDED, banded_solve_kernel<float><<<grid, 128, 0, s>>>((const float *)t.Lband, 0, h->order, h->nb, kp.ng, kp.ldg, nbands, x, y));
    }
    MB_CUDA(cudaGetLastError());
    return MB_OK;
}

}  // namespace mb

// ---------------------------------------------------------------------------
// mb_autotune: time the candidate plane-kernel launch shapes for a batch of
// `nbands` bands at every k-point of the handle and keep the fastest.
namespace mb {
int autotune(mb_handle *h, int nbands, int prec, int *best_bt, int *best_waves, double *best_ms) {
    if (nbands < 1 || nbands > h->max_bands) return MB_EINVAL;
    if (prec != MB_FP64 && prec != MB_FP32 && prec != MB_BF16) return MB_EINVAL;
    MB_CUDA(cudaSetDevice(h->device));
    const int nk = (int)h->kp.size();
    const size_t c2 = prec == MB_FP64 ? 16 : 8;
    std::vector<void *> X(nk, nullptr), Y(nk, nullptr);
    std::vector<int> iks(nk);
    int rc = MB_OK;
    for (int i = 0; i < nk && rc == MB_OK; ++i) {
        iks[i] = i;
        size_t bytes = (size_t)nbands * h->nb * h->kp[i].ldg * c2;
        if (cudaMalloc(&X[i], bytes) != cudaSuccess || cudaMalloc(&Y[i], bytes) != cudaSuccess) rc = MB_ENOMEM;
        else cudaMemset(X[i], 0, bytes);
    }
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == MB_OK && (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
                        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        rc = MB_ECUDA;
    const bool small = h->n1 <= 32 && h->n2 <= 32;
    const auto key = std::make_tuple(std::min(nk, kMaxK), nbands, c2 == 16 ? 1 : 0);
    double best = 1e300;
    std::pair<int, int> bestp(small ? 2 : 1, 2);
    for (int bt = small ? 2 : 1; bt >= 1 && rc == MB_OK; --bt)
        for (int waves : {1, 2, 4, 8}) {
            h->tuned[key] = std::make_pair(bt, waves);
            for (int w = 0; w < 2 && rc == MB_OK; ++w)
                rc = apply_H_batch(h, nk, iks.data(), (const void *const *)X.data(), Y.data(), nbands, prec, s);
            if (rc) break;
            cudaEventRecord(e0, s);
            for (int r = 0; r < 5 && rc == MB_OK; ++r)
                rc = apply_H_batch(h, nk, iks.data(), (const void *const *)X.data(), Y.data(), nbands, prec, s);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) rc = MB_ECUDA;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rc == MB_OK && ms / 5 < best) {
                best = ms / 5;
                bestp = std::make_pair(bt, waves);
            }
        }
    h->tuned[key] = bestp;
    if (best_bt) *best_bt = bestp.first;
    if (best_waves) *best_waves = bestp.second;
    if (best_ms) *best_ms = best;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    for (int i = 0; i < nk; ++i) {
        if (X[i]) cudaFree(X[i]);
        if (Y[i]) cudaFree(Y[i]);
    }
    return rc;
}
}  // namespace mb

extern "C" int mb_autotune(mb_handle *h, int nbands, int prec, int *best_bt, int *best_waves, double *best_ms) {
    if (!h) return MB_EINVAL;
    return mb::autotune(h, nbands, prec, best_bt, best_waves, best_ms);
}
