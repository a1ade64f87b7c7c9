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
//  epilogue       kinetic term Eq. (9) (banded in j, diagonal in G), the
//                 boundary-row sums and the back-projection of Eq. (17).
//  nl_zx/nl_coef  projector overlaps of Eq. (17) through the factorized
//                 projectors u_p(G, j) = z_p(j) q_p(G), one j-contraction per
//                 distinct z factor (the tensor-core variant, tc_gemm.cu,
//                 contracts the unfactorized (band, j) x G block instead).
//  banded_*       S (Eqs. (7)-(8)), S^-1 and the eigensolver's
//                 preconditioner through banded Cholesky factors.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>

#include "apply_common.cuh"
#include "cplx.cuh"
#include "fft_smem.cuh"
#include "mb_internal.h"

namespace mb {

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
    const int t0 = chunk_begin(c, a.nint, a.nchunks), t1 = chunk_begin(c + 1, a.nint, a.nchunks);

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
// Kleinman-Bylander term of Eq. (17).  Every projector is a sum of
// separable terms u_p(G, j) = sum_{t in p} z_t(j) q_t(G) (one term for 1s
// and p, two for 2s), and the z factors repeat (s, p_x, p_y of one atom; all
// atoms at one height and radius), so with f(t) the distinct z factor of
// term t:
//   Zx[b][f][G] = sum_j z_f(j) X[b][j][G]                            (nl_zx)
//   F_p(b)      = sum_{t in p} sum_G conj(q_t(G)) Zx[b][f(t)][G]
//   c_p(b)      = E_p F_p(b) + E'_p F_{partner(p)}(b)                (nl_coef)
//   Y[b][j][G] += sum_f z_f(j) sum_{t: f(t)=f} c_{p(t)}(b) q_t(G)     (epilogue)
// which is sum_pq E_pq u_p (u_q^H X) with nb*nz + nterm (not nb*nterm)
// multiply-adds per (band, G).
template <typename R> struct NlArgs {
    const R *zf;                    // nz x nb distinct z factors
    const R *E;                     // nkb strengths E_p, then nkb couplings E'_p
    const int *pgroup;              // nterm: f(t)
    const int *partner;             // nkb: coupled projector or -1
    const int *pstart, *plist;      // terms of projector p: plist[pstart[p] .. pstart[p+1])
    const typename V2<R>::T *Q;     // q_t(G), all k (offset qofs)
    int nb, nbands, nterm, nkb, nz, nseg;
    KDesc d[kMaxK];
};

// Zx for 64 consecutive G of one (band, k-point): threadIdx.y takes one run
// of rows j, and the runs' partial sums are added in run order through
// shared memory.
template <typename R, int NZB>
__global__ void __launch_bounds__(512) nl_zx_kernel(const __grid_constant__ NlArgs<R> a) {
    typedef typename V2<R>::T R2;
    extern __shared__ __align__(16) unsigned char nsm[];
    R2 *red = reinterpret_cast<R2 *>(nsm);                  // nseg x NZB x 64 partial sums
    R *zs = reinterpret_cast<R *>(red + a.nseg * NZB * 64); // nz x nb
    const int tx = threadIdx.x, seg = threadIdx.y;
    const int tid = seg * 64 + tx, nthr = 64 * a.nseg;
    const int g = blockIdx.x * 64 + tx, b = blockIdx.y;
    const KDesc &d = a.d[blockIdx.z];
    const int ldg = d.ldg, nb = a.nb;
    for (int e = tid; e < a.nz * nb; e += nthr) zs[e] = a.zf[e];
    __syncthreads();
    const int j0 = (seg * nb) / a.nseg, j1 = ((seg + 1) * nb) / a.nseg, nr = j1 - j0;
    const bool live = g < d.ng;
    const R2 *X = reinterpret_cast<const R2 *>(d.X) + ((size_t)b * nb + j0) * ldg + g;
    for (int f0 = 0; f0 < a.nz; f0 += NZB) {
        R2 acc[NZB];
#pragma unroll
        for (int f = 0; f < NZB; ++f) acc[f] = czero<R2>();
        if (live) {
            int j = 0;
            for (; j + 4 <= nr; j += 4) {
                R2 x[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) x[u] = X[(size_t)(j + u) * ldg];
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int f = 0; f < NZB; ++f)
                        if (f0 + f < a.nz) rfma(acc[f], zs[(f0 + f) * nb + j0 + j + u], x[u]);
            }
            for (; j < nr; ++j) {
                const R2 x = X[(size_t)j * ldg];
#pragma unroll
                for (int f = 0; f < NZB; ++f)
                    if (f0 + f < a.nz) rfma(acc[f], zs[(f0 + f) * nb + j0 + j], x);
            }
        }
        // every factor's partial sums at once, then each output summed over
        // the segments in segment order (one barrier per factor chunk)
#pragma unroll
        for (int f = 0; f < NZB; ++f) red[(seg * NZB + f) * 64 + tx] = acc[f];
        __syncthreads();
        const int nzc = min(NZB, a.nz - f0);
        R2 *Zb = reinterpret_cast<R2 *>(d.W) + (size_t)b * a.nz * ldg + blockIdx.x * 64;
        for (int o = tid; o < nzc * 64; o += nthr) {
            const int f = o / 64, x = o % 64;
            if (blockIdx.x * 64 + x >= d.ng) continue;
            R2 t = red[f * 64 + x];
            for (int sg = 1; sg < a.nseg; ++sg) t = t + red[(sg * NZB + f) * 64 + x];
            Zb[(size_t)(f0 + f) * ldg + x] = t;
        }
        __syncthreads();
    }
}

// F_p(b) of one projector (all its terms) summed by one warp in a fixed order
template <typename R>
__device__ __forceinline__ typename V2<R>::T nl_overlap(const NlArgs<R> &a, const KDesc &d, int b, int p,
                                                        int lane) {
    typedef typename V2<R>::T R2;
    const int ldg = d.ldg;
    R2 s = czero<R2>();
    for (int i = a.pstart[p]; i < a.pstart[p + 1]; ++i) {
        const int t = a.plist[i];
        const R2 *z = reinterpret_cast<const R2 *>(d.W) + ((size_t)b * a.nz + a.pgroup[t]) * ldg;
        const R2 *q = a.Q + d.qofs + (size_t)t * ldg;
#pragma unroll 4
        for (int g = lane; g < d.ng; g += 32) {
            const R2 qg = q[g];
            cfma(s, mk(qg.x, -qg.y), z[g]);
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        s.x += __shfl_down_sync(0xffffffffu, s.x, off);
        s.y += __shfl_down_sync(0xffffffffu, s.y, off);
    }
    return s;   // complete in lane 0
}

// one warp per (band, k-point, projector): c_p = E_p F_p + E'_p F_partner
template <typename R>
__global__ void __launch_bounds__(256) nl_coef_kernel(const __grid_constant__ NlArgs<R> a) {
    typedef typename V2<R>::T R2;
    const int b = blockIdx.x;
    const KDesc &d = a.d[blockIdx.y];
    const int p = blockIdx.z * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (p >= a.nkb) return;
    R2 c = rscale(a.E[p], nl_overlap(a, d, b, p, lane));
    const int q = a.partner[p];
    if (q >= 0) {
        const R2 fq = nl_overlap(a, d, b, q, lane);
        rfma(c, a.E[a.nkb + p], fq);
    }
    if (lane == 0) reinterpret_cast<R2 *>(d.C)[(size_t)b * a.nkb + p] = c;
}

// R[b][f][G] = sum_{t: f(t)=f} c_{p(t)}(b) q_t(G), written over Zx (which
// nl_coef has consumed); one thread per (band, z factor, G).
template <typename R>
__global__ void __launch_bounds__(128) nl_back_kernel(const __grid_constant__ NlArgs<R> a, const int *zstart,
                                                      const int *zlist, const int *tproj) {
    typedef typename V2<R>::T R2;
    extern __shared__ __align__(16) unsigned char bsm[];
    R2 *cl = reinterpret_cast<R2 *>(bsm);                     // c_{p(t)} of the factor's terms
    int *tl = reinterpret_cast<int *>(cl + a.nterm);          // the terms
    const int g = blockIdx.x * blockDim.x + threadIdx.x, f = blockIdx.y;
    const int b = blockIdx.z % a.nbands;
    const KDesc &d = a.d[blockIdx.z / a.nbands];
    const int i0 = zstart[f], n = zstart[f + 1] - i0;
    const R2 *c = reinterpret_cast<const R2 *>(d.C) + (size_t)b * a.nkb;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int t = zlist[i0 + e];
        tl[e] = t;
        cl[e] = c[tproj[t]];
    }
    __syncthreads();
    if (g >= d.ldg) return;
    R2 r = czero<R2>();
    if (g < d.ng) {
        const R2 *Qg = a.Q + d.qofs + g;
#pragma unroll 4
        for (int e = 0; e < n; ++e) cfma(r, cl[e], Qg[(size_t)tl[e] * d.ldg]);
    }
    reinterpret_cast<R2 *>(d.W)[((size_t)b * a.nz + f) * d.ldg + g] = r;
}

// ---------------------------------------------------------------------------
// epilogue: Y[j] = local(j) + (D/2 + |k+G|^2/2 S) X (Eq. (9)) + KB term.
// One thread per (band, G, run of rows j); the local part comes from Y (rows
// inside one plane-kernel run) or from the two boundary partials (rows shared
// by neighbouring runs), added in a fixed order.  `base` = 0 runs only the KB
// term for the distinct z factors [f0, f1) (when there are more than NZB).
constexpr int kMaxEpiRows = 1024;   // B-splines the epilogue's row table covers
template <typename R> struct EpiArgs {
    const R *Sband, *Dband, *q2;
    const R *zf;                    // nz x nb
    int order, nb, nbands, nchunks, nint, nz, f0, f1, base, njseg;
    KDesc d[kMaxK];
    short src[kMaxEpiRows];         // row j: its first boundary partial row, or -1 (its own Y row)
};

// N values (N a multiple of 4) from 16-byte aligned shared memory in 128-bit
// loads (FP32) or 128-bit pairs (FP64)
template <typename R, int N> __device__ __forceinline__ void load_row(const R *p, R (&out)[N]);
template <typename R, int N> __device__ __forceinline__ void load_row(const R *p, R (&out)[N]) {
    if constexpr (sizeof(R) == 4) {
#pragma unroll
        for (int q = 0; q < N / 4; ++q) {
            const float4 v = reinterpret_cast<const float4 *>(p)[q];
            out[4 * q] = v.x;
            out[4 * q + 1] = v.y;
            out[4 * q + 2] = v.z;
            out[4 * q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < N / 2; ++q) {
            const double2 v = reinterpret_cast<const double2 *>(p)[q];
            out[2 * q] = v.x;
            out[2 * q + 1] = v.y;
        }
    }
}

// HW = largest half-width of the band (order - 1) the instance handles.  A
// thread takes at most RM consecutive rows j and issues every load before it
// computes: the X rows j0-HW .. j0+RM-1+HW (clamped to the basis: the band
// coefficients are zero outside it) and the local part of each row, so it
// waits on memory once.  Per row, the band coefficients (padded to a multiple
// of 4) and the z factors come from shared memory in 128-bit loads at
// compile-time offsets, and where the row's local part lives (its Y row or
// the two boundary partials) is decided once per CTA.
template <typename R, int NZB, int HW, int RM>
__global__ void __launch_bounds__(64) epilogue_kernel(const __grid_constant__ EpiArgs<R> a) {
    typedef typename V2<R>::T R2;
    constexpr int WW = 2 * HW + 1, WP = (WW + 3) / 4 * 4;
    extern __shared__ __align__(16) unsigned char esm[];
    R *cS = reinterpret_cast<R *>(esm);                 // [RM][WP]: S[j][j+o], o = i - HW
    R *cD = cS + RM * WP;                               // [RM][WP]: D[j][j+o] / 2
    R *zs = cD + RM * WP;                               // [RM][NZB]: z_f(j), zero for f >= nf
    const int b = blockIdx.y / a.njseg, js = blockIdx.y % a.njseg;
    const KDesc &d = a.d[blockIdx.z];
    const int K = a.order, W = 2 * K - 1, ldg = d.ldg, nb = a.nb;
    const int j0 = (js * nb) / a.njseg, j1 = ((js + 1) * nb) / a.njseg, nr = j1 - j0;
    const int nf = a.f1 - a.f0;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = g < d.ng;
    // every global load of the thread first, then the shared coefficient
    // tables: the thread waits on memory once
    R2 r[NZB];                  // KB: R[b][f][G] = sum_{t: f(t) = f} c_{p(t)}(b) q_t(G) (nl_back)
    R2 xw[RM + 2 * HW];         // xw[i] = X[j0 - HW + i]
    R2 loc[RM];
    R hq = R(0);
    R2 *Y = reinterpret_cast<R2 *>(d.Y) + ((size_t)b * nb + j0) * ldg + g;
    if (live) {
        const R2 *Rg = reinterpret_cast<const R2 *>(d.W) + ((size_t)b * a.nz + a.f0) * ldg + g;
#pragma unroll
        for (int f = 0; f < NZB; ++f) r[f] = f < nf ? Rg[(size_t)f * ldg] : czero<R2>();
        hq = R(0.5) * a.q2[d.kofs + g];
        if (a.base) {
            const R2 *X = reinterpret_cast<const R2 *>(d.X) + (size_t)b * nb * ldg + g;
#pragma unroll
            for (int i = 0; i < RM + 2 * HW; ++i) {
                const int row = min(max(j0 - HW + i, 0), nb - 1);
                xw[i] = X[(size_t)row * ldg];
            }
            const R2 *part = reinterpret_cast<const R2 *>(d.part) + (size_t)b * (a.nchunks - 1) * 2 * (K - 1) * ldg + g;
#pragma unroll
            for (int rr = 0; rr < RM; ++rr) {
                if (rr >= nr) break;
                const int s = a.src[j0 + rr];
                loc[rr] = s < 0 ? Y[(size_t)rr * ldg] : part[(size_t)s * ldg] + part[(size_t)(s + K - 1) * ldg];
            }
        } else {
#pragma unroll
            for (int rr = 0; rr < RM; ++rr) loc[rr] = rr < nr ? Y[(size_t)rr * ldg] : czero<R2>();
        }
    }
    for (int e = threadIdx.x; e < RM * WP; e += blockDim.x) {
        const int rr = e / WP, i = e % WP, dd = i - HW + K - 1;
        const bool in = a.base && rr < nr && i < WW && dd >= 0 && dd < W;
        cS[e] = in ? a.Sband[(size_t)(j0 + rr) * W + dd] : R(0);
        cD[e] = in ? R(0.5) * a.Dband[(size_t)(j0 + rr) * W + dd] : R(0);
    }
    for (int e = threadIdx.x; e < RM * NZB; e += blockDim.x) {
        const int rr = e / NZB, f = e % NZB;
        zs[e] = (rr < nr && f < nf) ? a.zf[(size_t)(a.f0 + f) * nb + j0 + rr] : R(0);
    }
    __syncthreads();
    if (g >= ldg) return;
    if (!live) {
        if (a.base)
            for (int rr = 0; rr < nr; ++rr) Y[(size_t)rr * ldg] = czero<R2>();
        return;
    }
#pragma unroll
    for (int rr = 0; rr < RM; ++rr) {
        if (rr >= nr) break;
        R2 v = loc[rr];
        if (a.base) {
            R sr[WP], dr[WP];
            load_row<R, WP>(cS + rr * WP, sr);
            load_row<R, WP>(cD + rr * WP, dr);
#pragma unroll
            for (int i = 0; i < WW; ++i) rfma(v, fma(hq, sr[i], dr[i]), xw[rr + i]);
        }
        R zr[NZB];
        load_row<R, NZB>(zs + rr * NZB, zr);
#pragma unroll
        for (int f = 0; f < NZB; ++f) rfma(v, zr[f], r[f]);
        Y[(size_t)rr * ldg] = v;
    }
}

// Tensor-core path, per term t of projector p: W[(b,j)][t] = sum_G X conj(q_t);
// F_p(b) = sum_{t in p} sum_j z_t(j) W[(b,j)][t];
// c_p = E_p F_p + E'_p F_partner;  C[(b,j)][t] = z_t(j) c_{p(t)}(b)
template <typename R> struct CoefArgs {
    const R *zproj, *E;
    const int *partner, *pstart, *plist;
    int nb, nbands, nterm, nkb;
    KDesc d[kMaxK];
};

template <typename R>
__device__ __forceinline__ typename V2<R>::T coef_overlap(const CoefArgs<R> &a, const KDesc &d, int b, int p) {
    typedef typename V2<R>::T R2;
    const R2 *W = reinterpret_cast<const R2 *>(d.W) + (size_t)b * a.nb * a.nterm;
    R2 F = czero<R2>();
    for (int i = a.pstart[p]; i < a.pstart[p + 1]; ++i) {
        const int t = a.plist[i];
        const R *z = a.zproj + (size_t)t * a.nb;
        for (int j = 0; j < a.nb; ++j) rfma(F, z[j], W[(size_t)j * a.nterm + t]);
    }
    return F;
}

template <typename R>
__global__ void coef_kernel(const __grid_constant__ CoefArgs<R> a) {
    typedef typename V2<R>::T R2;
    const int ks = blockIdx.y;
    const KDesc &d = a.d[ks];
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= a.nbands * a.nkb) return;
    const int b = idx / a.nkb, p = idx % a.nkb;
    R2 c = rscale(a.E[p], coef_overlap(a, d, b, p));
    if (a.partner[p] >= 0) rfma(c, a.E[a.nkb + p], coef_overlap(a, d, b, a.partner[p]));
    R2 *C = reinterpret_cast<R2 *>(d.C) + (size_t)b * a.nb * a.nterm;
    for (int i = a.pstart[p]; i < a.pstart[p + 1]; ++i) {
        const int t = a.plist[i];
        const R *z = a.zproj + (size_t)t * a.nb;
        for (int j = 0; j < a.nb; ++j) C[(size_t)j * a.nterm + t] = rscale(z[j], c);
    }
}

// ---------------------------------------------------------------------------
// banded solve along j (the S^-1 of orders without the tile kernel)
// L L^T y = x with L[j][j-d] = Lb[(j*K + d)], one thread per (band, G)
// column; the recurrence keeps the last K-1 results in registers and runs
// over tiles of PD rows whose right-hand sides are all loaded first.
template <typename R>
__global__ void __launch_bounds__(64) banded_solve_kernel(const R *Lb, int order, int nb, int ng, int ldg,
                                                          int nbands, const typename V2<R>::T *X,
                                                          typename V2<R>::T *Y) {
    typedef typename V2<R>::T R2;
    constexpr int KM = 8, PD = 8;            // largest order; rows per tile
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (g >= ldg) return;
    const int K = order;
    const R2 *x = X + (size_t)b * nb * ldg + g;
    R2 *y = Y + (size_t)b * nb * ldg + g;
    if (g >= ng) {
        for (int j = 0; j < nb; ++j) y[(size_t)j * ldg] = czero<R2>();
        return;
    }
    R2 win[KM];                              // win[d-1] = y[j - d]
#pragma unroll
    for (int i = 0; i < KM; ++i) win[i] = czero<R2>();
    for (int j0 = 0; j0 < nb; j0 += PD) {
        R2 xs[PD];
#pragma unroll
        for (int u = 0; u < PD; ++u) xs[u] = j0 + u < nb ? x[(size_t)(j0 + u) * ldg] : czero<R2>();
#pragma unroll
        for (int u = 0; u < PD; ++u) {
            const int j = j0 + u;
            if (j >= nb) break;
            R2 s = xs[u];
#pragma unroll
            for (int dd = 1; dd < KM; ++dd)
                if (dd < K && dd <= j) rfma(s, -__ldg(&Lb[(size_t)j * K + dd]), win[dd - 1]);
            const R2 yj = rscale(R(1) / __ldg(&Lb[(size_t)j * K]), s);
            y[(size_t)j * ldg] = yj;
#pragma unroll
            for (int i = KM - 1; i > 0; --i) win[i] = win[i - 1];
            win[0] = yj;
        }
    }
#pragma unroll
    for (int i = 0; i < KM; ++i) win[i] = czero<R2>();
    for (int j1 = nb - 1; j1 >= 0; j1 -= PD) {
        R2 xs[PD];
#pragma unroll
        for (int u = 0; u < PD; ++u) xs[u] = j1 - u >= 0 ? y[(size_t)(j1 - u) * ldg] : czero<R2>();
#pragma unroll
        for (int u = 0; u < PD; ++u) {
            const int j = j1 - u;
            if (j < 0) break;
            R2 s = xs[u];
#pragma unroll
            for (int dd = 1; dd < KM; ++dd)
                if (dd < K && j + dd < nb) rfma(s, -__ldg(&Lb[(size_t)(j + dd) * K + dd]), win[dd - 1]);
            const R2 zj = rscale(R(1) / __ldg(&Lb[(size_t)j * K]), s);
            y[(size_t)j * ldg] = zj;
#pragma unroll
            for (int i = KM - 1; i > 0; --i) win[i] = win[i - 1];
            win[0] = zj;
        }
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


cudaMemPool_t mb_pool(int device) {
    static std::mutex mu;
    static std::map<int, cudaMemPool_t> pools;
    std::lock_guard<std::mutex> lock(mu);
    auto it = pools.find(device);
    if (it != pools.end()) return it->second;
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
    uint64_t keep = 16ull << 30;     // up to 16 GiB of freed memory stays reserved for the next handle
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[device] = pool;
    return pool;
}

void dev_free(mb_handle *h, void **p) {
    if (*p) cudaFreeAsync(*p, h->hs);
    *p = nullptr;
}

int dev_upload(mb_handle *h, void **dst, const void *src, size_t bytes) {
    dev_free(h, dst);
    if (!bytes) return MB_OK;
    cudaMemPool_t pool = mb_pool(h->device);
    if (!pool) return MB_ECUDA;
    MB_CUDA(cudaMallocFromPoolAsync(dst, bytes, pool, h->hs));
    if (src) MB_CUDA(cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, h->hs));
    return MB_OK;
}

template <typename R>
static int upload(mb_handle *h, void **dst, const std::vector<double> &src) {
    std::vector<R> tmp(src.begin(), src.end());
    return dev_upload(h, dst, tmp.data(), tmp.size() * sizeof(R));
}

template <typename R>
static int upload_complex(mb_handle *h, void **dst, const std::vector<cdouble> &src) {
    std::vector<R> tmp(2 * src.size());
    for (size_t i = 0; i < src.size(); ++i) {
        tmp[2 * i] = (R)src[i].real();
        tmp[2 * i + 1] = (R)src[i].imag();
    }
    return dev_upload(h, dst, tmp.data(), tmp.size() * sizeof(R));
}

template <typename R>
static int upload_set(mb_handle *h, DevTables &t) {
    int rc;
    if ((rc = upload<R>(h, &t.Bq, h->Bq))) return rc;
    if ((rc = upload<R>(h, &t.Sband, h->Sb))) return rc;
    {
        const int W = 2 * h->order - 1, WP = band_pad(h->order);
        std::vector<double> sp((size_t)h->nb * WP, 0.0);
        for (int j = 0; j < h->nb; ++j)
            for (int d = 0; d < W; ++d) sp[(size_t)j * WP + d] = h->Sb[(size_t)j * W + d];
        if ((rc = upload<R>(h, &t.SbandP, sp))) return rc;
    }
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
    if ((rc = upload<R>(h, &t.zf, h->zfun))) return rc;
    {
        std::vector<double> e(h->Ekb);
        e.insert(e.end(), h->Ecoup.begin(), h->Ecoup.end());
        if ((rc = upload<R>(h, &t.E, e))) return rc;
        if (h->uspp) {
            std::vector<double> q(h->Qkb);
            q.insert(q.end(), h->Qcoup.begin(), h->Qcoup.end());
            if ((rc = upload<R>(h, &t.Q, q))) return rc;
            std::vector<double> id(2 * (size_t)h->nkb, 0.0);
            std::fill(id.begin(), id.begin() + h->nkb, 1.0);
            if ((rc = upload<R>(h, &t.Eid, id))) return rc;
        }
    }
    const int nmax = std::max(h->n1, h->n2);
    std::vector<cdouble> tw(nmax / 2);
    for (int i = 0; i < nmax / 2; ++i) tw[i] = std::polar(1.0, 2.0 * 3.14159265358979323846 * i / nmax);
    if ((rc = upload_complex<R>(h, &t.tw, tw))) return rc;
    return MB_OK;
}

// The local potential's tables: built on the device from the atoms' analytic
// terms (vloc.cu).
int upload_potential(mb_handle *h) { return vloc_build(h); }

int upload_tables(mb_handle *h) {
    MB_CUDA(cudaSetDevice(h->device));
    if (!h->hs) {
        // set-up work at the highest priority: a new handle's uploads and
        // table kernels are scheduled ahead of the kernels of running solves
        int lo = 0, hi = 0;
        MB_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        MB_CUDA(cudaStreamCreateWithPriority(&h->hs, cudaStreamNonBlocking, hi));
    }
    int rc;
    if ((rc = upload_set<double>(h, h->t64))) return rc;
    if ((rc = upload_set<float>(h, h->t32))) return rc;
    if ((rc = upload_potential(h))) return rc;
    std::vector<int> goff((size_t)h->total_ldg, 0);
    for (size_t ik = 0; ik < h->kp.size(); ++ik)
        for (int g = 0; g < h->kp[ik].ng; ++g) goff[h->kofs[ik] + g] = h->kp[ik].goff[g];
    if ((rc = dev_upload(h, (void **)&h->d_goff, goff.data(), goff.size() * sizeof(int)))) return rc;
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
    if ((rc = dev_upload(h, (void **)&h->d_rows, rows.data(), rows.size() * sizeof(int)))) return rc;
    // compact planes: the disc's rows n1min .. n1max become rows 0 .. nocc-1
    // (row stride N2 + 1); the positions of those rows outside the disc
    {
        const int N2 = h->n2, LDP = N2 + 1;
        const size_t nk = h->kp.size();
        std::vector<int> cpos((size_t)h->total_ldg, 0), zpos;
        h->nocc.assign(nk, 1);
        h->zofs.assign(nk, 0);
        h->nzero.assign(nk, 0);
        for (size_t ik = 0; ik < nk; ++ik) {
            const KPoint &kp = h->kp[ik];
            int lo = 0, hi = 0;
            for (int g = 0; g < kp.ng; ++g) {
                lo = g ? std::min(lo, kp.n1[g]) : kp.n1[g];
                hi = g ? std::max(hi, kp.n1[g]) : kp.n1[g];
            }
            const int nocc = kp.ng ? hi - lo + 1 : 1;
            std::vector<char> used((size_t)nocc * N2, 0);
            for (int g = 0; g < kp.ng; ++g) {
                const int r = kp.n1[g] - lo, i2 = ((kp.n2[g] % N2) + N2) % N2;
                used[(size_t)r * N2 + i2] = 1;
                cpos[h->kofs[ik] + g] = r * LDP + i2;
            }
            h->nocc[ik] = nocc;
            h->zofs[ik] = (int)zpos.size();
            for (int r = 0; r < nocc; ++r)
                for (int i2 = 0; i2 < N2; ++i2)
                    if (!used[(size_t)r * N2 + i2]) zpos.push_back(r * LDP + i2);
            h->nzero[ik] = (int)zpos.size() - h->zofs[ik];
        }
        if (zpos.empty()) zpos.push_back(0);
        if ((rc = dev_upload(h, (void **)&h->d_cpos, cpos.data(), cpos.size() * sizeof(int)))) return rc;
        if ((rc = dev_upload(h, (void **)&h->d_zpos, zpos.data(), zpos.size() * sizeof(int)))) return rc;
    }
    if (h->nterm > 0) {
        std::vector<int> zi(h->pgroup);
        zi.insert(zi.end(), h->zstart.begin(), h->zstart.end());
        zi.insert(zi.end(), h->zlist.begin(), h->zlist.end());
        zi.insert(zi.end(), h->tproj.begin(), h->tproj.end());
        zi.insert(zi.end(), h->partner.begin(), h->partner.end());
        zi.insert(zi.end(), h->pstart.begin(), h->pstart.end());
        zi.insert(zi.end(), h->plist.begin(), h->plist.end());
        if ((rc = dev_upload(h, (void **)&h->d_zidx, zi.data(), zi.size() * sizeof(int)))) return rc;
    }
    upload_fft_twiddles();
    if (!h->d_tcerr) {
        // status word of the kernels' bounded device waits (mb_status)
        const int zero = 0;
        if ((rc = dev_upload(h, &h->d_tcerr, &zero, sizeof(int)))) return rc;
    }
    {
        const int zeros[2] = {0, 0};
        if ((rc = dev_upload(h, (void **)&h->d_queue, zeros, sizeof(zeros)))) return rc;
    }
    MB_CUDA(cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking));
    MB_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    MB_CUDA(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    MB_CUDA(cudaEventCreateWithFlags(&h->scratch_ev, cudaEventDisableTiming));
    if ((rc = upload_proj_tables(h))) return rc;
    MB_CUDA(cudaStreamSynchronize(h->hs));      // tables in place before any other stream uses them
    MB_CUDA(cudaGetLastError());
    return MB_OK;
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
    MB_CUDA(cudaStreamSynchronize(h->hs));
    h->pfac_ready = true;
    return MB_OK;
}

static void free_set(mb_handle *h, DevTables &t) {
    void **ps[] = {&t.Bq, &t.V, &t.Vn, &t.tw, &t.Sband, &t.SbandP, &t.Dband, &t.Lband, &t.Lrecip, &t.q2, &t.qproj, &t.zproj, &t.zf, &t.E, &t.Pfac, &t.Vt, &t.Q, &t.Eid};
    for (void **p : ps) dev_free(h, p);
}

// The caller has finished its work on the handle (mb_destroy's contract):
// everything is freed stream-ordered on the handle's stream.
void free_tables(mb_handle *h) {
    cudaSetDevice(h->device);
    if (!h->hs) cudaStreamCreateWithFlags(&h->hs, cudaStreamNonBlocking);
    if (h->aux) cudaStreamSynchronize(h->aux);
    if (h->scratch_ev) cudaEventSynchronize(h->scratch_ev);
    free_set(h, h->t64);
    free_set(h, h->t32);
    dev_free(h, (void **)&h->d_goff);
    dev_free(h, (void **)&h->d_rows);
    dev_free(h, (void **)&h->d_cpos);
    dev_free(h, (void **)&h->d_zpos);
    dev_free(h, &h->d_projB);
    dev_free(h, (void **)&h->d_zidx);
    dev_free(h, &h->d_tcerr);
    dev_free(h, (void **)&h->d_queue);
    dev_free(h, (void **)&h->d_vloc);
    dev_free(h, &h->scratch.ptr);
    h->scratch = Scratch();
    if (h->aux) cudaStreamDestroy(h->aux);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->scratch_ev) cudaEventDestroy(h->scratch_ev);
    h->aux = nullptr;
    h->ev_fork = h->ev_join = h->scratch_ev = nullptr;
    if (h->hs) {
        cudaStreamSynchronize(h->hs);
        cudaStreamDestroy(h->hs);
    }
    h->hs = nullptr;
}

// Grows the apply scratch, stream-ordered on the caller's stream s: the old
// buffer is released once the last apply that used it has finished (its
// event), the new one is in place when this returns (a host wait on s only).
int ensure_scratch(mb_handle *h, size_t bytes, cudaStream_t s) {
    if (bytes <= h->scratch.bytes) return MB_OK;
    if (h->scratch.ptr && h->scratch_ev) MB_CUDA(cudaEventSynchronize(h->scratch_ev));
    cudaMemPool_t pool = mb_pool(h->device);
    if (!pool) return MB_ECUDA;
    if (h->scratch.ptr) MB_CUDA(cudaFreeAsync(h->scratch.ptr, s));
    h->scratch = Scratch();
    MB_CUDA(cudaMallocFromPoolAsync(&h->scratch.ptr, bytes, pool, s));
    MB_CUDA(cudaStreamSynchronize(s));
    h->scratch.bytes = bytes;
    return MB_OK;
}

// Launch plan of the plane kernel for one batched apply.
struct PlanePlan {
    bool reg = false;      // register-FFT kernel (else radix-2 shared-memory kernel)
    bool p32 = false;      // FP32 compact-plane kernel
    bool persist = false;  // its persistent, work-queue launch
    Plane32Shape sh;       // its instance
    int bt = 1;            // bands per CTA
    int np = 1;            // planes in flight
    int chunk = 1, nchunks = 1;
    size_t smem = 0;
};

// Run count of the wave model: a CTA's time ~ its run length + about one
// interval of run overhead (boundary rows); the launch takes
// ceil(items / slots) rounds of the longest run.
static int wave_model_chunks(const mb_handle *h, int pairs, int slots, int nmax_chunks, int waves) {
    if (waves > 0) {
        // explicit target: about `waves` CTAs per resident slot
        const int target = std::max(1, (waves * slots + pairs - 1) / pairs);
        return std::min(nmax_chunks, target);
    }
    double best = 1e300;
    int nch = 1;
    for (int n = 1; n <= nmax_chunks; ++n) {
        const long long items = (long long)pairs * n;
        const long long rounds = (items + slots - 1) / slots;
        const double cost = (double)rounds * ((h->nint + n - 1) / n + 1.0);
        if (cost < best - 1e-9) { best = cost; nch = n; }
    }
    return nch;
}

// Shared memory of a compact-plane instance at its CTAs per SM: planes,
// output-row ring (and X window slots), and the B values of a run of
// intervals; runs as short as the plan allows (K intervals) must fit.
static size_t p32_budget(const mb_handle *h, const Plane32Shape &sh) {
    return std::min((size_t)h->smem_optin, (size_t)228 * 1024 / sh.ctas_per_sm - 1024);
}
static size_t p32_smem(const mb_handle *h, const Plane32Shape &sh, int maxldg, int nch) {
    const int K = h->order, P = h->nquad;
    return sh.smem_fixed + (size_t)sh.bt * K * maxldg * sizeof(float2) +
           (size_t)((h->nint + nch - 1) / nch) * K * P * sizeof(float);
}
static bool p32_fits(const mb_handle *h, const Plane32Shape &sh, int maxldg) {
    const int nmax_chunks = std::max(1, std::min(kMaxChunks, h->nint / h->order));
    return p32_smem(h, sh, maxldg, nmax_chunks) <= p32_budget(h, sh);
}

static PlanePlan plan_plane(const mb_handle *h, int nsel, const int *iks, int nbands, size_t c2, bool reg_ok) {
    PlanePlan p;
    const int K = h->order, P = h->nquad;
    const size_t NN = (size_t)h->n1 * h->n2;
    int maxldg = 0, nocc_max = 0;
    for (int i = 0; i < nsel; ++i) {
        maxldg = std::max(maxldg, h->kp[iks[i]].ldg);
        nocc_max = std::max(nocc_max, h->nocc[iks[i]]);
    }
    int ctas_per_sm = 1;
    // defaults, or the shape mb_autotune measured fastest for this batch
    const bool small = h->n1 <= 32 && h->n2 <= 32;
    int bt_max = small ? 2 : 1, waves = 0, p32_id = -1, persist = 0;
    auto it = h->tuned.find(std::make_tuple(nsel, nbands, c2 == 16 ? 1 : 0));
    if (it != h->tuned.end()) {
        bt_max = it->second.bt;
        waves = it->second.waves;
        p32_id = it->second.p32;
        persist = it->second.persist;
    }
    const int nmax_chunks = std::max(1, std::min(kMaxChunks, h->nint / K));   // runs of >= K intervals
    if (c2 == 8 && p32_id != -2) {
        // FP32 compact-plane kernel: planes + output-row ring (+ X window
        // slots) + the run's B values.  The tuned instance if there is one,
        // else the first whose shared memory fits.
        Plane32Shape shapes[kMaxPlane32Shapes];
        const int ns = plane32_shapes(h->n1, h->n2, K, P, nocc_max, maxldg, shapes, kMaxPlane32Shapes);
        for (int pass = 0; pass < 2; ++pass)
            for (int v = 0; v < ns; ++v) {
                const Plane32Shape &sh = shapes[v];
                if (pass == 0 && sh.id != p32_id) continue;
                const int pairs = nsel * ((nbands + sh.bt - 1) / sh.bt);
                const int slots = h->num_sms * sh.ctas_per_sm;
                const size_t budget = p32_budget(h, sh);
                int nch = wave_model_chunks(h, pairs, slots, nmax_chunks, waves);
                auto smem_of = [&](int n) { return p32_smem(h, sh, maxldg, n); };
                while (nch < nmax_chunks && smem_of(nch) > budget) ++nch;
                if (smem_of(nch) > budget) continue;
                p.p32 = true;
                p.persist = persist != 0;
                p.sh = sh;
                p.bt = sh.bt;
                p.np = sh.bt * P;
                p.nchunks = nch;
                p.chunk = (h->nint + nch - 1) / nch;
                p.smem = smem_of(nch);
                return p;
            }
    }
    if (reg_ok) {
        const size_t plane_bytes = (size_t)h->n1 * (h->n2 + 1) * c2;
        // matches the kernel's launch bounds
        ctas_per_sm = c2 == 8 ? ((NN <= 512 || (h->n1 == 32 && h->n2 == 32)) ? 3 : small ? 2 : 1) : 1;
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
    const int slots = h->num_sms * ctas_per_sm;
    p.nchunks = wave_model_chunks(h, pairs, slots, nmax_chunks, waves);
    p.chunk = (h->nint + p.nchunks - 1) / p.nchunks;   // longest run
    return p;
}

// Largest j-segment count of the projector overlaps and of the epilogue.
static int nl_max_seg(const mb_handle *h) { return std::max(1, std::min(8, h->nb / 8)); }

// Scratch regions of one k-point: boundary partial rows; projector overlaps
// W (Zx[b][f][G] on CUDA cores, W[(b, j)][p] on tensor cores) and
// coefficients C (c[b][p], or C[(b, j)][p] on tensor cores).
struct KScratch {
    size_t part, w, c;
    size_t total() const { return al(part) + al(w) + al(c); }
    static size_t al(size_t x) { return (x + 255) / 256 * 256; }
};

static KScratch per_k_layout(const mb_handle *h, int ldg, int nbands, int nchunks, size_t c2, bool tensor) {
    KScratch k;
    k.part = (size_t)nbands * std::max(0, nchunks - 1) * 2 * (h->order - 1) * ldg * c2;
    if (tensor) {
        k.w = k.c = (size_t)nbands * h->nb * std::max(1, h->nterm) * c2;
    } else {
        k.w = (size_t)nbands * std::max(1, h->nzf) * ldg * c2;
        k.c = (size_t)nbands * std::max(1, h->nterm) * c2;
    }
    return k;
}

static size_t per_k_scratch(const mb_handle *h, int ldg, int nbands, int nchunks, size_t c2, bool tensor) {
    return per_k_layout(h, ldg, nbands, nchunks, c2, tensor).total();
}

// Scratch of a batched apply of k-points 0 .. nk-1 in order (the groups of
// kMaxK that apply_H_batch forms, each planned as it will be launched).
size_t apply_scratch_bytes(const mb_handle *h, int nk, int nbands, int prec) {
    const size_t c2 = prec == MB_FP64 ? 16 : 8;
    const bool reg = prec == MB_FP64 ? plane_reg_supported<double>(h->n1, h->n2, h->order)
                                     : plane_reg_supported<float>(h->n1, h->n2, h->order);
    nk = std::min(nk, (int)h->kp.size());
    size_t need = 0;
    for (int i0 = 0; i0 < nk; i0 += kMaxK) {
        const int nsel = std::min(kMaxK, nk - i0);
        int maxldg = 0;
        std::vector<int> ik(nsel);
        for (int i = i0; i < i0 + nsel; ++i) {
            maxldg = std::max(maxldg, h->kp[i].ldg);
            ik[i - i0] = i;
        }
        const PlanePlan p = plan_plane(h, nsel, ik.data(), nbands, c2, reg);
        need = std::max(need, (size_t)nsel * per_k_scratch(h, maxldg, nbands, p.nchunks, c2, prec == MB_BF16));
    }
    return need;
}

cudaError_t proj_tc_launch(mb_handle *h, int mode, int nsel, const int *iks, const KDesc *desc, int nbands,
                           cudaStream_t s);

template <typename R>
static int apply_H_launch(mb_handle *h, int nsel, const int *iks, const void *const *X, void *const *Y,
                          int nbands, cudaStream_t s, const DevTables &t, char *base, bool tensor = false);

// Scratch bytes one batched apply needs (boundary rows, projector overlaps W
// and coefficients C for every k-point of the group).
template <typename R>
static size_t apply_H_need(const mb_handle *h, int nsel, const int *iks, int nbands, bool tensor) {
    const size_t c2 = sizeof(typename V2<R>::T);
    int maxldg = 0;
    for (int i = 0; i < nsel; ++i) maxldg = std::max(maxldg, h->kp[iks[i]].ldg);
    const PlanePlan plan = plan_plane(h, nsel, iks, nbands, c2, plane_reg_supported<R>(h->n1, h->n2, h->order));
    return (size_t)nsel * per_k_scratch(h, maxldg, nbands, plan.nchunks, c2, tensor);
}

template <typename R>
static int apply_H_group(mb_handle *h, int nsel, const int *iks, const void *const *X, void *const *Y,
                         int nbands, cudaStream_t s, const DevTables &t, bool tensor = false) {
    int rc = ensure_scratch(h, apply_H_need<R>(h, nsel, iks, nbands, tensor), s);
    if (rc) return rc;
    rc = apply_H_launch<R>(h, nsel, iks, X, Y, nbands, s, t, reinterpret_cast<char *>(h->scratch.ptr), tensor);
    if (rc) return rc;
    // the scratch is in use until this point of s (not recorded during a
    // capture: scratch never grows then)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    MB_CUDA(cudaStreamIsCapturing(s, &cs));
    if (cs == cudaStreamCaptureStatusNone) MB_CUDA(cudaEventRecord(h->scratch_ev, s));
    return MB_OK;
}

// Scratch need of a single-k-point apply, and the apply itself on a scratch
// region supplied by the caller of this function (no allocation here).
size_t apply_H_scratch_need(const mb_handle *h, int ik, int nbands, int prec) {
    return prec == MB_FP64 ? apply_H_need<double>(h, 1, &ik, nbands, false)
                           : apply_H_need<float>(h, 1, &ik, nbands, prec == MB_BF16);
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
    const PlanePlan plan = plan_plane(h, nsel, iks, nbands, c2, plane_reg_supported<R>(h->n1, h->n2, h->order));
    const int chunk = plan.chunk, nchunks = plan.nchunks;
    (void)chunk;
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
        d.nocc = h->nocc[iks[i]];
        d.zofs = h->zofs[iks[i]];
        d.nz = h->nzero[iks[i]];
        // every k-point's regions are laid out for the batch's widest row (maxldg)
        const KScratch ks = per_k_layout(h, maxldg, nbands, nchunks, c2, tensor);
        d.part = base + off;
        off += al(ks.part);
        d.W = base + off;
        off += al(ks.w);
        d.C = base + off;
        off += al(ks.c);
    }
    // threads per (band, G) column for the j-contractions: aim at ~2 resident
    // waves of 128-thread CTAs, with runs of at least 8 rows
    long long cols = 0;
    for (int i = 0; i < nsel; ++i) cols += (long long)nbands * h->kp[iks[i]].ldg;
    const int want_threads = h->num_sms * 2048;
    const int nseg = (int)std::max<long long>(1, std::min<long long>(nl_max_seg(h), (want_threads + cols - 1) / cols));
    // index tables (layout of d_zidx: pgroup | zstart | zlist | tproj | partner | pstart | plist)
    const int *d_pgroup = h->d_zidx;
    const int *d_zstart = h->d_zidx ? d_pgroup + h->nterm : nullptr;
    const int *d_zlist = h->d_zidx ? d_zstart + h->nzf + 1 : nullptr;
    const int *d_tproj = h->d_zidx ? d_zlist + h->nterm : nullptr;
    const int *d_partner = h->d_zidx ? d_tproj + h->nterm : nullptr;
    const int *d_pstart = h->d_zidx ? d_partner + h->nkb : nullptr;
    const int *d_plist = h->d_zidx ? d_pstart + h->nkb + 1 : nullptr;
    bool forked = false;
    // projector overlaps first (they read X only)
    if (h->nterm > 0 && tensor) {
        cudaError_t e = cudaSuccess;
        MB_LAUNCH(h, s, KN_PROJ, e = proj_tc_launch(h, 0, nsel, iks, desc, nbands, s));
        MB_CUDA(e);
        CoefArgs<R> ca;
        ca.zproj = reinterpret_cast<const R *>(t.zproj);
        ca.E = reinterpret_cast<const R *>(t.E);
        ca.partner = d_partner;
        ca.pstart = d_pstart;
        ca.plist = d_plist;
        ca.nb = h->nb;
        ca.nbands = nbands;
        ca.nterm = h->nterm;
        ca.nkb = h->nkb;
        std::copy(desc, desc + nsel, ca.d);
        MB_LAUNCH(h, s, KN_COEF, coef_kernel<R><<<dim3((nbands * h->nkb + 127) / 128, nsel), 128, 0, s>>>(ca));
    } else if (h->nterm > 0) {
        // the overlaps read X only: they run on the aux stream beside the
        // plane kernel and are joined before the epilogue
        MB_CUDA(cudaEventRecord(h->ev_fork, s));
        MB_CUDA(cudaStreamWaitEvent(h->aux, h->ev_fork, 0));
        cudaStream_t sa = h->aux;
        NlArgs<R> na;
        na.zf = reinterpret_cast<const R *>(t.zf);
        na.E = reinterpret_cast<const R *>(t.E);
        na.pgroup = d_pgroup;
        na.partner = d_partner;
        na.pstart = d_pstart;
        na.plist = d_plist;
        na.Q = reinterpret_cast<const R2 *>(t.qproj);
        na.nb = h->nb;
        na.nbands = nbands;
        na.nterm = h->nterm;
        na.nkb = h->nkb;
        na.nz = h->nzf;
        na.nseg = nseg;
        std::copy(desc, desc + nsel, na.d);
        const int zseg = std::max(1, std::min(8, h->nb / 8));
        na.nseg = zseg;
        const dim3 gz((maxldg + 63) / 64, nbands, nsel), bz(64, zseg);
#define MB_ZX(NZ)                                                                                  \
    do {                                                                                           \
        const size_t zsm = (size_t)zseg * NZ * 64 * sizeof(R2) + (size_t)h->nzf * h->nb * sizeof(R); \
        MB_CUDA(smem_limit_once((const void *)nl_zx_kernel<R, NZ>, h->device, h->smem_optin));   \
        MB_LAUNCH(h, sa, KN_PROJ, (nl_zx_kernel<R, NZ><<<gz, bz, zsm, sa>>>(na)));                 \
    } while (0)
        if (h->nzf <= 2) MB_ZX(2);
        else if (h->nzf <= 4) MB_ZX(4);
        else if (h->nzf <= 8) MB_ZX(8);
        else if (h->nzf <= 12) MB_ZX(12);
        else MB_ZX(16);
#undef MB_ZX
        MB_LAUNCH(h, sa, KN_COEF, nl_coef_kernel<R><<<dim3(nbands, nsel, (h->nkb + 7) / 8), 256, 0, sa>>>(na));
        const size_t bsm = (size_t)h->nterm * (sizeof(R2) + sizeof(int));
        MB_CUDA(smem_limit_once((const void *)nl_back_kernel<R>, h->device, h->smem_optin));
        MB_LAUNCH(h, sa, KN_COEF, nl_back_kernel<R><<<dim3((maxldg + 127) / 128, h->nzf, nbands * nsel), 128, bsm, sa>>>(
                                     na, d_zstart, d_zlist, d_tproj));
        MB_CUDA(cudaEventRecord(h->ev_join, sa));
        forked = true;
    }
    // local potential through the planes
    PlaneArgs<R> pa;
    pa.Bq = reinterpret_cast<const R *>(t.Bq);
    pa.V = reinterpret_cast<const R *>(t.V);
    pa.Vn = reinterpret_cast<const R *>(t.Vn);
    pa.rows = h->d_rows;
    pa.tw = reinterpret_cast<const R2 *>(t.tw);
    pa.goff = h->d_goff;
    pa.Vt = reinterpret_cast<const R *>(t.Vt);
    pa.cpos = h->d_cpos;
    pa.zpos = h->d_zpos;
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
    pa.queue = plan.persist ? h->d_queue : nullptr;
    std::copy(desc, desc + nsel, pa.d);
    if (plan.p32) {
        if constexpr (sizeof(R) == 4) {
            const unsigned items = (unsigned)(nsel * ((nbands + plan.bt - 1) / plan.bt) * nchunks);
            const unsigned grid =
                plan.persist ? std::min(items, (unsigned)(h->num_sms * plan.sh.ctas_per_sm)) : items;
            cudaError_t e = cudaSuccess;
            MB_LAUNCH(h, s, KN_PLANE, e = plane32_launch(pa, plan.sh, grid, plan.smem, s));
            MB_CUDA(e);
        }
    } else if (plan.reg) {
        const unsigned grid = (unsigned)(nsel * ((nbands + plan.bt - 1) / plan.bt) * nchunks);
        cudaError_t e = cudaSuccess;
        MB_LAUNCH(h, s, KN_PLANE, e = plane_reg_launch<R>(pa, grid, plan.smem, s));
        MB_CUDA(e);
    } else {
        MB_CUDA(smem_limit_once((const void *)plane_kernel<R>, h->device, h->smem_optin));
        MB_LAUNCH(h, s, KN_PLANE, plane_kernel<R><<<nsel * nbands * nchunks, 256, plan.smem, s>>>(pa));
    }
    if (forked) MB_CUDA(cudaStreamWaitEvent(s, h->ev_join, 0));
    EpiArgs<R> ea;
    ea.Sband = reinterpret_cast<const R *>(t.Sband);
    ea.Dband = reinterpret_cast<const R *>(t.Dband);
    ea.q2 = reinterpret_cast<const R *>(t.q2);
    ea.zf = reinterpret_cast<const R *>(t.zf);

    ea.order = h->order;
    ea.nb = h->nb;
    ea.nbands = nbands;
    ea.nchunks = nchunks;
    ea.nint = h->nint;
    ea.nz = h->nzf;
    // rows per epilogue thread: at most 8 (FP32) / 4 (FP64), all loaded at once
    constexpr int ERM = sizeof(R) == 4 ? 8 : 4;
    const int ejseg = (h->nb + ERM - 1) / ERM;
    ea.njseg = ejseg;
    // where each row's local part lives: run boundary bc (between runs bc and
    // bc+1) starts at interval t1 and owns rows [t1 - 1, t1 + K - 3]
    if (h->nb > kMaxEpiRows) return MB_EUNSUPPORTED;
    for (int j = 0; j < h->nb; ++j) {
        int sv = -1;
        for (int bc = 0; bc + 1 < nchunks && sv < 0; ++bc) {
            const int t1 = chunk_begin(bc + 1, h->nint, nchunks);
            if (j >= t1 - 1 && j <= t1 + h->order - 3) sv = (bc * 2 + 0) * (h->order - 1) + (j - (t1 - 1));
        }
        ea.src[j] = (short)sv;
    }
    std::copy(desc, desc + nsel, ea.d);
    // kinetic term, boundary sums and the KB term of the first 16 z factors;
    // further passes add the KB term of the rest
    const int nzf = (h->nterm > 0 && !tensor) ? h->nzf : 0;
    const dim3 ge((maxldg + 63) / 64, nbands * ejseg, nsel);
    for (int f0 = 0, pass = 0; pass == 0 || f0 < nzf; f0 += 16, ++pass) {
        ea.f0 = f0;
        ea.f1 = std::min(nzf, f0 + 16);
        ea.base = pass == 0;
        const int HWn = h->order <= 6 ? 5 : 7;
        const int nfp = ea.f1 - ea.f0;
        const int nzb = nfp <= 4 ? 4 : nfp <= 8 ? 8 : nfp <= 12 ? 12 : 16;
        const size_t esm = ((size_t)2 * ERM * ((2 * HWn + 1 + 3) / 4 * 4) + (size_t)ERM * nzb) * sizeof(R);
#define MB_EPI(NZ, HWV)                                                                                        \
    do {                                                                                                       \
        MB_CUDA(smem_limit_once((const void *)epilogue_kernel<R, NZ, HWV, ERM>, h->device, h->smem_optin));  \
        MB_LAUNCH(h, s, KN_EPILOGUE, (epilogue_kernel<R, NZ, HWV, ERM><<<ge, 64, esm, s>>>(ea)));            \
    } while (0)
        if (HWn == 5) {
            if (nzb == 4) MB_EPI(4, 5);
            else if (nzb == 8) MB_EPI(8, 5);
            else if (nzb == 12) MB_EPI(12, 5);
            else MB_EPI(16, 5);
        } else {
            if (nzb == 4) MB_EPI(4, 7);
            else if (nzb == 8) MB_EPI(8, 7);
            else if (nzb == 12) MB_EPI(12, 7);
            else MB_EPI(16, 7);
        }
#undef MB_EPI
    }
    if (h->nterm > 0 && tensor) {
        cudaError_t e = cudaSuccess;
        MB_LAUNCH(h, s, KN_BACKPROJ, e = proj_tc_launch(h, 1, nsel, iks, desc, nbands, s));
        MB_CUDA(e);
    }
    MB_CUDA(cudaGetLastError());
    return MB_OK;
}

// ---------------------------------------------------------------------------
// Ultrasoft overlap term (§II.B.2): Y += sum_pq q_pq beta_p (beta_q^H X), by
// the KB kernels with the strengths q in place of E (same sparsity: diagonal
// and the 1s-2s partner), the back-projection added to Y by the epilogue's
// KB-only pass.  Scratch: the projector regions of the apply's layout.
size_t uspp_scratch_group(const mb_handle *h, int nsel, const int *iks, int nbands, int prec) {
    const size_t c2 = prec == MB_FP64 ? 16 : 8;
    int maxldg = 0;
    for (int i = 0; i < nsel; ++i) maxldg = std::max(maxldg, h->kp[iks[i]].ldg);
    return (size_t)nsel * per_k_scratch(h, maxldg, nbands, 1, c2, false);
}

size_t uspp_scratch_bytes(const mb_handle *h, int nk, int nbands, int prec) {
    nk = std::min(nk, (int)h->kp.size());
    size_t need = 0;
    for (int i0 = 0; i0 < nk; i0 += kMaxK) {
        std::vector<int> ik;
        for (int i = i0; i < std::min(nk, i0 + kMaxK); ++i) ik.push_back(i);
        need = std::max(need, uspp_scratch_group(h, (int)ik.size(), ik.data(), nbands, prec));
    }
    return need;
}

// The KB contraction of X with strengths Es (device, the layout of E) into
// the scratch's c[b][p] (coef_only) or, further, back-projected and added
// to Y.
template <typename R>
static int projector_pass(mb_handle *h, int nsel, const int *iks, const void *const *X, void *const *Y, int nbands,
                          cudaStream_t s, const DevTables &t, const void *Es, bool coef_only, KDesc *desc_out) {
    typedef typename V2<R>::T R2;
    if (h->nterm <= 0) return MB_OK;
    const size_t c2 = sizeof(R2);
    int maxldg = 0;
    for (int i = 0; i < nsel; ++i) maxldg = std::max(maxldg, h->kp[iks[i]].ldg);
    if (h->scratch.bytes < uspp_scratch_group(h, nsel, iks, nbands, sizeof(R) == 8 ? MB_FP64 : MB_FP32))
        return MB_EUNSUPPORTED;
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    char *base = reinterpret_cast<char *>(h->scratch.ptr);
    KDesc desc[kMaxK];
    size_t off = 0;
    for (int i = 0; i < nsel; ++i) {
        const KPoint &kp = h->kp[iks[i]];
        KDesc &d = desc[i];
        d = KDesc();
        d.X = X[i];
        d.Y = Y ? Y[i] : nullptr;
        d.ng = kp.ng;
        d.ldg = kp.ldg;
        d.kofs = h->kofs[iks[i]];
        d.qofs = h->qofs[iks[i]];
        const KScratch ks = per_k_layout(h, maxldg, nbands, 1, c2, false);
        d.part = base + off;
        off += al(ks.part);
        d.W = base + off;
        off += al(ks.w);
        d.C = base + off;
        off += al(ks.c);
    }
    if (desc_out) std::copy(desc, desc + nsel, desc_out);
    const int *d_pgroup = h->d_zidx;
    const int *d_zstart = d_pgroup + h->nterm;
    const int *d_zlist = d_zstart + h->nzf + 1;
    const int *d_tproj = d_zlist + h->nterm;
    const int *d_partner = d_tproj + h->nterm;
    const int *d_pstart = d_partner + h->nkb;
    const int *d_plist = d_pstart + h->nkb + 1;
    NlArgs<R> na;
    na.zf = reinterpret_cast<const R *>(t.zf);
    na.E = reinterpret_cast<const R *>(Es);
    na.pgroup = d_pgroup;
    na.partner = d_partner;
    na.pstart = d_pstart;
    na.plist = d_plist;
    na.Q = reinterpret_cast<const R2 *>(t.qproj);
    na.nb = h->nb;
    na.nbands = nbands;
    na.nterm = h->nterm;
    na.nkb = h->nkb;
    na.nz = h->nzf;
    std::copy(desc, desc + nsel, na.d);
    const int zseg = std::max(1, std::min(8, h->nb / 8));
    na.nseg = zseg;
    const dim3 gz((maxldg + 63) / 64, nbands, nsel), bz(64, zseg);
#define MB_ZX(NZ)                                                                                  \
    do {                                                                                           \
        const size_t zsm = (size_t)zseg * NZ * 64 * sizeof(R2) + (size_t)h->nzf * h->nb * sizeof(R); \
        MB_CUDA(smem_limit_once((const void *)nl_zx_kernel<R, NZ>, h->device, h->smem_optin));   \
        MB_LAUNCH(h, s, KN_PROJ, (nl_zx_kernel<R, NZ><<<gz, bz, zsm, s>>>(na)));                   \
    } while (0)
    if (h->nzf <= 2) MB_ZX(2);
    else if (h->nzf <= 4) MB_ZX(4);
    else if (h->nzf <= 8) MB_ZX(8);
    else if (h->nzf <= 12) MB_ZX(12);
    else MB_ZX(16);
#undef MB_ZX
    MB_LAUNCH(h, s, KN_COEF, nl_coef_kernel<R><<<dim3(nbands, nsel, (h->nkb + 7) / 8), 256, 0, s>>>(na));
    if (coef_only) {
        MB_CUDA(cudaGetLastError());
        return MB_OK;
    }
    const size_t bsm = (size_t)h->nterm * (sizeof(R2) + sizeof(int));
    MB_CUDA(smem_limit_once((const void *)nl_back_kernel<R>, h->device, h->smem_optin));
    MB_LAUNCH(h, s, KN_COEF, nl_back_kernel<R><<<dim3((maxldg + 127) / 128, h->nzf, nbands * nsel), 128, bsm, s>>>(
                                 na, d_zstart, d_zlist, d_tproj));
    // Y += sum_f z_f(j) R_f(G): the epilogue's KB-only passes
    EpiArgs<R> ea;
    ea.Sband = reinterpret_cast<const R *>(t.Sband);
    ea.Dband = reinterpret_cast<const R *>(t.Dband);
    ea.q2 = reinterpret_cast<const R *>(t.q2);
    ea.zf = reinterpret_cast<const R *>(t.zf);
    ea.order = h->order;
    ea.nb = h->nb;
    ea.nbands = nbands;
    ea.nchunks = 1;
    ea.nint = h->nint;
    ea.nz = h->nzf;
    constexpr int ERM = sizeof(R) == 4 ? 8 : 4;
    const int ejseg = (h->nb + ERM - 1) / ERM;
    ea.njseg = ejseg;
    if (h->nb > kMaxEpiRows) return MB_EUNSUPPORTED;
    for (int j = 0; j < h->nb; ++j) ea.src[j] = -1;
    std::copy(desc, desc + nsel, ea.d);
    const dim3 ge((maxldg + 63) / 64, nbands * ejseg, nsel);
    for (int f0 = 0; f0 < h->nzf; f0 += 16) {
        ea.f0 = f0;
        ea.f1 = std::min(h->nzf, f0 + 16);
        ea.base = 0;
        const int nfp = ea.f1 - ea.f0;
        const int nzb = nfp <= 4 ? 4 : nfp <= 8 ? 8 : nfp <= 12 ? 12 : 16;
        constexpr int HWn = 5;   // unused by the KB-only pass (no band rows)
        const size_t esm = ((size_t)2 * ERM * ((2 * HWn + 1 + 3) / 4 * 4) + (size_t)ERM * nzb) * sizeof(R);
#define MB_EPI(NZ)                                                                                            \
    do {                                                                                                      \
        MB_CUDA(smem_limit_once((const void *)epilogue_kernel<R, NZ, HWn, ERM>, h->device, h->smem_optin));  \
        MB_LAUNCH(h, s, KN_EPILOGUE, (epilogue_kernel<R, NZ, HWn, ERM><<<ge, 64, esm, s>>>(ea)));            \
    } while (0)
        if (nzb == 4) MB_EPI(4);
        else if (nzb == 8) MB_EPI(8);
        else if (nzb == 12) MB_EPI(12);
        else MB_EPI(16);
#undef MB_EPI
    }
    MB_CUDA(cudaGetLastError());
    return MB_OK;
}

int uspp_S_add(mb_handle *h, int nsel, const int *iks, const void *const *X, void *const *Y, int nbands, int prec,
               cudaStream_t s) {
    if (!h->uspp) return MB_OK;
    for (int i0 = 0; i0 < nsel; i0 += kMaxK) {
        const int n = std::min(kMaxK, nsel - i0);
        const int rc = prec == MB_FP64
                           ? projector_pass<double>(h, n, iks + i0, X + i0, Y + i0, nbands, s, h->t64, h->t64.Q,
                                                    false, nullptr)
                           : projector_pass<float>(h, n, iks + i0, X + i0, Y + i0, nbands, s, h->t32, h->t32.Q,
                                                   false, nullptr);
        if (rc) return rc;
    }
    return MB_OK;
}

int uspp_overlaps(mb_handle *h, const void *evecs, int nbands, double *F, cudaStream_t s) {
    if (!h->uspp || h->nkb == 0) return MB_EINVAL;
    const int nk = (int)h->kp.size();
    std::vector<int> iks(nk);
    std::vector<const void *> xs(nk);
    size_t off = 0;
    for (int k = 0; k < nk; ++k) {
        iks[k] = k;
        xs[k] = reinterpret_cast<const double2 *>(evecs) + off;
        off += (size_t)nbands * h->nb * h->kp[k].ldg;
    }
    int rc = ensure_scratch(h, uspp_scratch_bytes(h, nk, nbands, MB_FP64), s);
    if (rc) return rc;
    for (int k0 = 0; k0 < nk; k0 += kMaxK) {
        const int n = std::min(kMaxK, nk - k0);
        KDesc desc[kMaxK];
        if ((rc = projector_pass<double>(h, n, iks.data() + k0, xs.data() + k0, nullptr, nbands, s, h->t64,
                                         h->t64.Eid, true, desc)))
            return rc;
        for (int i = 0; i < n; ++i)
            MB_CUDA(cudaMemcpyAsync(F + 2 * (size_t)(k0 + i) * nbands * h->nkb, desc[i].C,
                                    sizeof(double2) * (size_t)nbands * h->nkb, cudaMemcpyDeviceToHost, s));
        MB_CUDA(cudaStreamSynchronize(s));   // the next group reuses the scratch
    }
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

static int apply_sinv_per_k(mb_handle *h, int ik, const void *X, void *Y, int nbands, int prec, cudaStream_t s);

int apply_banded_batch(mb_handle *h, int which, int nsel, const int *iks, const void *const *X, void *const *Y,
                       int nbands, int prec, cudaStream_t s) {
    if (nsel <= 0 || !iks || !X || !Y || nbands <= 0) return MB_EINVAL;
    if (which != BAND_S && which != BAND_SINV) return MB_EINVAL;
    if (prec != MB_FP64 && prec != MB_FP32 && prec != MB_BF16) return MB_EINVAL;
    for (int i = 0; i < nsel; ++i) {
        if (iks[i] < 0 || iks[i] >= (int)h->kp.size() || !X[i] || !Y[i]) return MB_EINVAL;
        if (X[i] == Y[i]) return MB_EINVAL;
    }
    MB_CUDA(cudaSetDevice(h->device));
    if (h->uspp && which == BAND_SINV) return MB_EUNSUPPORTED;   // the inverse of the augmented S is not banded
    int rc = MB_OK;
    if (banded_block_supported(h, prec, which == BAND_SINV)) {
        rc = banded_block_apply(h, which == BAND_SINV, nsel, iks, X, Y, nbands, prec, s);
    } else {
        // S has the tile kernel at every order 3-8; this is S^-1 at orders other than 6
        for (int i = 0; i < nsel && rc == MB_OK; ++i) rc = apply_sinv_per_k(h, iks[i], X[i], Y[i], nbands, prec, s);
    }
    if (rc == MB_OK && h->uspp) {
        // the ultrasoft term on top of S_0 X (grows the scratch: not during stream capture)
        size_t need = 0;
        for (int i0 = 0; i0 < nsel; i0 += kMaxK) {
            std::vector<int> ik(iks + i0, iks + std::min(nsel, i0 + kMaxK));
            need = std::max(need, uspp_scratch_group(h, (int)ik.size(), ik.data(), nbands, prec));
        }
        if ((rc = ensure_scratch(h, need, s))) return rc;
        rc = uspp_S_add(h, nsel, iks, X, Y, nbands, prec, s);
    }
    return rc;
}

// S^-1 X for one k-point with the per-column solve kernel (orders whose
// S^-1 has no tile kernel)
static int apply_sinv_per_k(mb_handle *h, int ik, const void *X, void *Y, int nbands, int prec, cudaStream_t s) {
    if (ik < 0 || ik >= (int)h->kp.size() || !X || !Y || X == Y || nbands <= 0) return MB_EINVAL;
    if (prec != MB_FP64 && prec != MB_FP32 && prec != MB_BF16) return MB_EINVAL;
    MB_CUDA(cudaSetDevice(h->device));
    const KPoint &kp = h->kp[ik];
    const dim3 gL((kp.ldg + 63) / 64, nbands);
    if (prec == MB_FP64) {
        MB_LAUNCH(h, s, KN_BANDED, banded_solve_kernel<double><<<gL, 64, 0, s>>>(
                                       (const double *)h->t64.Lband, h->order, h->nb, kp.ng, kp.ldg, nbands,
                                       reinterpret_cast<const double2 *>(X), reinterpret_cast<double2 *>(Y)));
    } else {
        MB_LAUNCH(h, s, KN_BANDED, banded_solve_kernel<float><<<gL, 64, 0, s>>>(
                                       (const float *)h->t32.Lband, h->order, h->nb, kp.ng, kp.ldg, nbands,
                                       reinterpret_cast<const float2 *>(X), reinterpret_cast<float2 *>(Y)));
    }
    MB_CUDA(cudaGetLastError());
    return MB_OK;
}

}  // namespace mb

// ---------------------------------------------------------------------------
// mb_autotune: time the candidate plane-kernel launch shapes for a batch of
// `nbands` bands at every k-point of the handle and keep the fastest.
namespace mb {
int plane_kernel_name(const mb_handle *h, int nk, int nbands, int prec, char *buf, int len);

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
    // candidates: every compact-plane instance that can run the batch (FP32),
    // and the register-FFT / radix-2 kernels with 1..4 bands per CTA; each
    // with the wave model's run count and with explicit wave targets
    std::vector<mb_handle::Tuned> cand;
    if (c2 == 8) {
        int nocc_max = 0, maxldg = 0;
        for (int i = 0; i < std::min(nk, kMaxK); ++i) {
            nocc_max = std::max(nocc_max, h->nocc[i]);
            maxldg = std::max(maxldg, h->kp[i].ldg);
        }
        Plane32Shape shapes[kMaxPlane32Shapes];
        const int ns = plane32_shapes(h->n1, h->n2, h->order, h->nquad, nocc_max, maxldg, shapes, kMaxPlane32Shapes);
        for (int v = 0; v < ns; ++v)
            for (int persist : {0, 1})
                for (int waves : {0, 1, 2, 4, 8}) {
                    mb_handle::Tuned t;
                    t.p32 = shapes[v].id;
                    t.waves = waves;
                    t.persist = persist;
                    cand.push_back(t);
                }
    }
    for (int bt = small ? 4 : 2; bt >= 1; --bt)
        for (int waves : {0, 1, 2, 4, 8}) {
            mb_handle::Tuned t;
            t.bt = bt;
            t.waves = waves;
            t.p32 = -2;            // not the compact-plane kernel
            cand.push_back(t);
        }
    double best = 1e300;
    mb_handle::Tuned bestp = cand.empty() ? mb_handle::Tuned() : cand[0];
    h->tune_report.clear();
    for (const auto &c : cand) {
        if (rc != MB_OK) break;
        h->tuned[key] = c;
        char name[160];
        plane_kernel_name(h, nk, nbands, prec, name, sizeof(name));
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
        if (rc == MB_OK) {
            char line[256];
            std::snprintf(line, sizeof(line), "%s bands/CTA %d waves %d: %.4f ms\n", name,
                          c.p32 >= 0 ? 0 : c.bt, c.waves, ms / 5);   // the name says "persistent" for the queue launch
            h->tune_report += line;
        }
        if (rc == MB_OK && ms / 5 < best) {
            best = ms / 5;
            bestp = c;
        }
    }
    h->tuned[key] = bestp;
    if (best_bt) *best_bt = bestp.p32 >= 0 ? -1 - bestp.p32 : bestp.bt;
    if (best_waves) *best_waves = bestp.waves;
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

// Name of the plane-kernel instance an apply of `nbands` bands at k-points
// 0 .. min(nk, kMaxK)-1 launches now (after any mb_autotune of that shape).
int plane_kernel_name(const mb_handle *h, int nk, int nbands, int prec, char *buf, int len) {
    if (!buf || len < 1 || nk < 1 || nbands < 1) return MB_EINVAL;
    nk = std::min(std::min(nk, (int)h->kp.size()), kMaxK);
    std::vector<int> iks(nk);
    for (int i = 0; i < nk; ++i) iks[i] = i;
    const size_t c2 = prec == MB_FP64 ? 16 : 8;
    const bool reg = prec == MB_FP64 ? plane_reg_supported<double>(h->n1, h->n2, h->order)
                                     : plane_reg_supported<float>(h->n1, h->n2, h->order);
    const PlanePlan p = plan_plane(h, nk, iks.data(), nbands, c2, reg);
    char tmp[128];
    if (p.p32) std::snprintf(tmp, sizeof(tmp), "%s%s", p.sh.name, p.persist ? " persistent" : "");
    else if (p.reg) std::snprintf(tmp, sizeof(tmp), "plane_reg_kernel<%s, %d, %d, %d>", c2 == 8 ? "float" : "double", h->n1, h->n2, h->order);
    else std::snprintf(tmp, sizeof(tmp), "plane_kernel<%s>", c2 == 8 ? "float" : "double");
    std::snprintf(buf, (size_t)len, "%s", tmp);
    return MB_OK;
}
}  // namespace mb

extern "C" int mb_autotune(mb_handle *h, int nbands, int prec, int *best_bt, int *best_waves, double *best_ms) {
    if (!h) return MB_EINVAL;
    return mb::autotune(h, nbands, prec, best_bt, best_waves, best_ms);
}

extern "C" int mb_plane_kernel_name(const mb_handle *h, int nk, int nbands, int prec, char *buf, int len) {
    if (!h) return MB_EINVAL;
    return mb::plane_kernel_name(h, nk, nbands, prec, buf, len);
}

namespace mb {
static int plane_candidates(const mb_handle *h, int nk, int prec, int *ids, int max) {
    if (prec == MB_FP64) return 0;
    nk = std::min(std::min(nk, (int)h->kp.size()), kMaxK);
    int nocc_max = 0, maxldg = 0;
    for (int i = 0; i < nk; ++i) {
        nocc_max = std::max(nocc_max, h->nocc[i]);
        maxldg = std::max(maxldg, h->kp[i].ldg);
    }
    Plane32Shape shapes[kMaxPlane32Shapes];
    const int ns = plane32_shapes(h->n1, h->n2, h->order, h->nquad, nocc_max, maxldg, shapes, kMaxPlane32Shapes);
    int n = 0;   // the instances whose shared memory fits this batch
    for (int v = 0; v < ns; ++v)
        if (p32_fits(h, shapes[v], maxldg)) {
            if (n < max) ids[n] = shapes[v].id;
            ++n;
        }
    return n;
}
}  // namespace mb

extern "C" int mb_plane_kernel_candidates(const mb_handle *h, int nk, int nbands, int prec, int *ids, int max) {
    if (!h || !ids || nk < 1 || nbands < 1 || max < 0) return -MB_EINVAL;
    if (prec != MB_FP64 && prec != MB_FP32 && prec != MB_BF16) return -MB_EINVAL;
    return mb::plane_candidates(h, nk, prec, ids, max);
}

extern "C" int mb_plane_kernel_select(mb_handle *h, int nk, int nbands, int prec, int id, int waves,
                                      int persistent) {
    if (!h || nk < 1 || nbands < 1 || waves < 0 || id < -2) return MB_EINVAL;
    if (prec != MB_FP64 && prec != MB_FP32 && prec != MB_BF16) return MB_EINVAL;
    if (id >= 0) {
        int ids[mb::kMaxPlane32Shapes];
        const int n = mb::plane_candidates(h, nk, prec, ids, mb::kMaxPlane32Shapes);
        bool ok = false;
        for (int i = 0; i < n; ++i) ok = ok || ids[i] == id;
        if (!ok) return MB_EINVAL;
    }
    mb_handle::Tuned t;
    t.p32 = id;
    t.waves = waves;
    t.persist = persistent ? 1 : 0;
    t.bt = h->n1 <= 32 && h->n2 <= 32 ? 2 : 1;
    h->tuned[std::make_tuple(std::min(std::min(nk, (int)h->kp.size()), mb::kMaxK), nbands, prec == MB_FP64 ? 1 : 0)] = t;
    return MB_OK;
}

extern "C" int mb_autotune_report(const mb_handle *h, char *buf, int len) {
    if (!h || !buf || len < 1) return MB_EINVAL;
    std::snprintf(buf, (size_t)len, "%s", h->tune_report.c_str());
    return MB_OK;
}
