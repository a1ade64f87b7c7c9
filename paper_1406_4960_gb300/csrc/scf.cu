// The self-consistent loop of §II.B.1 and §III.A on the device, in FP64.
//
//  density_kernel      rho(r, z_q) = sum_{k,n} f_nk |phi_nk(r, z_q)|^2 with
//                      phi = A_c^(-1/2) sum_{G,j} c_{Gj} e^{i(k+G).r} B_j(z)
//                      (Eq. (6)): B-spline evaluation on the Gauss planes of
//                      one knot interval, inverse 2D FFT in shared memory,
//                      f |.|^2 accumulated into the CTA's own partial table;
//                      density_reduce_kernel sums the partials in a fixed
//                      order (deterministic, no atomics).
//  hartree_*           the electrons' Coulomb potential through the 2D
//                      transform of 1/r (the Coulomb integral of §II.B.1):
//                      per in-plane component g,
//                        V(z_q, g) = sum_q' w_q' rho(z_q', g) (2 pi/g) e^{-g |z_q - z_q'|}
//                      as two exponentially weighted sweeps over the planes
//                      (every factor e^{-g dz} <= 1), and at g = 0
//                        V(z_q, 0) = -2 pi sum_q' w_q' rho(z_q', 0) |z_q - z_q'|
//                      by prefix sums (the net-charge constant (2 pi/g) Q is
//                      dropped, as for the core term).
//  xc_lda_kernel       LDA exchange and the Perdew-Zunger (1981)
//                      parametrization of the Ceperley-Alder correlation.
//  mixing kernels      the paper's Kerker form on g != 0; the g = 0 profile
//                      (which the printed factor would freeze) scaled by the
//                      factor of the grid's first nonzero shell, so the
//                      mixing stays local in z and keeps the electron count;
//                      Pulay over the last steps (§III.A).
//  aug_integral_kernel int V_eff g_a d^3r for the ultrasoft atoms' normalized
//                      augmentation Gaussians g_a, in the planes' components.
// mb_scf drives the loop: V_scf = V_H + V_xc of the input density is added
// to the atoms' table, the eigensolver runs on the handle, Fermi-Dirac
// occupations give the output density, and the mixer the next input, until
// V_scf changes by less than the tolerance.  With ultrasoft atoms (§II.B.2)
// every iteration also sets the strengths D_pq = E_pq + q_pq int V_eff g_a
// (Q_pq = q_pq g_a) and augments the output density by
// g_a sum_n f_n sum_pq q_pq <phi_n|beta_p><beta_q|phi_n>.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "cplx.cuh"
#include "fft_smem.cuh"
#include "mb_internal.h"

namespace mb {

namespace {

constexpr int kDensMaxK = 32;   // k-points per density launch (descriptors are kernel parameters)
constexpr int kMaxPulay = 8;
constexpr double kTwoPi = 6.283185307179586476925;

// Perdew-Zunger (1981) parametrization of the Ceperley-Alder correlation
// energy per electron of the unpolarized electron gas (Hartree)
constexpr double kPzGamma = -0.1423, kPzBeta1 = 1.0529, kPzBeta2 = 0.3334;
constexpr double kPzA = 0.0311, kPzB = -0.048, kPzC = 0.0020, kPzD = -0.0116;
// The LDA is evaluated at max(rho, kRhoFloor) (bohr^-3): the vacuum's densities
// of 1e-16 and below are noise of the FP64 sums and of the eigenvectors, and
// their cube root would dominate every change of V_xc; below the floor the
// potential is the small constant v_xc(kRhoFloor), continuous in rho.
constexpr double kRhoFloor = 1e-10;

struct DensK {
    const double2 *X;   // nbands x nb x ldg coefficients of this k-point
    int ng, ldg, kofs, kg;
};

struct DensArgs {
    const double *Bq;    // nq x order
    const int *goff;     // all k: natural grid offset of each G
    const double *occ;   // nk x nbands occupations
    double *part;        // (nk nslice) x nq x N1 N2, bit-reversed plane layout
    const double2 *tw;   // nmax/2 twiddles exp(+2 pi i k / nmax)
    int n1, n2, nmax, order, nquad, nb, nint, nbands, nslice, np, nq;
    DensK d[kDensMaxK];
};

// One (knot interval t, band slice, k-point): the density of its bands on the
// interval's Gauss planes, into the CTA's own partial planes.
__global__ void __launch_bounds__(256) density_kernel(const __grid_constant__ DensArgs a) {
    extern __shared__ __align__(16) unsigned char dsm[];
    const int NN = a.n1 * a.n2, K = a.order, P = a.nquad;
    double2 *tw = reinterpret_cast<double2 *>(dsm);
    double2 *buf = tw + a.nmax / 2;
    for (int i = threadIdx.x; i < a.nmax / 2; i += blockDim.x) tw[i] = a.tw[i];
    const int t = blockIdx.x, sl = blockIdx.y;
    const DensK &d = a.d[blockIdx.z];
    const int n0 = sl * a.nbands / a.nslice, n1 = (sl + 1) * a.nbands / a.nslice;
    double *part = a.part + ((size_t)(d.kg * a.nslice + sl) * a.nq + (size_t)t * P) * NN;
    for (int e = threadIdx.x; e < P * NN; e += blockDim.x) part[e] = 0.0;
    const int *goff = a.goff + d.kofs;
    for (int n = n0; n < n1; ++n) {
        const double f = a.occ[(size_t)d.kg * a.nbands + n];
        if (f == 0.0) continue;                  // uniform over the CTA
        const double2 *X = d.X + (size_t)n * a.nb * d.ldg;
        for (int s0 = 0; s0 < P; s0 += a.np) {
            const int ns = min(a.np, P - s0), q0 = t * P + s0;
            __syncthreads();                     // the previous group's planes are consumed
            for (int e = threadIdx.x; e < ns * NN; e += blockDim.x) buf[e] = czero<double2>();
            __syncthreads();
            // psi_q(G) = sum_m B_{t+m}(z_q) c[t+m-1][G]
            for (int g = threadIdx.x; g < d.ng; g += blockDim.x) {
                double2 x[8];
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    const int j = t + m - 1;
                    x[m] = (m < K && j >= 0 && j < a.nb) ? X[(size_t)j * d.ldg + g] : czero<double2>();
                }
                const int o = goff[g];
                for (int s = 0; s < ns; ++s) {
                    const double *bq = a.Bq + (size_t)(q0 + s) * K;
                    double2 psi = czero<double2>();
#pragma unroll
                    for (int m = 0; m < 8; ++m)
                        if (m < K) rfma(psi, bq[m], x[m]);
                    buf[s * NN + o] = psi;
                }
            }
            __syncthreads();
            fft_axis<double2, true>(buf, ns, a.n1, a.n2, 2, tw, a.nmax);
            fft_axis<double2, true>(buf, ns, a.n1, a.n2, 1, tw, a.nmax);
            for (int e = threadIdx.x; e < ns * NN; e += blockDim.x) {
                const double2 p = buf[e];
                part[(size_t)s0 * NN + e] += f * (p.x * p.x + p.y * p.y);
            }
        }
    }
}

__device__ __forceinline__ int brev_bits(int x, int bits) { return (int)(__brev((unsigned)x) >> (32 - bits)); }

// rho[q][i1][i2] = scale * sum over the partials (in order) at the bit-reversed position
__global__ void density_reduce_kernel(const double *part, int nparts, int nq, int N1, int N2, int l1, int l2,
                                      double scale, double *rho) {
    const int NN = N1 * N2;
    const size_t total = (size_t)nq * NN;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int q = (int)(e / NN), r = (int)(e % NN), i1 = r / N2, i2 = r % N2;
        const size_t pb = (size_t)q * NN + (size_t)brev_bits(i1, l1) * N2 + brev_bits(i2, l2);
        double s = 0.0;
        for (int p = 0; p < nparts; ++p) s += part[(size_t)p * total + pb];
        rho[e] = scale * s;
    }
}

// 2D transforms of np planes per CTA in shared memory.
// Forward (INV = false): natural real (in_r) or complex (in_c) input ->
//   out_c[q][m] = scale * sum_r f(r) e^{-i g_m . r}, natural order.
// Inverse (INV = true): natural complex spectrum in_c ->
//   out_r[q][r] = scale * Re sum_m c(m) e^{+i g_m . r}.
template <bool INV>
__global__ void __launch_bounds__(256) plane_fft2_kernel(const double *in_r, const double2 *in_c, double *out_r,
                                                         double2 *out_c, int nq, int N1, int N2, int l1, int l2,
                                                         int nmax, int np, const double2 *twg, double scale) {
    extern __shared__ __align__(16) unsigned char fsm[];
    double2 *tw = reinterpret_cast<double2 *>(fsm);
    double2 *buf = tw + nmax / 2;
    for (int i = threadIdx.x; i < nmax / 2; i += blockDim.x) tw[i] = twg[i];
    const int NN = N1 * N2, q0 = blockIdx.x * np, ns = min(np, nq - q0);
    for (int e = threadIdx.x; e < ns * NN; e += blockDim.x) {
        const int s = e / NN, r = e % NN;
        const size_t src = (size_t)(q0 + s) * NN + r;
        if (INV) {
            buf[e] = in_c[src];
        } else {
            const int i1 = r / N2, i2 = r % N2;
            const double2 v = in_r ? make_double2(in_r[src], 0.0) : in_c[src];
            buf[s * NN + brev_bits(i1, l1) * N2 + brev_bits(i2, l2)] = v;   // DIT input order
        }
    }
    __syncthreads();
    if (INV) {
        fft_axis<double2, true>(buf, ns, N1, N2, 2, tw, nmax);
        fft_axis<double2, true>(buf, ns, N1, N2, 1, tw, nmax);
    } else {
        fft_axis<double2, false>(buf, ns, N1, N2, 1, tw, nmax);
        fft_axis<double2, false>(buf, ns, N1, N2, 2, tw, nmax);
    }
    for (int e = threadIdx.x; e < ns * NN; e += blockDim.x) {
        const int s = e / NN, r = e % NN;
        const size_t dst = (size_t)(q0 + s) * NN + r;
        if (INV) {
            const int i1 = r / N2, i2 = r % N2;
            out_r[dst] = scale * buf[s * NN + brev_bits(i1, l1) * N2 + brev_bits(i2, l2)].x;
        } else {
            const double2 v = buf[e];
            out_c[dst] = make_double2(scale * v.x, scale * v.y);
        }
    }
}

__device__ __forceinline__ double2 shfl_up2(double2 v, int d) {
    return make_double2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
}
__device__ __forceinline__ double2 shfl_down2(double2 v, int d) {
    return make_double2(__shfl_down_sync(0xffffffffu, v.x, d), __shfl_down_sync(0xffffffffu, v.y, d));
}
__device__ __forceinline__ double2 axpy2(double a, double2 x, double2 y) {
    return make_double2(fma(a, x.x, y.x), fma(a, x.y, y.y));
}

// Coulomb integral per in-plane component, one warp per component g, the
// planes (in z order) split into 32 consecutive chunks, one per lane.
// g != 0: the forward sums L_q = f_q L_{q-1} + a_q (a = w rho, f_q =
// e^{-g (z_q - z_{q-1})} <= 1) and the backward sums R_{q-1} = f_q (R_q + a_q)
// are affine maps per chunk (L_out = A L_in + B, A = e^{-g (z_last - z_{first-1})}),
// combined across the lanes by shuffle scans and then re-run with the carry:
// V_q = (2 pi/g)(L_q + R_q).  g = 0: -2 pi sum_q' a_q' |z_q - z_q'| from the
// prefix sums of a and a z, scanned the same way.
__global__ void __launch_bounds__(128) hartree_sweep_kernel(const double2 *rg, double2 *vg, const double *zq,
                                                            const double *wq, int nq, int N1, int N2, double b1x,
                                                            double b1y, double b2x, double b2y) {
    const int NN = N1 * N2;
    const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (e >= NN) return;                         // whole warps
    const int u = e / N2, v = e % N2;
    const int m1 = u < N1 / 2 ? u : u - N1, m2 = v < N2 / 2 ? v : v - N2;
    const double gx = m1 * b1x + m2 * b2x, gy = m1 * b1y + m2 * b2y;
    const double g = sqrt(gx * gx + gy * gy);
    const int C = (nq + 31) / 32, q0 = min(nq, lane * C), q1 = min(nq, q0 + C);
    auto a_at = [&](int q) {
        const double2 r = rg[(size_t)q * NN + e];
        return make_double2(wq[q] * r.x, wq[q] * r.y);
    };
    if (g == 0.0) {
        double2 P = czero<double2>(), Pz = czero<double2>();
        for (int q = q0; q < q1; ++q) {
            const double2 a = a_at(q);
            P = P + a;
            Pz = axpy2(zq[q], a, Pz);
        }
        // inclusive sums over the lanes, totals from the last lane
        for (int d = 1; d < 32; d <<= 1) {
            const double2 p = shfl_up2(P, d), pz = shfl_up2(Pz, d);
            if (lane >= d) {
                P = P + p;
                Pz = Pz + pz;
            }
        }
        const double2 PT = make_double2(__shfl_sync(0xffffffffu, P.x, 31), __shfl_sync(0xffffffffu, P.y, 31));
        const double2 PzT = make_double2(__shfl_sync(0xffffffffu, Pz.x, 31), __shfl_sync(0xffffffffu, Pz.y, 31));
        P = shfl_up2(P, 1);
        Pz = shfl_up2(Pz, 1);
        if (lane == 0) P = Pz = czero<double2>();
        for (int q = q0; q < q1; ++q) {
            const double2 a = a_at(q);
            const double z = zq[q];
            P = P + a;
            Pz = axpy2(z, a, Pz);
            const double re = z * P.x - Pz.x + (PzT.x - Pz.x) - z * (PT.x - P.x);
            const double im = z * P.y - Pz.y + (PzT.y - Pz.y) - z * (PT.y - P.y);
            vg[(size_t)q * NN + e] = make_double2(-kTwoPi * re, -kTwoPi * im);
        }
        return;
    }
    auto f_at = [&](int q) { return q > 0 ? exp(-g * (zq[q] - zq[q - 1])) : 0.0; };
    // this chunk's maps: forward L and backward R (same multiplier A)
    double A = 1.0;
    double2 BL = czero<double2>(), BR = czero<double2>();
    if (q1 > q0) {
        A = q0 > 0 ? exp(-g * (zq[q1 - 1] - zq[q0 - 1])) : 0.0;
        for (int q = q0; q < q1; ++q) BL = axpy2(f_at(q), BL, a_at(q));
        for (int q = q1 - 1; q >= q0; --q) {
            const double2 a = a_at(q);
            const double f = f_at(q);
            BR = make_double2(f * (BR.x + a.x), f * (BR.y + a.y));
        }
    }
    // forward: inclusive scan from lane 0 (earlier chunks applied first)
    double IA = A;
    double2 IB = BL;
    for (int d = 1; d < 32; d <<= 1) {
        const double pa = __shfl_up_sync(0xffffffffu, IA, d);
        const double2 pb = shfl_up2(IB, d);
        if (lane >= d) {
            IB = axpy2(IA, pb, IB);
            IA *= pa;
        }
    }
    double2 L = shfl_up2(IB, 1);
    if (lane == 0) L = czero<double2>();
    for (int q = q0; q < q1; ++q) {
        L = axpy2(f_at(q), L, a_at(q));
        vg[(size_t)q * NN + e] = L;
    }
    // backward: inclusive scan from lane 31 (later chunks applied first)
    double JA = A;
    double2 JB = BR;
    for (int d = 1; d < 32; d <<= 1) {
        const double pa = __shfl_down_sync(0xffffffffu, JA, d);
        const double2 pb = shfl_down2(JB, d);
        if (lane + d < 32) {
            JB = axpy2(JA, pb, JB);
            JA *= pa;
        }
    }
    double2 R = shfl_down2(JB, 1);
    if (lane == 31) R = czero<double2>();
    const double c = kTwoPi / g;
    for (int q = q1 - 1; q >= q0; --q) {
        const double2 l = vg[(size_t)q * NN + e];
        vg[(size_t)q * NN + e] = make_double2(c * (l.x + R.x), c * (l.y + R.y));
        const double2 a = a_at(q);
        const double f = f_at(q);
        R = make_double2(f * (R.x + a.x), f * (R.y + a.y));
    }
}

__global__ void xc_lda_kernel(const double *rho, double *vxc, double *exc, size_t n) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const double d = fmax(rho[e], kRhoFloor);
        const double rs = cbrt(3.0 / (4.0 * 3.14159265358979323846 * d));
        const double ex = -0.75 * cbrt(3.0 * d / 3.14159265358979323846);
        double ec, vc;
        if (rs >= 1.0) {
            const double sr = sqrt(rs), den = 1.0 + kPzBeta1 * sr + kPzBeta2 * rs;
            ec = kPzGamma / den;
            vc = ec * (1.0 + (7.0 / 6.0) * kPzBeta1 * sr + (4.0 / 3.0) * kPzBeta2 * rs) / den;
        } else {
            const double lr = log(rs);
            ec = kPzA * lr + kPzB + kPzC * rs * lr + kPzD * rs;
            vc = kPzA * lr + (kPzB - kPzA / 3.0) + (2.0 / 3.0) * kPzC * rs * lr + (2.0 * kPzD - kPzC) * rs / 3.0;
        }
        const double v = (4.0 / 3.0) * ex + vc, en = ex + ec;
        vxc[e] = v;
        if (exc) exc[e] = en;
    }
}

// One (plane q, ultrasoft atom a): Ac w_q sum_m Re(conj(V(z_q, m)) g_a(z_q, m)),
// g_a's components (1/(sqrt(pi) r_Q A_c)) e^{-g^2 r_Q^2/4 - dz^2/r_Q^2} e^{-i g.R}.
// The host adds the planes in order: int V g_a = sum_q out[a][q].
__global__ void __launch_bounds__(256) aug_integral_kernel(const double2 *Vg, const double *atoms, const double *zq,
                                                           const double *wq, int nq, int N1, int N2, double b1x,
                                                           double b1y, double b2x, double b2y, double Ac,
                                                           double *out) {
    __shared__ double red[256];
    const int q = blockIdx.x, at = blockIdx.y, NN = N1 * N2;
    const double x = atoms[4 * at], y = atoms[4 * at + 1], dz = zq[q] - atoms[4 * at + 2], rq = atoms[4 * at + 3];
    const double pre = 0.56418958354775628695 / (rq * Ac) * exp(-(dz / rq) * (dz / rq));
    double acc = 0.0;
    for (int e = threadIdx.x; e < NN; e += 256) {
        const int u = e / N2, v = e % N2;
        const int m1 = u < N1 / 2 ? u : u - N1, m2 = v < N2 / 2 ? v : v - N2;
        const double gx = m1 * b1x + m2 * b2x, gy = m1 * b1y + m2 * b2y;
        double sn, cs;
        sincos(-(gx * x + gy * y), &sn, &cs);
        const double a = pre * exp(-0.25 * (gx * gx + gy * gy) * rq * rq);
        const double2 V = Vg[(size_t)q * NN + e];
        acc += V.x * a * cs + V.y * a * sn;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[(size_t)at * nq + q] = Ac * wq[q] * red[0];
}

// out = a + b (+ c)
__global__ void add_kernel(const double *a, const double *b, const double *c, double *out, size_t n) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        out[e] = a[e] + b[e] + (c ? c[e] : 0.0);
}

// out = a - b (complex)
__global__ void csub_kernel(const double2 *a, const double2 *b, double2 *out, size_t n) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        out[e] = a[e] - b[e];
}

// One block per plane (256 threads): out[q] = w_q sum_e Re(conj(a) b)  (or,
// with MAXDIFF, max_e |a - b| of real fields), fixed-order tree.
template <bool MAXDIFF>
__global__ void __launch_bounds__(256) plane_reduce_kernel(const void *pa, const void *pb, const double *wq, int NN,
                                                           double *out) {
    __shared__ double red[256];
    const int q = blockIdx.x;
    double s = 0.0;
    for (int e = threadIdx.x; e < NN; e += 256) {
        if (MAXDIFF) {
            const double *a = reinterpret_cast<const double *>(pa) + (size_t)q * NN;
            const double *b = reinterpret_cast<const double *>(pb) + (size_t)q * NN;
            s = fmax(s, fabs(a[e] - b[e]));
        } else {
            const double2 *a = reinterpret_cast<const double2 *>(pa) + (size_t)q * NN;
            const double2 *b = reinterpret_cast<const double2 *>(pb) + (size_t)q * NN;
            s += a[e].x * b[e].x + a[e].y * b[e].y;
        }
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            red[threadIdx.x] = MAXDIFF ? fmax(red[threadIdx.x], red[threadIdx.x + w]) : red[threadIdx.x] + red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = MAXDIFF ? red[0] : wq[q] * red[0];
}

struct MixArgs {
    const double2 *rin[kMaxPulay], *res[kMaxPulay];
    double a[kMaxPulay];
    int m, N1, N2, NN;
    double b1x, b1y, b2x, b2y, W, gmax2, K0;
};

// out(z, g) = sum_i a_i rho_in_i + K(g) sum_i a_i R_i, K = W g^2/(g^2 + g_max^2)
// (g != 0), K0 = the same factor on the grid's first nonzero shell (g = 0)
__global__ void mix_combine_kernel(const __grid_constant__ MixArgs a, double2 *out, size_t n) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e % a.NN), u = r / a.N2, v = r % a.N2;
        const int m1 = u < a.N1 / 2 ? u : u - a.N1, m2 = v < a.N2 / 2 ? v : v - a.N2;
        const double gx = m1 * a.b1x + m2 * a.b2x, gy = m1 * a.b1y + m2 * a.b2y, g2 = gx * gx + gy * gy;
        const double K = g2 > 0.0 ? a.W * g2 / (g2 + a.gmax2) : a.K0;
        double2 x = czero<double2>(), y = czero<double2>();
        for (int i = 0; i < a.m; ++i) {
            const double2 p = a.rin[i][e], q = a.res[i][e];
            x = make_double2(x.x + a.a[i] * p.x, x.y + a.a[i] * p.y);
            y = make_double2(y.x + a.a[i] * q.x, y.y + a.a[i] * q.y);
        }
        out[e] = make_double2(x.x + K * y.x, x.y + K * y.y);
    }
}

int grid_blocks(const mb_handle *h, size_t n) {
    return (int)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, (size_t)h->num_sms * 8));
}

// planes of N1 x N2 complex doubles per CTA of the shared-memory FFTs
int fft_planes(const mb_handle *h, int cap) {
    const size_t NN = (size_t)h->n1 * h->n2, tw = (size_t)std::max(h->n1, h->n2) / 2 * sizeof(double2);
    const size_t room = (size_t)h->smem_optin > tw ? (size_t)h->smem_optin - tw : 0;
    return (int)std::min<size_t>((size_t)cap, room / (NN * sizeof(double2)));
}

struct Buf {
    mb_handle *h;
    cudaStream_t s;
    std::vector<void *> ptrs;
    int rc = MB_OK;
    template <typename T> T *get(size_t n) {
        void *p = nullptr;
        cudaMemPool_t pool = mb_pool(h->device);
        if (rc || !pool) {
            rc = rc ? rc : MB_ECUDA;
            return nullptr;
        }
        cudaError_t e = cudaMallocFromPoolAsync(&p, std::max<size_t>(n, 1) * sizeof(T), pool, s);
        if (e != cudaSuccess) {
            rc = cuda_fail(h, e);
            return nullptr;
        }
        ptrs.push_back(p);
        return reinterpret_cast<T *>(p);
    }
    ~Buf() {
        for (void *p : ptrs) cudaFreeAsync(p, s);
    }
};

int check_tables(mb_handle *h) {
    if (!h || !h->d_vloc || !h->t64.Bq || !h->t64.tw) return MB_EINVAL;
    if (fft_planes(h, 1) < 1) return MB_EUNSUPPORTED;   // one plane must fit in shared memory
    return MB_OK;
}

}  // namespace

// rho (device, nq x N1 x N2) from the eigenvectors evecs (the layout of
// mb_eigsolve's) and the occupations occ_dev (device, nk x nbands).
int scf_density(mb_handle *h, const void *evecs, int nbands, const double *occ_dev, double *rho, cudaStream_t s) {
    const int nk = (int)h->kp.size(), NN = h->n1 * h->n2, P = h->nquad;
    const int nmax = std::max(h->n1, h->n2);
    const int np = fft_planes(h, P);
    int nslice = std::max(1, std::min(nbands, (2 * h->num_sms + h->nint * nk - 1) / (h->nint * nk)));
    const int nparts = nk * nslice;
    Buf B{h, s};
    double *part = B.get<double>((size_t)nparts * h->nq * NN);
    if (B.rc) return B.rc;
    const size_t smem = (size_t)(nmax / 2 + (size_t)np * NN) * sizeof(double2);
    MB_CUDA(smem_limit_once((const void *)density_kernel, h->device, h->smem_optin));
    DensArgs a;
    a.Bq = reinterpret_cast<const double *>(h->t64.Bq);
    a.goff = h->d_goff;
    a.occ = occ_dev;
    a.part = part;
    a.tw = reinterpret_cast<const double2 *>(h->t64.tw);
    a.n1 = h->n1;
    a.n2 = h->n2;
    a.nmax = nmax;
    a.order = h->order;
    a.nquad = P;
    a.nb = h->nb;
    a.nint = h->nint;
    a.nbands = nbands;
    a.nslice = nslice;
    a.np = np;
    a.nq = h->nq;
    size_t off = 0;
    std::vector<size_t> koff(nk);
    for (int k = 0; k < nk; ++k) {
        koff[k] = off;
        off += (size_t)nbands * h->nb * h->kp[k].ldg;
    }
    for (int k0 = 0; k0 < nk; k0 += kDensMaxK) {
        const int n = std::min(kDensMaxK, nk - k0);
        for (int i = 0; i < n; ++i) {
            const int k = k0 + i;
            a.d[i].X = reinterpret_cast<const double2 *>(evecs) + koff[k];
            a.d[i].ng = h->kp[k].ng;
            a.d[i].ldg = h->kp[k].ldg;
            a.d[i].kofs = h->kofs[k];
            a.d[i].kg = k;
        }
        density_kernel<<<dim3(h->nint, nslice, n), 256, smem, s>>>(a);
        MB_CUDA(cudaGetLastError());
        ++h->launches;
    }
    const size_t total = (size_t)h->nq * NN;
    density_reduce_kernel<<<grid_blocks(h, total), 256, 0, s>>>(part, nparts, h->nq, h->n1, h->n2, h->l1, h->l2,
                                                                1.0 / h->Ac, rho);
    MB_CUDA(cudaGetLastError());
    ++h->launches;
    return MB_OK;
}

// 2D transform of the nq planes: forward (real or complex natural -> scaled
// natural spectrum) or inverse (spectrum -> real field).
static int plane_fft2(mb_handle *h, bool inv, const double *in_r, const double2 *in_c, double *out_r, double2 *out_c,
                      double scale, cudaStream_t s) {
    const int NN = h->n1 * h->n2, nmax = std::max(h->n1, h->n2);
    const int np = fft_planes(h, 8);
    const size_t smem = (size_t)(nmax / 2 + (size_t)np * NN) * sizeof(double2);
    const int grid = (h->nq + np - 1) / np;
    const double2 *tw = reinterpret_cast<const double2 *>(h->t64.tw);
    if (inv) {
        MB_CUDA(smem_limit_once((const void *)plane_fft2_kernel<true>, h->device, h->smem_optin));
        plane_fft2_kernel<true><<<grid, 256, smem, s>>>(in_r, in_c, out_r, out_c, h->nq, h->n1, h->n2, h->l1, h->l2,
                                                         nmax, np, tw, scale);
    } else {
        MB_CUDA(smem_limit_once((const void *)plane_fft2_kernel<false>, h->device, h->smem_optin));
        plane_fft2_kernel<false><<<grid, 256, smem, s>>>(in_r, in_c, out_r, out_c, h->nq, h->n1, h->n2, h->l1, h->l2,
                                                          nmax, np, tw, scale);
    }
    MB_CUDA(cudaGetLastError());
    ++h->launches;
    return MB_OK;
}

struct ScfPlanes {
    double *zq = nullptr, *wq = nullptr;   // device copies of the planes
};

static int hartree_g(mb_handle *h, const double2 *rg, double2 *vg, const ScfPlanes &pl, cudaStream_t s) {
    const int NN = h->n1 * h->n2;
    hartree_sweep_kernel<<<(NN + 3) / 4, 128, 0, s>>>(rg, vg, pl.zq, pl.wq, h->nq, h->n1, h->n2, h->b1[0],
                                                       h->b1[1], h->b2[0], h->b2[1]);
    MB_CUDA(cudaGetLastError());
    ++h->launches;
    return MB_OK;
}

static int upload_planes(mb_handle *h, Buf &B, ScfPlanes &pl, cudaStream_t s) {
    pl.zq = B.get<double>(h->nq);
    pl.wq = B.get<double>(h->nq);
    if (B.rc) return B.rc;
    MB_CUDA(cudaMemcpyAsync(pl.zq, h->zq.data(), sizeof(double) * h->nq, cudaMemcpyHostToDevice, s));
    MB_CUDA(cudaMemcpyAsync(pl.wq, h->wq.data(), sizeof(double) * h->nq, cudaMemcpyHostToDevice, s));
    return MB_OK;
}

// V_H (real field) of the density rho (real field)
static int hartree(mb_handle *h, const double *rho, double *vh, Buf &B, const ScfPlanes &pl, cudaStream_t s,
                   double2 *rg = nullptr, double2 *vg = nullptr) {
    const size_t n = (size_t)h->nq * h->n1 * h->n2;
    if (!rg) rg = B.get<double2>(n);
    if (!vg) vg = B.get<double2>(n);
    if (B.rc) return B.rc;
    int rc;
    if ((rc = plane_fft2(h, false, rho, nullptr, nullptr, rg, 1.0 / (h->n1 * h->n2), s))) return rc;
    if ((rc = hartree_g(h, rg, vg, pl, s))) return rc;
    return plane_fft2(h, true, nullptr, vg, vh, nullptr, 1.0, s);
}

static int xc(mb_handle *h, const double *rho, double *vxc, double *exc, cudaStream_t s) {
    const size_t n = (size_t)h->nq * h->n1 * h->n2;
    xc_lda_kernel<<<grid_blocks(h, n), 256, 0, s>>>(rho, vxc, exc, n);
    MB_CUDA(cudaGetLastError());
    ++h->launches;
    return MB_OK;
}

// Bordered Pulay system [[A, 1], [1^T, 0]] [a; l] = [0; 1] by Gaussian
// elimination with partial pivoting; false when it is singular.
static bool pulay_solve(std::vector<double> A, int m, std::vector<double> &a) {
    const int n = m + 1;
    std::vector<double> M((size_t)n * n, 0.0), b(n, 0.0);
    double scale = 0.0;
    for (int i = 0; i < m; ++i) scale = std::max(scale, std::fabs(A[(size_t)i * m + i]));
    if (!(scale > 0.0)) scale = 1.0;
    for (int i = 0; i < m; ++i) {
        for (int j = 0; j < m; ++j) M[(size_t)i * n + j] = A[(size_t)i * m + j] / scale;
        M[(size_t)i * n + m] = M[(size_t)m * n + i] = 1.0;
    }
    b[m] = 1.0;
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(M[(size_t)r * n + c]) > std::fabs(M[(size_t)p * n + c])) p = r;
        if (!(std::fabs(M[(size_t)p * n + c]) > 1e-14)) return false;
        if (p != c) {
            for (int j = 0; j < n; ++j) std::swap(M[(size_t)p * n + j], M[(size_t)c * n + j]);
            std::swap(b[p], b[c]);
        }
        for (int r = c + 1; r < n; ++r) {
            const double f = M[(size_t)r * n + c] / M[(size_t)c * n + c];
            for (int j = c; j < n; ++j) M[(size_t)r * n + j] -= f * M[(size_t)c * n + j];
            b[r] -= f * b[c];
        }
    }
    std::vector<double> x(n, 0.0);
    for (int r = n - 1; r >= 0; --r) {
        double v = b[r];
        for (int j = r + 1; j < n; ++j) v -= M[(size_t)r * n + j] * x[j];
        x[r] = v / M[(size_t)r * n + r];
    }
    a.assign(x.begin(), x.begin() + m);
    return true;
}

// Fermi-Dirac occupations (two electrons per state, k weights); mu by bisection.
static double occupations(const std::vector<double> &ev, const std::vector<double> &wk, int nbands, double nelec,
                          double sigma, std::vector<double> &f) {
    const int nk = (int)wk.size();
    auto fd = [&](double e, double mu) {
        const double x = std::min(700.0, std::max(-700.0, (e - mu) / sigma));
        return 1.0 / (1.0 + std::exp(x));
    };
    auto count = [&](double mu) {
        double c = 0.0;
        for (int k = 0; k < nk; ++k)
            for (int n = 0; n < nbands; ++n) c += 2.0 * wk[k] * fd(ev[(size_t)k * nbands + n], mu);
        return c;
    };
    double lo = *std::min_element(ev.begin(), ev.end()) - 40.0 * sigma;
    double hi = *std::max_element(ev.begin(), ev.end()) + 40.0 * sigma;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        (count(mid) < nelec ? lo : hi) = mid;
    }
    const double mu = 0.5 * (lo + hi);
    f.assign((size_t)nk * nbands, 0.0);
    for (int k = 0; k < nk; ++k)
        for (int n = 0; n < nbands; ++n) f[(size_t)k * nbands + n] = 2.0 * wk[k] * fd(ev[(size_t)k * nbands + n], mu);
    return mu;
}

// Ultrasoft strengths D = E + q int V g_a from the handle's current table
// (V_eff = V_H + V_xc + V_LOC), uploaded to both precisions' tables.
static int uspp_strengths(mb_handle *h, const ScfPlanes &pl, double2 *vg, double *atoms, double *out,
                          std::vector<double> &Ehost, cudaStream_t s) {
    const int na = (int)h->aug.size(), NN = h->n1 * h->n2;
    std::vector<double> ah(4 * (size_t)na), oh((size_t)na * h->nq);
    for (int a = 0; a < na; ++a) {
        ah[4 * a] = h->aug[a].x;
        ah[4 * a + 1] = h->aug[a].y;
        ah[4 * a + 2] = h->aug[a].z;
        ah[4 * a + 3] = h->aug[a].rQ;
    }
    MB_CUDA(cudaMemcpyAsync(atoms, ah.data(), sizeof(double) * ah.size(), cudaMemcpyHostToDevice, s));
    int rc = plane_fft2(h, false, h->d_vloc, nullptr, nullptr, vg, 1.0 / NN, s);
    if (rc) return rc;
    aug_integral_kernel<<<dim3(h->nq, na), 256, 0, s>>>(vg, atoms, pl.zq, pl.wq, h->nq, h->n1, h->n2, h->b1[0],
                                                         h->b1[1], h->b2[0], h->b2[1], h->Ac, out);
    MB_CUDA(cudaGetLastError());
    ++h->launches;
    MB_CUDA(cudaMemcpyAsync(oh.data(), out, sizeof(double) * oh.size(), cudaMemcpyDeviceToHost, s));
    MB_CUDA(cudaStreamSynchronize(s));
    Ehost.assign(h->Ekb.begin(), h->Ekb.end());
    Ehost.insert(Ehost.end(), h->Ecoup.begin(), h->Ecoup.end());
    for (int a = 0; a < na; ++a) {
        double I = 0.0;
        for (int q = 0; q < h->nq; ++q) I += oh[(size_t)a * h->nq + q];
        for (int p = h->aug[a].p0; p < h->aug[a].p0 + h->aug[a].np; ++p) {
            Ehost[p] += h->Qkb[p] * I;
            Ehost[h->nkb + p] += h->Qcoup[p] * I;
        }
    }
    std::vector<float> e32(Ehost.begin(), Ehost.end());
    MB_CUDA(cudaMemcpyAsync(h->t64.E, Ehost.data(), sizeof(double) * Ehost.size(), cudaMemcpyHostToDevice, s));
    MB_CUDA(cudaMemcpyAsync(h->t32.E, e32.data(), sizeof(float) * e32.size(), cudaMemcpyHostToDevice, s));
    MB_CUDA(cudaStreamSynchronize(s));   // e32 and Ehost are host buffers
    return MB_OK;
}

// Augmentation of the output density: rho += sum_a w_a g_a with
// w_a = sum_{k,n} f sum_pq q_pq conj(F_p) F_q, F_p = <beta_p|phi_n>.
static int uspp_augment(mb_handle *h, const void *evecs, int nbands, const std::vector<double> &f, double *rho,
                        double *aug, cudaStream_t s) {
    const int nk = (int)h->kp.size(), nkb = h->nkb, na = (int)h->aug.size();
    const size_t n = (size_t)h->nq * h->n1 * h->n2;
    std::vector<double> F((size_t)nk * nbands * nkb * 2);
    int rc = uspp_overlaps(h, evecs, nbands, F.data(), s);
    if (rc) return rc;
    std::vector<double> grp, ion;
    std::vector<int> start(1, 0);
    for (int a = 0; a < na; ++a) {
        double w = 0.0;
        for (int k = 0; k < nk; ++k)
            for (int b = 0; b < nbands; ++b) {
                const double fb = f[(size_t)k * nbands + b];
                if (fb == 0.0) continue;
                const double *Fk = F.data() + 2 * ((size_t)k * nbands + b) * nkb;
                for (int p = h->aug[a].p0; p < h->aug[a].p0 + h->aug[a].np; ++p) {
                    const double re = Fk[2 * p], im = Fk[2 * p + 1];
                    double t = h->Qkb[p] * (re * re + im * im);
                    const int q = h->partner[p];
                    if (q >= 0) t += h->Qcoup[p] * (re * Fk[2 * q] + im * Fk[2 * q + 1]);
                    w += fb * t;
                }
            }
        // one group per atom: the core-density profile of radius r_Q, weight w_a
        grp.insert(grp.end(), {1.0, h->aug[a].rQ, h->aug[a].z});
        ion.insert(ion.end(), {w, h->aug[a].x, h->aug[a].y});
        start.push_back(a + 1);
    }
    if ((rc = vloc_tabulate(h, 1, aug, s, &grp, &ion, &start))) return rc;
    add_kernel<<<grid_blocks(h, n), 256, 0, s>>>(rho, aug, nullptr, rho, n);
    MB_CUDA(cudaGetLastError());
    ++h->launches;
    return MB_OK;
}

}  // namespace mb

using namespace mb;

extern "C" {

int mb_density(mb_handle *h, const void *evecs, int nbands, const double *occ, double *rho, void *stream) {
    int rc = check_tables(h);
    if (rc) return rc;
    if (!evecs || !occ || !rho || nbands <= 0) return MB_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    MB_CUDA(cudaSetDevice(h->device));
    const size_t nocc = h->kp.size() * (size_t)nbands;
    Buf B{h, s};
    double *d_occ = B.get<double>(nocc);
    if (B.rc) return B.rc;
    MB_CUDA(cudaMemcpyAsync(d_occ, occ, sizeof(double) * nocc, cudaMemcpyHostToDevice, s));
    if ((rc = scf_density(h, evecs, nbands, d_occ, rho, s))) return rc;
    MB_CUDA(cudaStreamSynchronize(s));   // the host occupations are read by the copy above
    return MB_OK;
}

int mb_hartree(mb_handle *h, const double *rho, double *vh, void *stream) {
    int rc = check_tables(h);
    if (rc) return rc;
    if (!rho || !vh) return MB_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    MB_CUDA(cudaSetDevice(h->device));
    Buf B{h, s};
    ScfPlanes pl;
    if ((rc = upload_planes(h, B, pl, s))) return rc;
    if ((rc = hartree(h, rho, vh, B, pl, s))) return rc;
    MB_CUDA(cudaStreamSynchronize(s));   // the plane tables come from host vectors
    return MB_OK;
}

int mb_xc_lda(mb_handle *h, const double *rho, double *vxc, double *exc, void *stream) {
    int rc = check_tables(h);
    if (rc) return rc;
    if (!rho || !vxc) return MB_EINVAL;
    MB_CUDA(cudaSetDevice(h->device));
    return xc(h, rho, vxc, exc, (cudaStream_t)stream);
}

int mb_scf(mb_handle *h, const mb_scf_opts *o, double *evals, double *rho_out, mb_scf_info *info) {
    using clk = std::chrono::steady_clock;
    const auto t_start = clk::now();
    int rc = check_tables(h);
    if (rc) return rc;
    if (!o || !evals || o->nbands <= 0 || !(o->sigma > 0.0) || !(o->tol > 0.0)) return MB_EINVAL;
    if (o->prec != MB_FP64 && o->prec != MB_FP32) return MB_EINVAL;
    const int nk = (int)h->kp.size(), nbands = o->nbands;
    const int depth = o->pulay_depth > 0 ? std::min(o->pulay_depth, kMaxPulay) : 4;
    const int max_iter = o->max_iter > 0 ? o->max_iter : 60;
    const double W = o->mix_weight > 0.0 ? o->mix_weight : 0.5;
    const double gmax = o->g_max > 0.0 ? o->g_max : 1.0;
    const double eig_tol = o->eig_tol > 0.0 ? o->eig_tol : 0.1 * o->tol;
    double nelec = o->nelec;
    if (!(nelec > 0.0)) {
        nelec = 0.0;
        for (size_t g = 0; g + 1 < h->lstart.size(); ++g)
            if (h->lgrp[3 * g] == 1.0)
                for (int i = h->lstart[g]; i < h->lstart[g + 1]; ++i) nelec += h->lion[3 * i];
    }
    if (!(nelec > 0.0) || nelec > 2.0 * nbands) return MB_EINVAL;
    // |g|^2 of the grid's first nonzero shell (the g = 0 profile's mixing factor)
    double g1sq = INFINITY;
    for (int u = 0; u < h->n1; ++u)
        for (int v = 0; v < h->n2; ++v) {
            const int m1 = u < h->n1 / 2 ? u : u - h->n1, m2 = v < h->n2 / 2 ? v : v - h->n2;
            const double gx = m1 * h->b1[0] + m2 * h->b2[0], gy = m1 * h->b1[1] + m2 * h->b2[1];
            const double g2 = gx * gx + gy * gy;
            if (g2 > 0.0) g1sq = std::min(g1sq, g2);
        }
    std::vector<double> wk(nk, 1.0 / nk);
    if (o->kweights) {
        double sw = 0.0;
        for (int k = 0; k < nk; ++k) sw += (wk[k] = o->kweights[k]);
        if (!(std::fabs(sw - 1.0) < 1e-9)) return MB_EINVAL;
    }
    MB_CUDA(cudaSetDevice(h->device));
    cudaStream_t s = nullptr;
    MB_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    };
    int result = MB_OK;
    mb_scf_info inf{};
    {
        StreamGuard sg{s};   // destroyed after B: the frees B queues on s run before s goes away
        Buf B{h, s};
        const int NN = h->n1 * h->n2;
        const size_t n = (size_t)h->nq * NN;
        size_t nvec = 0;
        for (int k = 0; k < nk; ++k) nvec += (size_t)nbands * h->nb * h->kp[k].ldg;
        double *vext = B.get<double>(n), *rho_in = B.get<double>(n), *rho_o = B.get<double>(n);
        double *vh = B.get<double>(n), *vx = B.get<double>(n), *vscf = B.get<double>(n), *vprev = B.get<double>(n);
        double *occ = B.get<double>((size_t)nk * nbands), *red = B.get<double>(h->nq);
        double2 *evecs = B.get<double2>(nvec), *cur_in = B.get<double2>(n), *cur_out = B.get<double2>(n);
        std::vector<double2 *> hin(depth), hres(depth);
        for (int i = 0; i < depth; ++i) {
            hin[i] = B.get<double2>(n);
            hres[i] = B.get<double2>(n);
        }
        // work fields, allocated once: two spectra (the Coulomb step and the
        // ultrasoft integrals), the augmentation density, the ultrasoft atoms
        double2 *wk1 = B.get<double2>(n), *wk2 = B.get<double2>(n);
        double *aug = h->uspp ? B.get<double>(n) : nullptr;
        const size_t na = h->aug.size();
        double *aug_atoms = h->uspp ? B.get<double>(4 * na) : nullptr;
        double *aug_out = h->uspp ? B.get<double>(na * h->nq) : nullptr;
        ScfPlanes pl;
        if (B.rc) return B.rc;
        if ((rc = upload_planes(h, B, pl, s))) return rc;
        // the atoms' table, and the start density: their Gaussian core charges
        MB_CUDA(cudaMemcpyAsync(vext, h->d_vloc, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        if ((rc = vloc_tabulate(h, 1, rho_in, s))) return rc;
        std::vector<double> ev((size_t)nk * nbands), f, red_h(h->nq), Ahist((size_t)depth * depth, 0.0), Ehost;
        int nh = 0, head = 0;   // history entries and the slot the next one goes to
        double dv = INFINITY, mu = 0.0, t_eig = 0.0, t_dens = 0.0, t_pot = 0.0;
        int it = 0, cycles = 0;
        for (it = 1; it <= max_iter; ++it) {
            auto t0 = clk::now();
            // V_scf of the input density, its change, and the apply tables
            if ((rc = hartree(h, rho_in, vh, B, pl, s, wk1, wk2)) || (rc = xc(h, rho_in, vx, nullptr, s))) {
                result = rc;
                break;
            }
            add_kernel<<<grid_blocks(h, n), 256, 0, s>>>(vh, vx, nullptr, vscf, n);
            if (it > 1) {
                plane_reduce_kernel<true><<<h->nq, 256, 0, s>>>(vscf, vprev, nullptr, NN, red);
                MB_CUDA(cudaMemcpyAsync(red_h.data(), red, sizeof(double) * h->nq, cudaMemcpyDeviceToHost, s));
            }
            MB_CUDA(cudaMemcpyAsync(vprev, vscf, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
            add_kernel<<<grid_blocks(h, n), 256, 0, s>>>(vext, vscf, nullptr, h->d_vloc, n);
            MB_CUDA(cudaGetLastError());
            h->launches += it > 1 ? 3 : 2;
            MB_CUDA(cudaStreamSynchronize(s));
            if (it > 1) dv = *std::max_element(red_h.begin(), red_h.end());
            if ((rc = vloc_derive_tables(h))) {
                result = rc;
                break;
            }
            if (h->uspp && (rc = uspp_strengths(h, pl, wk1, aug_atoms, aug_out, Ehost, s))) {
                result = rc;
                break;
            }
            auto t1 = clk::now();
            t_pot += std::chrono::duration<double>(t1 - t0).count();
            mb_solve_info si{};
            mb_solve_opts so{};
            so.warm_start = it > 1;          // from the roots of the previous potential
            // while the potential still moves by dv, roots more accurate than
            // about dv / 10 buy nothing: the tolerance follows dv down to
            // eig_tol (reached once dv < tol, so the final roots are exact to it)
            const double tol_it = std::min(std::max(eig_tol, 1e-3), std::max(eig_tol, 0.1 * dv));
            rc = mb_eigsolve(h, nbands, tol_it, o->prec, ev.data(), evecs, &so, &si, s);
            cycles += si.cycles;
            auto t2 = clk::now();
            t_eig += std::chrono::duration<double>(t2 - t1).count();
            if (rc != MB_OK && rc != MB_ENOTCONV) {
                result = rc;
                break;
            }
            if (dv < o->tol) break;
            // output density and the mixed next input
            mu = occupations(ev, wk, nbands, nelec, o->sigma, f);
            MB_CUDA(cudaMemcpyAsync(occ, f.data(), sizeof(double) * f.size(), cudaMemcpyHostToDevice, s));
            if ((rc = scf_density(h, evecs, nbands, occ, rho_o, s))) {
                result = rc;
                break;
            }
            if (h->uspp && (rc = uspp_augment(h, evecs, nbands, f, rho_o, aug, s))) {
                result = rc;
                break;
            }
            MB_CUDA(cudaStreamSynchronize(s));   // f is reused on the host
            auto t3 = clk::now();
            t_dens += std::chrono::duration<double>(t3 - t2).count();
            const double sc = 1.0 / NN;
            if ((rc = plane_fft2(h, false, rho_in, nullptr, nullptr, hin[head], sc, s)) ||
                (rc = plane_fft2(h, false, rho_o, nullptr, nullptr, cur_out, sc, s))) {
                result = rc;
                break;
            }
            csub_kernel<<<grid_blocks(h, n), 256, 0, s>>>(cur_out, hin[head], hres[head], n);
            ++h->launches;
            nh = std::min(nh + 1, depth);
            // Gram row of the new residual against the history (slots in age order)
            std::vector<int> order(nh);
            for (int i = 0; i < nh; ++i) order[i] = (head - (nh - 1) + i + depth) % depth;
            for (int i = 0; i < nh; ++i) {
                plane_reduce_kernel<false><<<h->nq, 256, 0, s>>>(hres[order[i]], hres[head], pl.wq, NN, red);
                ++h->launches;
                MB_CUDA(cudaMemcpyAsync(red_h.data(), red, sizeof(double) * h->nq, cudaMemcpyDeviceToHost, s));
                MB_CUDA(cudaStreamSynchronize(s));
                double d = 0.0;
                for (int q = 0; q < h->nq; ++q) d += red_h[q];
                Ahist[(size_t)order[i] * depth + head] = Ahist[(size_t)head * depth + order[i]] = d;
            }
            std::vector<double> A((size_t)nh * nh), a;
            int m = nh;
            for (;;) {
                const int first = nh - m;   // drop the oldest entries while the system is singular
                for (int i = 0; i < m; ++i)
                    for (int j = 0; j < m; ++j)
                        A[(size_t)i * m + j] = Ahist[(size_t)order[first + i] * depth + order[first + j]];
                if (pulay_solve(A, m, a)) break;
                if (--m == 0) {
                    m = 1;
                    a.assign(1, 1.0);
                    break;
                }
            }
            MixArgs ma;
            ma.m = m;
            for (int i = 0; i < m; ++i) {
                ma.rin[i] = hin[order[nh - m + i]];
                ma.res[i] = hres[order[nh - m + i]];
                ma.a[i] = a[i];
            }
            ma.N1 = h->n1;
            ma.N2 = h->n2;
            ma.NN = NN;
            ma.b1x = h->b1[0];
            ma.b1y = h->b1[1];
            ma.b2x = h->b2[0];
            ma.b2y = h->b2[1];
            ma.W = W;
            ma.gmax2 = gmax * gmax;
            ma.K0 = W * g1sq / (g1sq + gmax * gmax);
            mix_combine_kernel<<<grid_blocks(h, n), 256, 0, s>>>(ma, cur_in, n);
            MB_CUDA(cudaGetLastError());
            ++h->launches;
            if ((rc = plane_fft2(h, true, nullptr, cur_in, rho_in, nullptr, 1.0, s))) {
                result = rc;
                break;
            }
            head = (head + 1) % depth;
        }
        if (result == MB_OK) {
            std::memcpy(evals, ev.data(), sizeof(double) * ev.size());
            if (rho_out) MB_CUDA(cudaMemcpyAsync(rho_out, rho_in, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
            // electrons in the final input density
            std::vector<double> rh(n);
            MB_CUDA(cudaMemcpyAsync(rh.data(), rho_in, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
            MB_CUDA(cudaStreamSynchronize(s));
            double ne = 0.0;
            for (int q = 0; q < h->nq; ++q) {
                double sq = 0.0;
                for (int e = 0; e < NN; ++e) sq += rh[(size_t)q * NN + e];
                ne += h->wq[q] * sq;
            }
            inf.nelec = ne * h->Ac / NN;
        }
        inf.iterations = std::min(it, max_iter);
        inf.dv = dv;
        inf.mu = mu;
        inf.eig_cycles = cycles;
        inf.seconds_eig = t_eig;
        inf.seconds_density = t_dens;
        inf.seconds_potential = t_pot;
        if (result == MB_OK && !(dv < o->tol)) result = MB_ENOTCONV;
    }
    inf.seconds = std::chrono::duration<double>(clk::now() - t_start).count();
    if (info) *info = inf;
    return result;
}

}  // extern "C"
