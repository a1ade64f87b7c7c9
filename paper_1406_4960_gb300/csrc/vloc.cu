// The local potential V(r, z_q) on the quadrature planes, built on the device
// from the analytic in-plane components of the atoms' local pseudopotentials
// (§II.B.1, Eq. (10)):
//   Gaussian term A exp(-a r^2) (Eq. (13)):
//       (A / A_c)(pi / a) exp(-g^2 / 4a) exp(-a dz^2)
//   core term -Z erf(r / R_c) / r: the Coulomb potential of the Gaussian core
//   charge through the 2D transform of 1/r (the Coulomb integral of §II.B.1),
//   in closed form
//       -(Z / A_c)(pi / g) [T(dz) + T(-dz)],  T(z) = exp(g z) erfc(g R_c / 2 + z / R_c),
//   written exp(-g^2 R_c^2 / 4 - z^2 / R_c^2) erfcx(x) where the erfc argument
//   x is >= 0; at g = 0 the divergent constant (2 pi / g)(Z / A_c) is dropped
//   and +(2 pi Z / A_c)[dz erf(dz / R_c) + (R_c / sqrt(pi)) exp(-dz^2 / R_c^2)]
//   kept,
// each times exp(-i g . R_par), summed over the grid frequencies g_m
// (m in [-N/2, N/2) per axis) into the real table
//   V(r, z_q) = Re sum_m c(m, z_q) exp(i g_m . r),  r = (i1/N1) a1 + (i2/N2) a2.
//
// Atoms that share a profile (kind, width, height) share its z dependence,
// so their phases are summed once into a structure factor per group
// (vloc_sfac_kernel).  Per plane the components are the groups' profiles
// times their structure factors, summed along m2 (vloc_rows_kernel) and then
// along m1, keeping the real part (vloc_cols_kernel): plain O(N) sums per
// output with N <= 256, in FP64, twiddles from sincospi of exact ratios.
// The tables the apply kernels read (weight and 1/(N1 N2) folded in,
// bit-reversed, per column, FP32 copies) are derived from the natural table
// by vloc_tables_kernel, which also serves a table set by the caller.
#include <algorithm>
#include <vector>

#include "mb_internal.h"

namespace mb {

namespace {

constexpr double kPiD = 3.14159265358979323846;
constexpr double kInvSqrtPi = 0.56418958354775628695;
constexpr size_t kVlocChunkBytes = 64ull << 20;   // planes per pass of the two-step transform

struct VlocGeom {
    int N1, N2, nq, ngrp;
    double b1x, b1y, b2x, b2y, Ac;
};

__device__ __forceinline__ void grid_g(const VlocGeom &G, int u, int v, double &gx, double &gy) {
    const int m1 = u < G.N1 / 2 ? u : u - G.N1, m2 = v < G.N2 / 2 ? v : v - G.N2;
    gx = m1 * G.b1x + m2 * G.b2x;
    gy = m1 * G.b1y + m2 * G.b2y;
}

// z profile of one group at |g| and height dz above the group's atoms, per
// unit weight (A of a Gaussian, Z of a core term) and per unit cell area.
// mode 0: the potential; mode 1: the core charge density
// rho_c = Z exp(-r^2/R_c^2) / (pi^(3/2) R_c^3), whose components are
// exp(-g^2 R_c^2/4) exp(-dz^2/R_c^2) / (sqrt(pi) R_c A_c) (Gaussians: none).
__device__ double profile(int mode, int kind, double p, double g, double dz, double Ac) {
    if (mode == 1) {
        if (kind != 1) return 0.0;
        const double u = dz / p;
        return kInvSqrtPi / (p * Ac) * exp(-0.25 * (g * p) * (g * p) - u * u);
    }
    if (kind == 0) {   // Gaussian, p = a
        return (kPiD / p) / Ac * exp(-g * g / (4.0 * p)) * exp(-p * dz * dz);
    }
    const double Rc = p;   // core term
    if (g == 0.0) {
        const double u = dz / Rc;
        return (2.0 * kPiD / Ac) * (dz * erf(u) + Rc * kInvSqrtPi * exp(-u * u));
    }
    double t = 0.0;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const double z = s ? -dz : dz;
        const double x = 0.5 * g * Rc + z / Rc;
        t += x >= 0.0 ? exp(-0.25 * (g * Rc) * (g * Rc) - (z / Rc) * (z / Rc)) * erfcx(x) : exp(g * z) * erfc(x);
    }
    return -(kPiD / g) / Ac * t;
}

// S[grp][u N2 + v] = sum_{atoms of grp} weight exp(-i g_m . R_par)
__global__ void vloc_sfac_kernel(VlocGeom G, const double *ion, const int *start, double2 *S) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x, grp = blockIdx.y;
    const int NN = G.N1 * G.N2;
    if (e >= NN) return;
    double gx, gy;
    grid_g(G, e / G.N2, e % G.N2, gx, gy);
    double re = 0.0, im = 0.0;
    for (int i = start[grp]; i < start[grp + 1]; ++i) {
        double sn, cs;
        sincos(-(gx * ion[3 * i + 1] + gy * ion[3 * i + 2]), &sn, &cs);
        re += ion[3 * i] * cs;
        im += ion[3 * i] * sn;
    }
    S[(size_t)grp * NN + e] = make_double2(re, im);
}

// One (row u, plane q) per threadIdx.y slice: c(m, z_q) for the N2
// frequencies of the row, then tmp[q][u][i2] = sum_v c(u, v) exp(2 pi i v i2 / N2).
// blockDim = (N2, planes per block).
__global__ void vloc_rows_kernel(VlocGeom G, int mode, const double *grp, const double2 *S, const double *zq, int q0,
                                 int nqc, double2 *tmp) {
    extern __shared__ double2 rs[];
    double2 *tw = rs, *c = rs + G.N2 + threadIdx.y * G.N2;
    const int u = blockIdx.x, qq = blockIdx.y * blockDim.y + threadIdx.y, v = threadIdx.x, NN = G.N1 * G.N2;
    if (threadIdx.y == 0) {
        double sn, cs;
        sincospi(2.0 * v / G.N2, &sn, &cs);
        tw[v] = make_double2(cs, sn);
    }
    const bool live = qq < nqc;
    if (live) {
        double gx, gy;
        grid_g(G, u, v, gx, gy);
        const double g = sqrt(gx * gx + gy * gy), z = zq[q0 + qq];
        double re = 0.0, im = 0.0;
        for (int k = 0; k < G.ngrp; ++k) {
            const double f = profile(mode, (int)grp[3 * k], grp[3 * k + 1], g, z - grp[3 * k + 2], G.Ac);
            const double2 s = S[(size_t)k * NN + u * G.N2 + v];
            re += f * s.x;
            im += f * s.y;
        }
        c[v] = make_double2(re, im);
    }
    __syncthreads();
    if (!live) return;
    double sr = 0.0, si = 0.0;
    for (int w = 0; w < G.N2; ++w) {
        const double2 a = c[w], t = tw[(w * v) & (G.N2 - 1)];
        sr += a.x * t.x - a.y * t.y;
        si += a.x * t.y + a.y * t.x;
    }
    tmp[((size_t)qq * G.N1 + u) * G.N2 + v] = make_double2(sr, si);
}

// One (column i2, plane q) per threadIdx.y slice:
// V[q][i1][i2] = Re sum_u tmp[q][u][i2] exp(2 pi i u i1 / N1).  blockDim = (N1, planes per block).
__global__ void vloc_cols_kernel(VlocGeom G, const double2 *tmp, int q0, int nqc, double *V) {
    extern __shared__ double2 cs_[];
    double2 *tw = cs_, *col = cs_ + G.N1 + threadIdx.y * G.N1;
    const int i2 = blockIdx.x, qq = blockIdx.y * blockDim.y + threadIdx.y, i1 = threadIdx.x;
    const bool live = qq < nqc;
    if (live) col[i1] = tmp[((size_t)qq * G.N1 + i1) * G.N2 + i2];
    if (threadIdx.y == 0) {
        double sn, cs;
        sincospi(2.0 * i1 / G.N1, &sn, &cs);
        tw[i1] = make_double2(cs, sn);
    }
    __syncthreads();
    if (!live) return;
    double s = 0.0;
    for (int u = 0; u < G.N1; ++u) {
        const double2 a = col[u], t = tw[(u * i1) & (G.N1 - 1)];
        s += a.x * t.x - a.y * t.y;
    }
    V[((size_t)(q0 + qq) * G.N1 + i1) * G.N2 + i2] = s;
}

// The apply kernels' tables from the natural table V (nq x N1 x N2):
// val = (w_q / (N1 N2)) V; Vn natural, Vp bit-reversed on both axes, Vt
// per column (i1 fastest).
__global__ void vloc_tables_kernel(int nq, int N1, int N2, int l1, int l2, const double *V, const double *wq,
                                   double *Vn64, float *Vn32, double *Vp64, float *Vp32, float *Vt32) {
    const int NN = N1 * N2;
    const size_t total = (size_t)nq * NN;
    const double scale = 1.0 / NN;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int q = (int)(e / NN), r = (int)(e % NN), i1 = r / N2, i2 = r % N2;
        const double val = wq[q] * scale * V[e];
        Vn64[e] = val;
        Vn32[e] = (float)val;
        const int p1 = (int)(__brev((unsigned)i1) >> (32 - l1)), p2 = (int)(__brev((unsigned)i2) >> (32 - l2));
        const size_t pe = (size_t)q * NN + (size_t)p1 * N2 + p2;
        Vp64[pe] = val;
        Vp32[pe] = (float)val;
        Vt32[((size_t)q * N2 + i2) * N1 + i1] = (float)val;
    }
}

int pool_alloc(mb_handle *h, void **p, size_t bytes) {
    if (*p) return MB_OK;
    cudaMemPool_t pool = mb_pool(h->device);
    if (!pool) return MB_ECUDA;
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, h->hs);
    return e == cudaSuccess ? MB_OK : cuda_fail(h, e);
}

}  // namespace

size_t vloc_build_scratch_bytes(const mb_handle *h) {
    const size_t NN = (size_t)h->n1 * h->n2;
    const size_t ngrp = h->lstart.empty() ? 0 : h->lstart.size() - 1;
    const size_t per_plane = NN * sizeof(double2);
    const size_t qc = std::max<size_t>(1, std::min<size_t>(h->nq, kVlocChunkBytes / per_plane));
    return qc * per_plane + ngrp * NN * sizeof(double2) + (h->lion.size() + h->lgrp.size()) * sizeof(double) +
           h->lstart.size() * sizeof(int) + 2 * (size_t)h->nq * sizeof(double);
}

// The natural table d_vloc -> every table of t64 / t32 the apply kernels read.
int vloc_derive_tables(mb_handle *h) {
    const size_t NN = (size_t)h->n1 * h->n2, n = (size_t)h->nq * NN;
    int rc;
    if ((rc = pool_alloc(h, &h->t64.Vn, n * sizeof(double)))) return rc;
    if ((rc = pool_alloc(h, &h->t32.Vn, n * sizeof(float)))) return rc;
    if ((rc = pool_alloc(h, &h->t64.V, n * sizeof(double)))) return rc;
    if ((rc = pool_alloc(h, &h->t32.V, n * sizeof(float)))) return rc;
    if ((rc = pool_alloc(h, &h->t32.Vt, n * sizeof(float)))) return rc;
    double *wq = nullptr;
    if ((rc = dev_upload(h, (void **)&wq, h->wq.data(), h->wq.size() * sizeof(double)))) return rc;
    const int blocks = (int)std::min<size_t>((n + 255) / 256, (size_t)h->num_sms * 8);
    vloc_tables_kernel<<<blocks, 256, 0, h->hs>>>(h->nq, h->n1, h->n2, h->l1, h->l2, h->d_vloc, wq,
                                                 (double *)h->t64.Vn, (float *)h->t32.Vn, (double *)h->t64.V,
                                                 (float *)h->t32.V, (float *)h->t32.Vt);
    cudaError_t e = cudaGetLastError();
    dev_free(h, (void **)&wq);
    if (e != cudaSuccess) return cuda_fail(h, e);
    MB_CUDA(cudaStreamSynchronize(h->hs));
    return MB_OK;
}

// The real table of the atoms' analytic terms on the planes into out (nq x
// N1 x N2, device), on stream s: mode 0 the local potential V(r, z_q),
// mode 1 the Gaussian core charge density.
int vloc_tabulate(mb_handle *h, int mode, double *out, cudaStream_t s, const std::vector<double> *lgrp_in,
                  const std::vector<double> *lion_in, const std::vector<int> *lstart_in) {
    const std::vector<double> &lgrp = lgrp_in ? *lgrp_in : h->lgrp, &lion = lion_in ? *lion_in : h->lion;
    const std::vector<int> &lstart = lstart_in ? *lstart_in : h->lstart;
    const int N1 = h->n1, N2 = h->n2, NN = N1 * N2, nq = h->nq;
    const int ngrp = lstart.empty() ? 0 : (int)lstart.size() - 1;
    if (ngrp == 0) {
        MB_CUDA(cudaMemsetAsync(out, 0, (size_t)nq * NN * sizeof(double), s));
        return MB_OK;
    }
    VlocGeom G{N1, N2, nq, ngrp, h->b1[0], h->b1[1], h->b2[0], h->b2[1], h->Ac};
    const size_t per_plane = (size_t)NN * sizeof(double2);
    const int qc = (int)std::max<size_t>(1, std::min<size_t>(nq, kVlocChunkBytes / per_plane));
    cudaMemPool_t pool = mb_pool(h->device);
    if (!pool) return MB_ECUDA;
    // one pool block: ions | groups | planes | group starts (int) | S | tmp
    const size_t nion = lion.size(), ngv = lgrp.size();
    const size_t off_grp = nion * sizeof(double), off_zq = off_grp + ngv * sizeof(double);
    const size_t off_start = off_zq + (size_t)nq * sizeof(double);
    const size_t off_S = (off_start + lstart.size() * sizeof(int) + 255) / 256 * 256;
    const size_t off_tmp = off_S + (size_t)ngrp * per_plane, bytes = off_tmp + (size_t)qc * per_plane;
    unsigned char *blk = nullptr;
    MB_CUDA(cudaMallocFromPoolAsync((void **)&blk, bytes, pool, s));
    double *ion = reinterpret_cast<double *>(blk), *grp = reinterpret_cast<double *>(blk + off_grp);
    double *zq = reinterpret_cast<double *>(blk + off_zq);
    int *start = reinterpret_cast<int *>(blk + off_start);
    double2 *S = reinterpret_cast<double2 *>(blk + off_S), *tmp = reinterpret_cast<double2 *>(blk + off_tmp);
    cudaError_t e = cudaMemcpyAsync(ion, lion.data(), nion * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(grp, lgrp.data(), ngv * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(zq, h->zq.data(), nq * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(start, lstart.data(), lstart.size() * sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        vloc_sfac_kernel<<<dim3((NN + 255) / 256, ngrp), 256, 0, s>>>(G, ion, start, S);
        // planes per block: blocks of about 256 threads
        const int pr = std::max(1, 256 / N2), pc = std::max(1, 256 / N1);
        for (int q0 = 0; q0 < nq; q0 += qc) {
            const int n = std::min(qc, nq - q0);
            vloc_rows_kernel<<<dim3(N1, (n + pr - 1) / pr), dim3(N2, pr), (size_t)(1 + pr) * N2 * sizeof(double2), s>>>(
                G, mode, grp, S, zq, q0, n, tmp);
            vloc_cols_kernel<<<dim3(N2, (n + pc - 1) / pc), dim3(N1, pc), (size_t)(1 + pc) * N1 * sizeof(double2), s>>>(
                G, tmp, q0, n, out);
        }
        e = cudaGetLastError();
    }
    cudaFreeAsync(blk, s);
    if (e != cudaSuccess) return cuda_fail(h, e);
    // the host vectors copied above must stay untouched until the copies ran
    MB_CUDA(cudaStreamSynchronize(s));
    return MB_OK;
}

// V(r, z_q) from the atoms' analytic terms into d_vloc, then the derived tables.
int vloc_build(mb_handle *h) {
    int rc;
    if ((rc = pool_alloc(h, (void **)&h->d_vloc, (size_t)h->nq * h->n1 * h->n2 * sizeof(double)))) return rc;
    if ((rc = vloc_tabulate(h, 0, h->d_vloc, h->hs))) return rc;
    return vloc_derive_tables(h);
}

}  // namespace mb
