// Generalized Lanczos-Krylov eigensolver (§II.C) on the device.
//
// Per k-point the solver keeps M roots X with HX and SX, and runs two
// alternating grand cycles:
//   A  Rayleigh-Ritz on [X | K_A], K_A the Krylov space of the root with the
//      largest residual;
//   B  roots split into blocks of b; each block does Rayleigh-Ritz on
//      [X_b | K_b] and keeps the b Ritz pairs of maximum overlap with its
//      inputs (plus any new lower root).
// after which X is S-orthonormalized and rotated to Ritz vectors in one
// Cholesky-QR + Rayleigh-Ritz step.  Krylov vectors come from
// A = P (H - theta S), P the banded per-G solve (T(G) + c S)^-1,
// S-orthogonalized by classical Gram-Schmidt applied twice.  Every step runs
// for all k-points in one launch; from the second cycle of each phase a
// grand cycle is one CUDA graph launch.
//
// Precision.  MB_FP64: everything in FP64.  Mixed (MB_FP32 / MB_BF16): bulk
// cycles on FP32 vectors only (FP32 applies in place on the chain slots,
// Gram products on the tensor cores with a TF32 hi + lo split, FP32 S
// products, preconditioner solves, rotations, residuals, Cholesky and
// Jacobi); then finish cycles with FP64 roots: FP64 applies of the roots,
// FP64 Grams, Cholesky and Jacobi (FP32 sweeps first), and the root
// rotations in float-float arithmetic, while the chains stay FP32.  The FP64
// residual is the convergence test.
#include <algorithm>
#include <chrono>
#include <tuple>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "cplx.cuh"
#include "mb_internal.h"
#include "tc_gemm.cuh"

namespace mb {

constexpr int LD = 128;       // leading dimension of subspace matrices
constexpr int JMAX = 112;     // largest subspace the Jacobi kernel holds (matrix in shared memory)
constexpr int JPAIRS = 58;    // rotation slots per Jacobi round (>= JMAX/2 + 1, even so that
                              // 5*JPAIRS doubles keep the next double2 array 16-byte aligned)

struct EigK {
    double2 *base;            // FP64 vectors of this k-point, stride nvec
    float2 *stage;            // FP32 staging for mixed-precision applies
    float2 *v32;              // FP32 copies for the Krylov Gram-Schmidt (mixed precision)
    const double *pfac;       // preconditioner factors of this k-point
    const float *pfac32;      // the same in FP32 (the mixed-precision Krylov chains)
    long long nvec;           // nb * ldg
    int ldg, ng;
};

// vector index sets: i < c1 -> s1 + ch*cs1 + i*st1;  else s2 + ch*cs2 + (i - c1)*st2
// (st = 1: a contiguous run; st = nc: one slot of every chain, the layout of
// the FP32 Krylov chains, whose slot i of all chains is contiguous)
struct VSet {
    int s1, c1, cs1, s2, c2, cs2, st1, st2;
    __host__ __device__ int count() const { return c1 + c2; }
    __host__ __device__ int at(int i, int ch) const {
        return i < c1 ? s1 + ch * cs1 + i * st1 : s2 + ch * cs2 + (i - c1) * st2;
    }
};
static VSet vs(int s1, int c1, int cs1 = 0, int s2 = 0, int c2 = 0, int cs2 = 0, int st1 = 1, int st2 = 1) {
    VSet v;
    v.s1 = s1; v.c1 = c1; v.cs1 = cs1; v.s2 = s2; v.c2 = c2; v.cs2 = cs2; v.st1 = st1; v.st2 = st2;
    return v;
}

// ---------------------------------------------------------------------------
// Fixed-order reduction of per-chunk partial Gram products (deterministic):
// one warp per output, lane l sums chunks l, l+32, ... and a fixed shuffle
// tree combines the lanes.  lower: only entries j <= i were computed (a
// Hermitian product); the upper triangle is written as the conjugate of the
// lower one.  Grid: (outputs / 8, problems), 256 threads.
__global__ void gram_reduce_kernel(const double2 *part, int nsplit, int ma, int mb, double2 *G, int lower) {
    const int prob = blockIdx.y;
    const int nout = ma * mb;
    const int o = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (o >= nout) return;                        // whole warp leaves together
    int i = o / mb, j = o % mb;
    const bool up = lower && j > i;
    const int src = up ? j * mb + i : o;
    const double2 *p = part + (size_t)prob * nsplit * nout + src;
    double2 s = make_double2(0.0, 0.0);
    for (int sp = lane; sp < nsplit; sp += 32) s = s + p[(size_t)sp * nout];
    for (int off = 16; off > 0; off >>= 1) {
        s.x += __shfl_down_sync(0xffffffffu, s.x, off);
        s.y += __shfl_down_sync(0xffffffffu, s.y, off);
    }
    if (lane == 0) {
        if (up) s.y = -s.y;
        G[(size_t)prob * LD * LD + i * LD + j] = s;
    }
}

// dst_i = src_i for index sets (FP64 -> FP64), or into / out of the FP32 stage
__global__ void copy_kernel(const EigK *ks, int nch, VSet S, VSet D, int mode) {
    // grid: (blocks along the vector, vector of the set, problem)
    // mode 0: base -> base; 1: base -> stage (to float); 2: stage -> base (to double);
    // 3: base -> v32 (to float); 4: v32 -> base (to double); 5: v32 -> v32
    const int prob = blockIdx.z, i = blockIdx.y;
    const int k = prob / nch, ch = prob % nch;
    const EigK d = ks[k];
    if (i >= S.count()) return;
    const long long sb = (long long)S.at(i, ch) * d.nvec, db = (long long)D.at(i, ch) * d.nvec;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < d.nvec;
         t += (long long)gridDim.x * blockDim.x) {
        const long long si = sb + t, di = db + t;
        if (mode == 0) d.base[di] = d.base[si];
        else if (mode == 1) d.stage[di] = make_float2((float)d.base[si].x, (float)d.base[si].y);
        else if (mode == 2) d.base[di] = make_double2((double)d.stage[si].x, (double)d.stage[si].y);
        else if (mode == 3) d.v32[di] = make_float2((float)d.base[si].x, (float)d.base[si].y);
        else if (mode == 4) d.base[di] = make_double2((double)d.v32[si].x, (double)d.v32[si].y);
        else d.v32[di] = d.v32[si];
    }
}

// W_ch = H_src - theta_ch S_src   (per-(k, ch) source indices); to32: W goes
// to the FP32 Gram-Schmidt copies (slot dst + ch of v32) instead
__global__ void krylov_residual_kernel(const EigK *ks, int nch, const int *srcH, const int *srcS,
                                       const double *theta, int dst, int to32) {
    const int prob = blockIdx.y;
    const int k = prob / nch, ch = prob % nch;
    const EigK d = ks[k];
    const double th = theta[prob];
    const double2 *h = d.base + (long long)srcH[prob] * d.nvec;
    const double2 *s = d.base + (long long)srcS[prob] * d.nvec;
    double2 *w = d.base + (long long)(dst + ch) * d.nvec;
    float2 *w32 = to32 ? d.v32 + (long long)(dst + ch) * d.nvec : nullptr;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < d.nvec;
         t += (long long)gridDim.x * blockDim.x) {
        const double2 r = h[t] - rscale(th, s[t]);
        if (to32) w32[t] = make_float2((float)r.x, (float)r.y);
        else w[t] = r;
    }
}

// Bulk cycles of the mixed solver, on the FP32 copies (v32):
// W_ch = HX_seed - theta SX_seed (slot 0) or HK_{slot-1} - theta SK_{slot-1}
// of chain ch, the chains' slot s of chain ch at base + s*nc + ch
__global__ void krylov_residual32_kernel(const EigK *ks, int nch, int slot, const int *seed, const double *theta,
                                         int oHX, int oSX, int oHK, int oSK, int nc, int dst) {
    const int prob = blockIdx.y;
    const int k = prob / nch, ch = prob % nch;
    const EigK d = ks[k];
    __shared__ float th_s;
    if (threadIdx.x == 0) th_s = (float)theta[prob];
    __syncthreads();
    const float th = th_s;
    const int ih = slot == 0 ? oHX + seed[prob] : oHK + (slot - 1) * nc + ch;
    const int is = slot == 0 ? oSX + seed[prob] : oSK + (slot - 1) * nc + ch;
    const float2 *h = d.v32 + (long long)ih * d.nvec;
    const float2 *s = d.v32 + (long long)is * d.nvec;
    float2 *w = d.v32 + (long long)(dst + ch) * d.nvec;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < d.nvec;
         t += (long long)gridDim.x * blockDim.x) {
        const float2 hv = h[t], sv = s[t];
        w[t] = make_float2(fmaf(-th, sv.x, hv.x), fmaf(-th, sv.y, hv.y));
    }
}

// R_i = HX_i - eps_i SX_i on the FP32 copies
__global__ void residual32_kernel(const EigK *ks, int M, int oHX, int oSX, int dst, const double *eps) {
    const int k = blockIdx.y;
    const EigK d = ks[k];
    const long long total = (long long)M * d.nvec;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / d.nvec);
        const long long t = e - (long long)i * d.nvec;
        const float ev = (float)eps[k * M + i];
        const float2 hv = d.v32[(long long)(oHX + i) * d.nvec + t], sv = d.v32[(long long)(oSX + i) * d.nvec + t];
        d.v32[(long long)(dst + i) * d.nvec + t] = make_float2(fmaf(-ev, sv.x, hv.x), fmaf(-ev, sv.y, hv.y));
    }
}

// R_i = HX_i - eps_i SX_i into dst
__global__ void residual_kernel(const EigK *ks, int M, int oX, int oHX, int oSX, int dst, const double *eps) {
    const int k = blockIdx.y;
    const EigK d = ks[k];
    const long long total = (long long)M * d.nvec;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int i = (int)(e / d.nvec);
        long long t = e - (long long)i * d.nvec;
        double ev = eps[k * M + i];
        d.base[(long long)(dst + i) * d.nvec + t] =
            d.base[(long long)(oHX + i) * d.nvec + t] - rscale(ev, d.base[(long long)(oSX + i) * d.nvec + t]);
    }
    (void)oX;
}

// out[prob*m + i] = Re <A_i, B_i>   (block reduction with warp shuffles)
// F32: on the FP32 copies, per-thread sums in FP32 and the rest in FP64
template <bool F32>
__global__ void coldot_kernel(const EigK *ks, int nch, VSet A, VSet B, double *out) {
    typedef typename std::conditional<F32, float2, double2>::type T2;
    typedef typename std::conditional<F32, float, double>::type T;
    const int i = blockIdx.x, prob = blockIdx.y;
    const int k = prob / nch, ch = prob % nch;
    const EigK d = ks[k];
    const T2 *vb = F32 ? reinterpret_cast<const T2 *>(d.v32) : reinterpret_cast<const T2 *>(d.base);
    const T2 *a = vb + (long long)A.at(i, ch) * d.nvec;
    const T2 *b = vb + (long long)B.at(i, ch) * d.nvec;
    T st = T(0);
    for (long long t = threadIdx.x; t < d.nvec; t += blockDim.x) st = fma(a[t].x, b[t].x, fma(a[t].y, b[t].y, st));
    double s = (double)st;
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    __shared__ double ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (threadIdx.x == 0) out[(size_t)prob * A.count() + i] = s;
    }
}

// new Krylov vector: K = W / ||W||_S, SK = SW / ||W||_S, HK slot cleared;
// a norm below the breakdown threshold marks the slot dead (zero vector).
__global__ void normalize_kernel(const EigK *ks, int nch, int oW, int oSW, int kV, int kS, int cs,
                                 int slot, const double *nrm2, int *alive, int kd, int k32, int sk32, int nc) {
    const int prob = blockIdx.y;
    const int k = prob / nch, ch = prob % nch;
    const EigK d = ks[k];
    __shared__ double inv_s;
    if (threadIdx.x == 0) {
        const double n2 = nrm2[prob];
        const bool ok = n2 > 1e-24;
        inv_s = ok ? 1.0 / sqrt(n2) : 0.0;
        if (blockIdx.x == 0) alive[prob * kd + slot] = ok ? 1 : 0;
    }
    __syncthreads();
    const double inv = inv_s;
    const double2 *w = d.base + (long long)(oW + ch) * d.nvec;
    const double2 *sw = d.base + (long long)(oSW + ch) * d.nvec;
    double2 *kv = d.base + (long long)(kV + ch * cs + slot) * d.nvec;
    double2 *ksv = d.base + (long long)(kS + ch * cs + slot) * d.nvec;
    // FP32 copies for later Gram-Schmidt steps (k32 < 0: none)
    float2 *kv32 = k32 >= 0 ? d.v32 + (long long)(k32 + slot * nc + ch) * d.nvec : nullptr;
    float2 *ks32 = k32 >= 0 ? d.v32 + (long long)(sk32 + slot * nc + ch) * d.nvec : nullptr;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < d.nvec;
         t += (long long)gridDim.x * blockDim.x) {
        const double2 a = rscale(inv, w[t]), b = rscale(inv, sw[t]);
        kv[t] = a;
        ksv[t] = b;
        if (kv32) {
            kv32[t] = make_float2((float)a.x, (float)a.y);
            ks32[t] = make_float2((float)b.x, (float)b.y);
        }
    }
}

// FP32 chain slot (bulk cycles): K[slot] = W / ||W||_S and SK[slot] (which
// holds S W) scaled in place; slot s of chain ch at base + s*nc + ch
__global__ void normalize32_kernel(const EigK *ks, int nch, int oW, int oK, int oSK, int nc, int slot,
                                   const double *nrm2, int *alive, int kd) {
    const int prob = blockIdx.y;
    const int k = prob / nch, ch = prob % nch;
    const EigK d = ks[k];
    // the scale once per block (FP64 square roots and divisions are slow)
    __shared__ float inv_s;
    if (threadIdx.x == 0) {
        const double n2 = nrm2[prob];
        const bool ok = n2 > 1e-24;
        inv_s = ok ? (float)(1.0 / sqrt(n2)) : 0.f;
        if (blockIdx.x == 0) alive[prob * kd + slot] = ok ? 1 : 0;
    }
    __syncthreads();
    const float inv = inv_s;
    const float2 *w = d.v32 + (long long)(oW + ch) * d.nvec;
    float2 *kv = d.v32 + (long long)(oK + slot * nc + ch) * d.nvec;
    float2 *sk = d.v32 + (long long)(oSK + slot * nc + ch) * d.nvec;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < d.nvec;
         t += (long long)gridDim.x * blockDim.x) {
        const float2 a = w[t], b = sk[t];
        kv[t] = make_float2(inv * a.x, inv * a.y);
        sk[t] = make_float2(inv * b.x, inv * b.y);
    }
}

// residual norms and seeds: res[k*M + i] = sqrt(max(0, dot)); seed = argmax over a range
__global__ void seed_kernel(const double *dots, int M, int mconv, int nk, int nch, int bsize, double *res,
                            const double *eps, int *seed, double *theta, int *srcH, int *srcS,
                            int oHX, int oSX) {
    const int prob = blockIdx.x * blockDim.x + threadIdx.x;
    if (prob >= nk * nch) return;
    const int k = prob / nch, ch = prob % nch;
    if (ch == 0)
        for (int i = 0; i < M; ++i) res[k * M + i] = sqrt(fmax(0.0, dots[k * M + i]));
    int lo = nch == 1 ? 0 : ch * bsize, hi = nch == 1 ? mconv : min(M, lo + bsize);
    int best = lo;
    double bv = -1.0;
    for (int i = lo; i < hi; ++i) {
        double v = sqrt(fmax(0.0, dots[k * M + i]));
        if (v > bv) { bv = v; best = i; }
    }
    seed[prob] = best;
    theta[prob] = eps[k * M + best];
    srcH[prob] = oHX + best;
    srcS[prob] = oSX + best;
}

// ---------------------------------------------------------------------------
// Jacobi diagonalization of one Hermitian m x m matrix per CTA (m <= JMAX),
// parallel (round-robin) ordering: m'/2 disjoint rotations per round.

// Per-round scratch of the sweeps (shared memory, sized for T = double).
struct JacobiScratch {
    unsigned char *rc;   // per pair: c, s, t*|apq|, app, aqq   (5 * JPAIRS T)
    unsigned char *re;   // per pair: phase e                     (JPAIRS T2)
    int *pp;             // per pair: p, q
    double *red;         // 32 partial sums
    int *stop;
};
constexpr int kJacobiThreads = 512;    // one CTA per problem
constexpr size_t kJacobiScratchBytes = 5 * JPAIRS * sizeof(double) + JPAIRS * sizeof(double2) + 2 * JPAIRS * sizeof(int);

// Sweeps until the off-diagonal Frobenius norm is <= rel_tol * sqrt(fro2).
// A (m x m, row-major) in shared memory; V is updated as V <- V J through
// vget/vset (shared or global memory).
template <typename T, typename VGet, typename VSet_>
__device__ void jacobi_sweeps(typename std::conditional<std::is_same<T, float>::value, float2, double2>::type *A,
                              int m, VGet vget, VSet_ vset, int max_sweeps, double rel_tol, double fro2,
                              JacobiScratch js) {
    typedef typename std::conditional<std::is_same<T, float>::value, float2, double2>::type T2;
    const T skip_rel = std::is_same<T, float>::value ? T(1e-7) : T(1e-15);
    T *rc = reinterpret_cast<T *>(js.rc);
    T2 *re = reinterpret_cast<T2 *>(js.re);
    int *pp = js.pp;
    const int mp = (m + 1) & ~1;      // players, padded to even
    const int npair = mp / 2;
    const int nblk2 = npair * (npair + 1) / 2;   // 2x2 blocks (I >= J) of the pair partition
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        for (int r = 0; r < mp - 1; ++r) {
            // rotation of every pair of the round (q >= m: an index left
            // alone this round, identity)
            for (int pi = threadIdx.x; pi < npair; pi += blockDim.x) {
                int a = pi == 0 ? 0 : ((r + pi - 1) % (mp - 1)) + 1;
                int b = ((r + mp - 1 - pi - 1) % (mp - 1)) + 1;
                if (pi == 0) b = ((r + mp - 2) % (mp - 1)) + 1;
                const int p = min(a, b), q = max(a, b);
                T c = 1, s = 0, tm = 0;
                T2 ep = mk(T(1), T(0));
                if (q < m) {
                    T2 apq = A[p * m + q];
                    T mag = hypot(apq.x, apq.y);
                    T app = A[p * m + p].x, aqq = A[q * m + q].x;
                    rc[5 * pi + 3] = app;
                    rc[5 * pi + 4] = aqq;
                    // rotations below rounding level of the diagonal are skipped
                    if (mag > skip_rel * sqrt(fabs(app * aqq)) && mag > T(1e-30)) {
                        ep = mk(apq.x / mag, apq.y / mag);
                        T th = (aqq - app) / (T(2) * mag);
                        T t = (th >= 0 ? T(1) : T(-1)) / (fabs(th) + sqrt(th * th + T(1)));
                        c = T(1) / sqrt(t * t + T(1));
                        s = t * c;
                        tm = t * mag;
                    }
                }
                pp[2 * pi] = p;
                pp[2 * pi + 1] = q;
                rc[5 * pi] = c;
                rc[5 * pi + 1] = s;
                rc[5 * pi + 2] = tm;
                re[pi] = ep;
            }
            __syncthreads();
            // A <- J^H A J by 2x2 blocks (rows of pair I, columns of pair J,
            // I >= J; the block above the diagonal is written as the
            // conjugate transpose), then V <- V J by (pair, row).
            // J = diag(1, e^-i phi) [[c, s], [-s, c]] on each pair's columns.
            for (int e = threadIdx.x; e < nblk2 + npair * m; e += blockDim.x) {
                if (e < nblk2) {
                    int I = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
                    while (I * (I + 1) / 2 > e) --I;
                    while ((I + 1) * (I + 2) / 2 <= e) ++I;
                    const int J = e - I * (I + 1) / 2;
                    const int pI = pp[2 * I], qI = pp[2 * I + 1], pJ = pp[2 * J], qJ = pp[2 * J + 1];
                    const bool vI = qI < m, vJ = qJ < m;
                    const T sI = rc[5 * I + 1], sJ = rc[5 * J + 1];
                    const bool actI = vI && sI != T(0), actJ = vJ && sJ != T(0);
                    T2 a00 = A[pI * m + pJ];
                    T2 a01 = vJ ? A[pI * m + qJ] : czero<T2>();
                    T2 a10 = vI ? A[qI * m + pJ] : czero<T2>();
                    T2 a11 = (vI && vJ) ? A[qI * m + qJ] : czero<T2>();
                    if (I == J && actI) {
                        a00 = mk(rc[5 * I + 3] - rc[5 * I + 2], T(0));
                        a11 = mk(rc[5 * I + 4] + rc[5 * I + 2], T(0));
                        a01 = a10 = czero<T2>();
                    } else {
                        if (actJ) {   // columns pJ, qJ
                            const T cJ = rc[5 * J];
                            const T2 ec = mk(re[J].x, -re[J].y);
                            T2 x = a00, y = cmul(ec, a01);
                            a00 = rscale(cJ, x) - rscale(sJ, y);
                            a01 = rscale(sJ, x) + rscale(cJ, y);
                            x = a10;
                            y = cmul(ec, a11);
                            a10 = rscale(cJ, x) - rscale(sJ, y);
                            a11 = rscale(sJ, x) + rscale(cJ, y);
                        }
                        if (actI) {   // rows pI, qI
                            const T cI = rc[5 * I];
                            T2 x = a00, y = cmul(re[I], a10);
                            a00 = rscale(cI, x) - rscale(sI, y);
                            a10 = rscale(sI, x) + rscale(cI, y);
                            x = a01;
                            y = cmul(re[I], a11);
                            a01 = rscale(cI, x) - rscale(sI, y);
                            a11 = rscale(sI, x) + rscale(cI, y);
                        }
                    }
                    A[pI * m + pJ] = a00;
                    if (vJ) A[pI * m + qJ] = a01;
                    if (vI) A[qI * m + pJ] = a10;
                    if (vI && vJ) A[qI * m + qJ] = a11;
                    if (I != J) {
                        A[pJ * m + pI] = mk(a00.x, -a00.y);
                        if (vJ) A[qJ * m + pI] = mk(a01.x, -a01.y);
                        if (vI) A[pJ * m + qI] = mk(a10.x, -a10.y);
                        if (vI && vJ) A[qJ * m + qI] = mk(a11.x, -a11.y);
                    }
                } else {
                    const int e2 = e - nblk2;
                    const int pi = e2 / m, row = e2 % m;
                    const int p = pp[2 * pi], q = pp[2 * pi + 1];
                    if (q >= m || rc[5 * pi + 1] == T(0)) continue;
                    const T c = rc[5 * pi], s = rc[5 * pi + 1];
                    const T2 ec = mk(re[pi].x, -re[pi].y);
                    T2 vp = vget(row, p), vq = cmul(ec, vget(row, q));
                    vset(row, p, rscale(c, vp) - rscale(s, vq));
                    vset(row, q, rscale(s, vp) + rscale(c, vq));
                }
            }
            __syncthreads();
        }
        // off-diagonal norm
        double o = 0.0;
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            int i = e / m, j = e % m;
            if (i != j) o += (double)A[e].x * A[e].x + (double)A[e].y * A[e].y;
        }
        for (int off = 16; off > 0; off >>= 1) o += __shfl_down_sync(0xffffffffu, o, off);
        if ((threadIdx.x & 31) == 0) js.red[threadIdx.x >> 5] = o;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += js.red[w];
            *js.stop = s <= rel_tol * rel_tol * fro2;
        }
        __syncthreads();
        if (*js.stop) break;
    }
}

// A (m x m) from the lower triangle of the problem's G (Hermitian
// completion: with the subspace ordered [roots | Krylov vectors], the
// coupling block comes from K^H (H X), which uses the roots' HX rather than
// the Krylov vectors' HK, which may come from a reduced-precision apply);
// dead slots become decoupled with a huge diagonal.  Returns the squared
// Frobenius norm of the live part (all threads).
template <typename T2>
__device__ double jacobi_load(const double2 *g, int m, const int *dead, int dead_stride, int dead_ofs, T2 *A,
                              double *red) {
    const int prob = blockIdx.x;
    double f = 0.0;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        int i = e / m, j = e % m;
        double2 v = i >= j ? g[i * LD + j] : g[j * LD + i];
        if (i < j) v.y = -v.y;
        if (i == j) v.y = 0.0;
        bool di = dead && dead[prob * dead_stride + i] == 0 && i >= dead_ofs;
        bool dj = dead && dead[prob * dead_stride + j] == 0 && j >= dead_ofs;
        if (di || dj) v = make_double2((i == j) ? 1e30 : 0.0, 0.0);
        else f += v.x * v.x + v.y * v.y;
        A[e] = mk((decltype(A[0].x))v.x, (decltype(A[0].x))v.y);
    }
    for (int off = 16; off > 0; off >>= 1) f += __shfl_down_sync(0xffffffffu, f, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = f;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        red[0] = s;
    }
    __syncthreads();
    const double fro2 = red[0];
    __syncthreads();
    return fro2;
}

// ascending order of the diagonal (selection sort by one thread)
template <typename T2>
__device__ void jacobi_sort(const T2 *A, int m, int *perm) {
    if (threadIdx.x == 0) {
        for (int i = 0; i < m; ++i) perm[i] = i;
        for (int i = 0; i < m; ++i) {
            int b = i;
            for (int j = i + 1; j < m; ++j)
                if (A[perm[j] * m + perm[j]].x < A[perm[b] * m + perm[b]].x) b = j;
            int t = perm[i]; perm[i] = perm[b]; perm[b] = t;
        }
    }
    __syncthreads();
}

// VS: the eigenvector matrix lives in shared memory beside A (m <= 84);
// otherwise it overwrites the input matrix G in global memory (m <= JMAX).
// T = float runs the rotations in FP32 (the mixed solver's bulk cycles).
template <bool VS, typename T>
__global__ void __launch_bounds__(kJacobiThreads) jacobi_kernel(double2 *G, int m, const int *dead, int dead_stride,
                                                     int dead_ofs, double *evals, double2 *evecs,
                                                     int max_sweeps, double rel_tol) {
    typedef typename std::conditional<std::is_same<T, float>::value, float2, double2>::type T2;
    extern __shared__ __align__(16) unsigned char sm[];
    const int prob = blockIdx.x;
    T2 *A = reinterpret_cast<T2 *>(sm);
    T2 *Vs = A + m * m;                                                  // eigenvectors in shared memory (VS)
    double2 *Vg = G + (size_t)prob * LD * LD;                            // or in place of G
    const int ldv = VS ? m : LD;
    unsigned char *scr = reinterpret_cast<unsigned char *>(A + (VS ? 2 : 1) * m * m);
    __shared__ double red[32];
    __shared__ int stop;
    __shared__ int perm[LD];
    JacobiScratch js{scr, scr + 5 * JPAIRS * sizeof(double), reinterpret_cast<int *>(scr + 5 * JPAIRS * sizeof(double) + JPAIRS * sizeof(double2)),
                     red, &stop};
    auto vget = [&](int r, int c) -> T2 {
        if (VS) return Vs[r * ldv + c];
        const double2 v = Vg[r * ldv + c];
        return mk((T)v.x, (T)v.y);
    };
    auto vset = [&](int r, int c, T2 v) {
        if (VS) Vs[r * ldv + c] = v;
        else Vg[r * ldv + c] = make_double2((double)v.x, (double)v.y);
    };
    const double fro2 = jacobi_load(G + (size_t)prob * LD * LD, m, dead, dead_stride, dead_ofs, A, red);
    // G is read completely (jacobi_load ends on a barrier) before V, possibly G itself, is initialised
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        int i = e / m, j = e % m;
        vset(i, j, mk(T(i == j ? 1 : 0), T(0)));
    }
    __syncthreads();
    jacobi_sweeps<T>(A, m, vget, vset, max_sweeps, rel_tol, fro2, js);
    jacobi_sort(A, m, perm);
    for (int c = threadIdx.x; c < m; c += blockDim.x) evals[(size_t)prob * LD + c] = A[perm[c] * m + perm[c]].x;
    double2 *out = evecs + (size_t)prob * LD * LD;
    if (!VS && out == Vg) {
        // eigenvectors already in place of G: permute their columns through
        // the (now free) shared matrix A, one row at a time
        for (int r = 0; r < m; ++r) {
            for (int c = threadIdx.x; c < m; c += blockDim.x) A[c] = vget(r, perm[c]);
            __syncthreads();
            for (int c = threadIdx.x; c < m; c += blockDim.x) out[r * LD + c] = make_double2(A[c].x, A[c].y);
            __syncthreads();
        }
    } else {
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            int r = e / m, c = e % m;
            const T2 v = vget(r, perm[c]);
            out[r * LD + c] = make_double2(v.x, v.y);
        }
    }
}

// FP64 result from FP32 sweeps (m <= JMIX_MAX): Jacobi in FP32 gives V0;
// B = V0^H A V0 is formed in FP64 (off-diagonal at the FP32 level), FP64
// sweeps on B converge in one or two (quadratic convergence), and the
// eigenvectors are V0 V1.  Same result as FP64 sweeps from the start, with
// most rotations at the FP32 rate.
constexpr int JMIX_MAX = 64;
__global__ void __launch_bounds__(kJacobiThreads) jacobi_mixed_kernel(const double2 *G, int m, const int *dead, int dead_stride,
                                                           int dead_ofs, double *evals, double2 *evecs,
                                                           int max_sweeps, double rel_tol) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int prob = blockIdx.x;
    double2 *A64 = reinterpret_cast<double2 *>(sm);
    double2 *W64 = A64 + m * m;
    float2 *A32 = reinterpret_cast<float2 *>(W64 + m * m);
    float2 *V32 = A32 + m * m;
    unsigned char *scr = reinterpret_cast<unsigned char *>(V32 + m * m);
    __shared__ double red[32];
    __shared__ int stop;
    __shared__ int perm[LD];
    JacobiScratch js{scr, scr + 5 * JPAIRS * sizeof(double), reinterpret_cast<int *>(scr + 5 * JPAIRS * sizeof(double) + JPAIRS * sizeof(double2)),
                     red, &stop};
    const double fro2 = jacobi_load(G + (size_t)prob * LD * LD, m, dead, dead_stride, dead_ofs, A64, red);
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int i = e / m, j = e % m;
        A32[e] = make_float2((float)A64[e].x, (float)A64[e].y);
        V32[e] = make_float2(i == j ? 1.f : 0.f, 0.f);
    }
    __syncthreads();
    auto v32get = [&](int r, int c) -> float2 { return V32[r * m + c]; };
    auto v32set = [&](int r, int c, float2 v) { V32[r * m + c] = v; };
    jacobi_sweeps<float>(A32, m, v32get, v32set, max_sweeps, 1e-6, fro2, js);
    // W = A V0, then A <- V0^H W  (FP64)
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int i = e / m, j = e % m;
        double2 s = make_double2(0.0, 0.0);
        for (int q = 0; q < m; ++q) {
            const float2 v = V32[q * m + j];
            cfma(s, A64[i * m + q], make_double2(v.x, v.y));
        }
        W64[e] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int i = e / m, j = e % m;
        double2 s = make_double2(0.0, 0.0);
        for (int q = 0; q < m; ++q) {
            const float2 v = V32[q * m + i];
            cfma(s, make_double2(v.x, -v.y), W64[q * m + j]);
        }
        A64[e] = s;
    }
    __syncthreads();
    // exact Hermitian symmetry and real diagonal before the FP64 sweeps
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int i = e / m, j = e % m;
        if (i > j) {
            const double2 lo = A64[e], up = A64[j * m + i];
            const double2 h = make_double2(0.5 * (lo.x + up.x), 0.5 * (lo.y - up.y));
            A64[e] = h;
            A64[j * m + i] = make_double2(h.x, -h.y);
        } else if (i == j) {
            A64[e].y = 0.0;
        }
        W64[e] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
    auto v64get = [&](int r, int c) -> double2 { return W64[r * m + c]; };
    auto v64set = [&](int r, int c, double2 v) { W64[r * m + c] = v; };
    jacobi_sweeps<double>(A64, m, v64get, v64set, max_sweeps, rel_tol, fro2, js);
    jacobi_sort(A64, m, perm);
    for (int c = threadIdx.x; c < m; c += blockDim.x) evals[(size_t)prob * LD + c] = A64[perm[c] * m + perm[c]].x;
    double2 *out = evecs + (size_t)prob * LD * LD;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int r = e / m, c = e % m, pc = perm[c];
        double2 s = make_double2(0.0, 0.0);
        for (int q = 0; q < m; ++q) {
            const float2 v = V32[r * m + q];
            cfma(s, make_double2(v.x, v.y), W64[q * m + pc]);
        }
        out[r * LD + c] = s;
    }
}

// U = L^{-H} with G = L L^H (G Hermitian positive definite, m <= JMAX).
// L lives in shared memory; U is written row by row to global memory.
// T = float: the arithmetic in FP32 (the bulk cycles' S-Grams, which are the
// identity up to the FP32 Gram-Schmidt error).
template <typename T>
__global__ void __launch_bounds__(128) cholinv_kernel(const double2 *G, int m, double2 *U, int *status) {
    typedef typename std::conditional<std::is_same<T, float>::value, float2, double2>::type T2;
    extern __shared__ __align__(16) unsigned char sm[];
    T2 *L = reinterpret_cast<T2 *>(sm);     // m x m, lower
    T *rdiag = reinterpret_cast<T *>(L + m * m);
    const int prob = blockIdx.x;
    const double2 *g = G + (size_t)prob * LD * LD;
    double2 *u = U + (size_t)prob * LD * LD;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        int i = e / m, j = e % m;
        const double2 v = i >= j ? g[i * LD + j] : make_double2(0.0, 0.0);
        L[e] = mk((T)v.x, (T)v.y);
    }
    __syncthreads();
    __shared__ T rpiv;
    for (int j = 0; j < m; ++j) {
        if (threadIdx.x == 0) {
            T d = L[j * m + j].x;
            if (!(d > T(0))) {
                status[prob] = 1;
                d = std::is_same<T, float>::value ? T(1e-30) : T(1e-300);
            }
            const T piv = sqrt(d);
            rpiv = T(1) / piv;
            L[j * m + j] = mk(piv, T(0));
        }
        __syncthreads();
        const T r = rpiv;
        for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) L[i * m + j] = rscale(r, L[i * m + j]);
        __syncthreads();
        // trailing update: L[i][c] -= L[i][j] conj(L[c][j]) for j < c <= i
        for (int e = threadIdx.x; e < (m - j - 1) * (m - j - 1); e += blockDim.x) {
            int i = j + 1 + e / (m - j - 1), c = j + 1 + e % (m - j - 1);
            if (c > i) continue;
            T2 lij = L[i * m + j], lcj = L[c * m + j];
            L[i * m + c] = L[i * m + c] - cmul_c(lij, lcj);
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) rdiag[i] = T(1) / L[i * m + i].x;
    __syncthreads();
    // column c of Z = L^{-1} by forward substitution (one thread per column);
    // U[c][i] = conj(Z[i][c]), and Z[q][c] is read back as conj(U[c][q])
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
        for (int i = 0; i < c; ++i) u[c * LD + i] = make_double2(0.0, 0.0);
        for (int i = c; i < m; ++i) {
            T2 acc = mk(T(i == c ? 1 : 0), T(0));
            for (int q = c; q < i; ++q) {
                const double2 uq = u[c * LD + q];
                acc = acc - cmul(L[i * m + q], mk((T)uq.x, (T)-uq.y));
            }
            const T2 z = rscale(rdiag[i], acc);
            u[c * LD + i] = make_double2((double)z.x, (double)-z.y);
        }
    }
}

// Maximum-overlap selection of bsz Ritz pairs in a block (+ new roots).
__global__ void select_kernel(const double *evals, const double2 *evecs, int mB, int b, int M, int nblk,
                              int nprob, double *eps, double2 *Ysel) {
    const int prob = blockIdx.x * blockDim.x + threadIdx.x;
    if (prob >= nprob) return;
    const int k = prob / nblk, blk = prob % nblk;
    const int lo = blk * b, bsz = min(b, M - lo);
    const double *w = evals + (size_t)prob * LD;
    const double2 *Y = evecs + (size_t)prob * LD * LD;
    double ov[LD];
    int chosen[LD];
    bool used[LD];
    for (int l = 0; l < mB; ++l) {
        double s = 0.0;
        for (int i = 0; i < bsz; ++i) s += Y[i * LD + l].x * Y[i * LD + l].x + Y[i * LD + l].y * Y[i * LD + l].y;
        ov[l] = s;
        used[l] = false;
    }
    for (int c = 0; c < bsz; ++c) {     // stable top-bsz by overlap
        int best = -1;
        for (int l = 0; l < mB; ++l)
            if (!used[l] && (best < 0 || ov[l] > ov[best])) best = l;
        chosen[c] = best;
        used[best] = true;
    }
    double lowest_in = 1e300;
    for (int i = 0; i < bsz; ++i) lowest_in = fmin(lowest_in, eps[k * M + lo + i]);
    for (int l = 0; l < mB; ++l) {
        if (used[l]) continue;
        if (w[l] < lowest_in && ov[l] < 0.5) {
            int worst = 0;
            for (int c = 1; c < bsz; ++c)
                if (w[chosen[c]] > w[chosen[worst]]) worst = c;
            if (w[l] < w[chosen[worst]]) {
                used[chosen[worst]] = false;
                chosen[worst] = l;
                used[l] = true;
            }
        }
    }
    for (int i = 1; i < bsz; ++i) {     // sort chosen by Ritz value
        int x = chosen[i], j = i - 1;
        while (j >= 0 && w[chosen[j]] > w[x]) { chosen[j + 1] = chosen[j]; --j; }
        chosen[j + 1] = x;
    }
    double2 *ys = Ysel + (size_t)prob * LD * LD;
    for (int c = 0; c < bsz; ++c) {
        for (int r = 0; r < mB; ++r) ys[r * LD + c] = Y[r * LD + chosen[c]];
        eps[k * M + lo + c] = w[chosen[c]];
    }
}

__global__ void take_evals_kernel(const double *evals, int M, int nk, double *eps) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < M * nk) eps[e] = evals[(size_t)(e / M) * LD + (e % M)];
}

// banded solves on vector ranges of every k-point (FP64)
// L L^T y = x, one thread per (vector, G) column; the last K-1 solution values
// ride in registers.  per_g: the k-point's factors L_G[j][d] stored as
// pfac[(j*K + d)*ldg + G] (coalesced over G); else the G-independent L_z.
// F32: on the FP32 Gram-Schmidt copies with FP32 factors (a preconditioner
// solve, whose rounding only changes which Krylov space is built).
template <int K, bool F32>
__global__ void eig_banded_solve_kernel(const EigK *ks, const void *Lbv, int per_g, int nb, int src, int dst,
                                        int nv) {
    typedef typename std::conditional<F32, float2, double2>::type T2;
    typedef typename std::conditional<F32, float, double>::type T;
    const int k = blockIdx.z / nv, v = blockIdx.z % nv;
    const EigK d = ks[k];
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= d.ldg) return;
    T2 *vb = F32 ? reinterpret_cast<T2 *>(d.v32) : reinterpret_cast<T2 *>(d.base);
    const T *Lb = reinterpret_cast<const T *>(Lbv);
    const T *pf = F32 ? reinterpret_cast<const T *>(d.pfac32) : reinterpret_cast<const T *>(d.pfac);
    const T2 *x = vb + (long long)(src + v) * d.nvec;
    T2 *y = vb + (long long)(dst + v) * d.nvec;
    const size_t ldg = d.ldg;
    if (g >= d.ng) {
        for (int j = 0; j < nb; ++j) y[(size_t)j * ldg + g] = czero<T2>();
        return;
    }
    // factors hold L[j][j-d] for d >= 1 and 1 / L[j][j] at d = 0
    auto L = [&](int j, int dd) -> T {
        return per_g ? pf[((size_t)j * K + dd) * ldg + g] : __ldg(&Lb[(size_t)j * K + dd]);
    };
    // rows are handled in tiles of PD: every load of a tile (right-hand
    // sides and factors, none of which depends on the recurrence) is issued
    // before the tile's recurrence runs
    constexpr int PD = F32 ? 8 : 4;
    T2 win[K];
#pragma unroll
    for (int i = 0; i < K; ++i) win[i] = czero<T2>();
    for (int j0 = 0; j0 < nb; j0 += PD) {
        T2 xs[PD];
        T fs[PD][K];
#pragma unroll
        for (int u = 0; u < PD; ++u) {
            const int j = j0 + u;
            xs[u] = j < nb ? x[(size_t)j * ldg + g] : czero<T2>();
#pragma unroll
            for (int dd = 0; dd < K; ++dd) fs[u][dd] = (j < nb && j - dd >= 0) ? L(j, dd) : T(0);
        }
#pragma unroll
        for (int u = 0; u < PD; ++u) {
            const int j = j0 + u;
            if (j >= nb) break;
            T2 s = xs[u];
#pragma unroll
            for (int dd = 1; dd < K; ++dd) rfma(s, -fs[u][dd], win[dd - 1]);
            const T2 yj = rscale(fs[u][0], s);
            y[(size_t)j * ldg + g] = yj;
#pragma unroll
            for (int i = K - 1; i > 0; --i) win[i] = win[i - 1];
            win[0] = yj;
        }
    }
#pragma unroll
    for (int i = 0; i < K; ++i) win[i] = czero<T2>();
    for (int j1 = nb - 1; j1 >= 0; j1 -= PD) {
        T2 xs[PD];
        T fs[PD][K];
#pragma unroll
        for (int u = 0; u < PD; ++u) {
            const int j = j1 - u;
            xs[u] = j >= 0 ? y[(size_t)j * ldg + g] : czero<T2>();
            fs[u][0] = j >= 0 ? L(j, 0) : T(0);
#pragma unroll
            for (int dd = 1; dd < K; ++dd) fs[u][dd] = (j >= 0 && j + dd < nb) ? L(j + dd, dd) : T(0);
        }
#pragma unroll
        for (int u = 0; u < PD; ++u) {
            const int j = j1 - u;
            if (j < 0) break;
            T2 s = xs[u];
#pragma unroll
            for (int dd = 1; dd < K; ++dd) rfma(s, -fs[u][dd], win[dd - 1]);
            const T2 zj = rscale(fs[u][0], s);
            y[(size_t)j * ldg + g] = zj;
#pragma unroll
            for (int i = K - 1; i > 0; --i) win[i] = win[i - 1];
            win[0] = zj;
        }
    }
}

// A^H B, one warp per row i and up to GJ columns: the lanes stride over an
// n-chunk with coalesced loads, each holding GJ complex partial sums in
// registers, then reduce them by warp shuffles.  Grid: (n-chunks, problems,
// row groups of 8 x column groups of GJ).
// GJ, the column-group width, is picked per call so that predicated-off
// column slots (which still occupy the FP64 pipe) are few.
// F32: the vectors are the FP32 Gram-Schmidt copies (v32) and the partial
// sums are FP32 (the reduction over chunks stays FP64).
template <bool F32, int GJ>
__global__ void __launch_bounds__(256) gram_rows_kernel(const EigK *ks, int nch, VSet A, VSet B, int nsplit,
                                                        int colgroups, double2 *part, int lower) {
    typedef typename std::conditional<F32, float2, double2>::type T2;
    typedef typename std::conditional<F32, float, double>::type T;
    const int split = blockIdx.x, prob = blockIdx.y;
    const int rg = blockIdx.z / colgroups, cg = blockIdx.z % colgroups;
    const int k = prob / nch, ch = prob % nch;
    const EigK d = ks[k];
    const int ma = A.count(), mb = B.count();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = rg * 8 + warp;
    const int j0 = cg * GJ, nj = min(GJ, mb - j0);
    if (i >= ma || nj <= 0) return;                     // whole warp leaves together
    if (lower && j0 > i) return;                        // tile above the diagonal
    const long long n = d.nvec;
    const long long chunk = (n + nsplit - 1) / nsplit;
    const long long t0 = split * chunk, t1 = min(n, t0 + chunk);
    const T2 *vb = F32 ? reinterpret_cast<const T2 *>(d.v32) : reinterpret_cast<const T2 *>(d.base);
    const T2 *a = vb + (long long)A.at(i, ch) * n;
    const T2 *bp[GJ];
#pragma unroll
    for (int jj = 0; jj < GJ; ++jj) bp[jj] = vb + (long long)B.at(j0 + (jj < nj ? jj : 0), ch) * n;
    T sx[GJ], sy[GJ];
#pragma unroll
    for (int jj = 0; jj < GJ; ++jj) sx[jj] = sy[jj] = T(0);
    for (long long t = t0 + lane; t < t1; t += 32) {
        const T2 av = a[t];
#pragma unroll
        for (int jj = 0; jj < GJ; ++jj) {
            if (jj < nj) {
                const T2 bv = bp[jj][t];
                sx[jj] = fma(av.x, bv.x, fma(av.y, bv.y, sx[jj]));
                sy[jj] = fma(av.x, bv.y, fma(-av.y, bv.x, sy[jj]));
            }
        }
    }
#pragma unroll
    for (int jj = 0; jj < GJ; ++jj) {
        if (jj >= nj) break;
        T x = sx[jj], y = sy[jj];
        for (int off = 16; off > 0; off >>= 1) {
            x += __shfl_down_sync(0xffffffffu, x, off);
            y += __shfl_down_sync(0xffffffffu, y, off);
        }
        if (lane == 0) part[((size_t)prob * nsplit + split) * ma * mb + (size_t)i * mb + j0 + jj] = make_double2(x, y);
    }
}

// A^H B for small ma, mb (<= 48) on the FP32 Gram-Schmidt copies: a CTA
// takes one chunk of the vector length for the whole ma x mb product,
// staging KC elements of every A and B vector in shared memory; each thread
// keeps a 3 x 3 block of outputs in registers.  Partial sums per chunk go to
// `part` (FP64) and are reduced in a fixed order by gram_reduce_kernel.
constexpr int GT_KC = 32, GT_MAX = 48;
// Larger products are covered by GT_MAX x GT_MAX tiles (blockIdx.z).
__global__ void __launch_bounds__(256) gram_tile32_kernel(const EigK *ks, int nch, VSet A, VSet B, int nsplit,
                                                          double2 *part) {
    __shared__ float2 As[GT_KC][GT_MAX + 1];
    __shared__ float2 Bs[GT_KC][GT_MAX + 1];
    const int split = blockIdx.x, prob = blockIdx.y;
    const int k = prob / nch, ch = prob % nch;
    const EigK d = ks[k];
    const int MA = A.count(), MB = B.count();
    const int ncb = (MB + GT_MAX - 1) / GT_MAX;
    const int r0 = (blockIdx.z / ncb) * GT_MAX, c0 = (blockIdx.z % ncb) * GT_MAX;
    const int ma = min(GT_MAX, MA - r0), mb = min(GT_MAX, MB - c0);
    const long long n = d.nvec;
    const long long chunk = (n + nsplit - 1) / nsplit;
    const long long t0 = split * chunk, t1 = min(n, t0 + chunk);
    const int ti = threadIdx.x / 16, tj = threadIdx.x % 16;   // rows 3*ti.., columns 3*tj..
    float2 acc[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) acc[i][j] = make_float2(0.f, 0.f);
    for (long long tb = t0; tb < t1; tb += GT_KC) {
        __syncthreads();
        for (int e = threadIdx.x; e < (ma + mb) * GT_KC; e += blockDim.x) {
            const int v = e / GT_KC, kk = e % GT_KC;
            const long long t = tb + kk;
            float2 val = make_float2(0.f, 0.f);
            if (v < ma) {
                if (t < t1) val = d.v32[(long long)A.at(r0 + v, ch) * n + t];
                As[kk][v] = val;
            } else {
                if (t < t1) val = d.v32[(long long)B.at(c0 + v - ma, ch) * n + t];
                Bs[kk][v - ma] = val;
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < GT_KC; ++kk) {
            float2 a[3], b[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) a[i] = As[kk][min(3 * ti + i, GT_MAX)];
#pragma unroll
            for (int j = 0; j < 3; ++j) b[j] = Bs[kk][min(3 * tj + j, GT_MAX)];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    acc[i][j].x = fmaf(a[i].x, b[j].x, fmaf(a[i].y, b[j].y, acc[i][j].x));
                    acc[i][j].y = fmaf(a[i].x, b[j].y, fmaf(-a[i].y, b[j].x, acc[i][j].y));
                }
        }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int r = 3 * ti + i, c = 3 * tj + j;
            if (r < ma && c < mb)
                part[((size_t)prob * nsplit + split) * MA * MB + (size_t)(r0 + r) * MB + c0 + c] =
                    make_double2(acc[i][j].x, acc[i][j].y);
        }
}

// Both Grams of a small pencil, V^H HV and V^H SV (lower triangles, m = M
// <= 8), on the FP32 copies: every thread reads the 3M vectors once per
// element and keeps all M(M+1) partial sums in registers; the CTA reduces
// them (FP64 across warps) into per-chunk partials for gram_reduce_kernel.
template <int M>
__global__ void __launch_bounds__(128) pencil_gram32_kernel(const EigK *ks, int nch, VSet V, VSet HV, VSet SV,
                                                           int nsplit, double2 *partH, double2 *partS) {
    constexpr int NL = M * (M + 1) / 2;
    constexpr int NW = 128 / 32;
    __shared__ float2 red[NW][2 * NL];
    const int split = blockIdx.x, prob = blockIdx.y;
    const int k = prob / nch, ch = prob % nch;
    const EigK d = ks[k];
    const long long n = d.nvec;
    const long long chunk = (n + nsplit - 1) / nsplit;
    const long long t0 = (long long)split * chunk, t1 = min(n, t0 + chunk);
    const float2 *vp[M], *hp[M], *sp[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        vp[i] = d.v32 + (long long)V.at(i, ch) * n;
        hp[i] = d.v32 + (long long)HV.at(i, ch) * n;
        sp[i] = d.v32 + (long long)SV.at(i, ch) * n;
    }
    float2 aH[NL], aS[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) aH[l] = aS[l] = make_float2(0.f, 0.f);
    for (long long t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
        float2 v[M], hv[M], sv[M];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            v[i] = vp[i][t];
            hv[i] = hp[i][t];
            sv[i] = sp[i][t];
        }
        int l = 0;
#pragma unroll
        for (int i = 0; i < M; ++i)
#pragma unroll
            for (int j = 0; j <= i; ++j, ++l) {      // G[i][j] = conj(v_i) x_j
                aH[l].x = fmaf(v[i].x, hv[j].x, fmaf(v[i].y, hv[j].y, aH[l].x));
                aH[l].y = fmaf(v[i].x, hv[j].y, fmaf(-v[i].y, hv[j].x, aH[l].y));
                aS[l].x = fmaf(v[i].x, sv[j].x, fmaf(v[i].y, sv[j].y, aS[l].x));
                aS[l].y = fmaf(v[i].x, sv[j].y, fmaf(-v[i].y, sv[j].x, aS[l].y));
            }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        float hx = aH[l].x, hy = aH[l].y, sx = aS[l].x, sy = aS[l].y;
        for (int off = 16; off > 0; off >>= 1) {
            hx += __shfl_down_sync(0xffffffffu, hx, off);
            hy += __shfl_down_sync(0xffffffffu, hy, off);
            sx += __shfl_down_sync(0xffffffffu, sx, off);
            sy += __shfl_down_sync(0xffffffffu, sy, off);
        }
        if (lane == 0) {
            red[warp][l] = make_float2(hx, hy);
            red[warp][NL + l] = make_float2(sx, sy);
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 2 * NL; e += blockDim.x) {
        double x = 0.0, y = 0.0;
        for (int w = 0; w < NW; ++w) {
            x += (double)red[w][e].x;
            y += (double)red[w][e].y;
        }
        const int l = e % NL;
        int i = 0;
        while ((i + 1) * (i + 2) / 2 <= l) ++i;
        const int j = l - i * (i + 1) / 2;
        double2 *part = e < NL ? partH : partS;
        part[((size_t)prob * nsplit + split) * M * M + (size_t)i * M + j] = make_double2(x, y);
    }
}

// A^H B on the tensor cores (tcgen05, TF32 inputs, FP32 accumulation in
// tensor memory) for the FP32 copies, to FP32 accuracy by splitting every
// value into x = hi + lo (hi = x rounded to TF32) and summing hi*hi + hi*lo +
// lo*hi.  Complex products become one real product over interleaved (re, im)
// rows: with the MMA's M side holding B_j and B'_j = (im, -re) of B_j, and its
// N side holding A_i,
//   D[j][i]      = sum (ar br + ai bi) = Re (A_i^H B_j)
//   D[mb + j][i] = sum (ar bi - ai br) = Im (A_i^H B_j).
// One CTA (128 threads, TMEM lane = row) takes one chunk of the vector length
// of one problem, in steps of GTC_KC complex elements staged in shared
// memory (canonical K-major layout without swizzle: 8-row x 16-byte core
// matrices, element (r, k) at (r/8)*SBO + (k/4)*LBO + (r%8)*16 + (k%4)*4).
// Requires 2 mb <= 128 and ma <= GTC_NMAX.  Partials go to `part` like the
// CUDA-core Gram kernels' (reduced by gram_reduce_kernel); a wait on the MMA
// barrier that runs out sets *err and skips the rest.
constexpr int GTC_KC = 32;                    // complex elements per step (64 TF32 values per row)
constexpr int GTC_NMAX = 64;
constexpr int GTC_LBO = 128, GTC_SBO = (2 * GTC_KC / 4) * 128;
__host__ __device__ constexpr size_t gtc_smem_bytes(int ntile) {
    return (size_t)2 * 128 * 2 * GTC_KC * 4 + (size_t)2 * ntile * 2 * GTC_KC * 4;
}
__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
__device__ __forceinline__ uint32_t gtc_off(int r, int k) {
    return (uint32_t)((r >> 3) * GTC_SBO + (k >> 2) * GTC_LBO + (r & 7) * 16 + (k & 3) * 4);
}
__global__ void __launch_bounds__(128) gram_tc32_kernel(const EigK *ks, int nch, VSet A, VSet B, int nsplit, int ntile,
                                                        double2 *part, int *err) {
    extern __shared__ __align__(1024) unsigned char gsm[];
    unsigned char *Mhi = gsm, *Mlo = gsm + 128 * 2 * GTC_KC * 4;
    unsigned char *Nhi = Mlo + 128 * 2 * GTC_KC * 4, *Nlo = Nhi + ntile * 2 * GTC_KC * 4;
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int failed;
    const int split = blockIdx.x, prob = blockIdx.y;
    const int k = prob / nch, ch = prob % nch;
    const EigK d = ks[k];
    const int ma = A.count(), mb = B.count();
    const long long n = d.nvec;
    const long long chunk = (n + nsplit - 1) / nsplit;
    const long long t0 = (long long)split * chunk, t1 = min(n, t0 + chunk);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int ncols = 32;
    while (ncols < ntile) ncols <<= 1;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&tmem_base)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        tc::mbar_init(&mbar, 1);
        failed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    // rows that no step writes (M side beyond 2 mb, N side beyond ma) stay zero
    for (int e = tid; e < (128 - 2 * mb) * 2 * GTC_KC; e += blockDim.x) {
        const int r = 2 * mb + e / (2 * GTC_KC), kk = e % (2 * GTC_KC);
        *reinterpret_cast<float *>(Mhi + gtc_off(r, kk)) = 0.f;
        *reinterpret_cast<float *>(Mlo + gtc_off(r, kk)) = 0.f;
    }
    for (int e = tid; e < (ntile - ma) * 2 * GTC_KC; e += blockDim.x) {
        const int r = ma + e / (2 * GTC_KC), kk = e % (2 * GTC_KC);
        *reinterpret_cast<float *>(Nhi + gtc_off(r, kk)) = 0.f;
        *reinterpret_cast<float *>(Nlo + gtc_off(r, kk)) = 0.f;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    // kind::tf32 instruction descriptor: D F32, A and B TF32, both K-major, M = 128, N = ntile
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(ntile >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    uint32_t phase = 0;
    bool any = false;
    // staging: element e = tid + 128 u of a side maps to row (e/8/KC)*8 + e%8
    // and element (e/8) % KC (a warp reads 8 rows x 4 consecutive elements);
    // each thread holds its elements of one step in registers, loaded while
    // the previous step's products run
    constexpr int UMAX = GTC_NMAX * GTC_KC / 128;     // 16
    const int nem = ((mb + 7) / 8) * 8 * GTC_KC, nea = ((ma + 7) / 8) * 8 * GTC_KC;
    float2 bv[UMAX], av[UMAX];
    auto fetch = [&](long long tb) {
#pragma unroll
        for (int u = 0; u < UMAX; ++u) {
            const int e = tid + 128 * u;
            const int rl = e & 7, c = (e >> 3) % GTC_KC, r = ((e >> 3) / GTC_KC) * 8 + rl;
            const long long t = tb + c;
            bv[u] = (e < nem && r < mb && t < t1) ? d.v32[(long long)B.at(r, ch) * n + t] : make_float2(0.f, 0.f);
            av[u] = (e < nea && r < ma && t < t1) ? d.v32[(long long)A.at(r, ch) * n + t] : make_float2(0.f, 0.f);
        }
    };
    if (t0 < t1) fetch(t0);
    for (long long tb = t0; tb < t1; tb += GTC_KC) {
#pragma unroll
        for (int u = 0; u < UMAX; ++u) {
            const int e = tid + 128 * u;
            const int rl = e & 7, c = (e >> 3) % GTC_KC, r = ((e >> 3) / GTC_KC) * 8 + rl;
            if (e < nem && r < mb) {
                const float2 v = bv[u];
                const float hx = tf32_rna(v.x), hy = tf32_rna(v.y);
                const float lx = v.x - hx, ly = v.y - hy;
                *reinterpret_cast<float2 *>(Mhi + gtc_off(r, 2 * c)) = make_float2(hx, hy);
                *reinterpret_cast<float2 *>(Mlo + gtc_off(r, 2 * c)) = make_float2(lx, ly);
                *reinterpret_cast<float2 *>(Mhi + gtc_off(mb + r, 2 * c)) = make_float2(hy, -hx);
                *reinterpret_cast<float2 *>(Mlo + gtc_off(mb + r, 2 * c)) = make_float2(ly, -lx);
            }
            if (e < nea && r < ma) {
                const float2 v = av[u];
                const float hx = tf32_rna(v.x), hy = tf32_rna(v.y);
                *reinterpret_cast<float2 *>(Nhi + gtc_off(r, 2 * c)) = make_float2(hx, hy);
                *reinterpret_cast<float2 *>(Nlo + gtc_off(r, 2 * c)) = make_float2(v.x - hx, v.y - hy);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) {
            const uint32_t mh = tc::smem_u32(Mhi), ml = tc::smem_u32(Mlo), nh = tc::smem_u32(Nhi), nl = tc::smem_u32(Nlo);
            for (int kk = 0; kk < 2 * GTC_KC / 8; ++kk) {
                const uint32_t o = kk * 2 * GTC_LBO;
                const uint64_t dmh = tc::smem_desc(mh + o, GTC_LBO, GTC_SBO), dml = tc::smem_desc(ml + o, GTC_LBO, GTC_SBO);
                const uint64_t dnh = tc::smem_desc(nh + o, GTC_LBO, GTC_SBO), dnl = tc::smem_desc(nl + o, GTC_LBO, GTC_SBO);
                const uint64_t da[3] = {dmh, dmh, dml}, db[3] = {dnh, dnl, dnh};
                for (int q = 0; q < 3; ++q) {
                    const uint32_t acc = (any || kk > 0 || q > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                        "l"(da[q]), "l"(db[q]), "r"(idesc), "r"(acc));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                tc::smem_u32(&mbar)));
        }
        any = true;
        if (tb + GTC_KC < t1) fetch(tb + GTC_KC);        // next step's loads overlap the products
        if (!tc::mbar_wait(&mbar, phase, 1ll << 24)) {
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
        // warp w holds rows (TMEM lanes) 32w .. 32w+31; 8 columns (A vectors) per load
        double *pd = reinterpret_cast<double *>(part + ((size_t)prob * nsplit + split) * ma * mb);
        const int r = 32 * warp + lane;
        for (int c0 = 0; c0 < ntile; c0 += 8) {
            uint32_t v[8];
            if (any) {
                const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                               "=r"(v[7])
                             : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
            } else {
                for (int j = 0; j < 8; ++j) v[j] = 0u;
            }
            for (int j = 0; j < 8; ++j) {
                const int c = c0 + j;
                if (c >= ma) break;
                if (r < mb) pd[2 * ((size_t)c * mb + r)] = (double)__uint_as_float(v[j]);
                else if (r < 2 * mb) pd[2 * ((size_t)c * mb + (r - mb)) + 1] = (double)__uint_as_float(v[j]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// Float-float arithmetic (a value is hi + lo, two FP32 numbers with
// |lo| <= ulp(hi)/2): Knuth's two-sum and the FMA two-product give the
// rounding error of a sum or product exactly, so sums of products carry
// about 48 significant bits on the FP32 pipe.
struct FF {
    float h, l;
};
__device__ __forceinline__ FF ff_from(double x) {
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}
// (the _rn intrinsics are never contracted into FMAs, which would break the
// exact error terms)
__device__ __forceinline__ void ff_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// acc += u v (u, v float-float; the lo*lo term is below the result's precision)
__device__ __forceinline__ void ff_mac(FF &acc, FF u, FF v) {
    const float ph = __fmul_rn(u.h, v.h);
    const float pl = fmaf(u.h, v.h, -ph) + fmaf(u.h, v.l, u.l * v.h);
    float s, e;
    ff_two_sum(acc.h, ph, s, e);
    acc.h = s;
    acc.l += e + pl;
}
__device__ __forceinline__ FF ff_neg(FF a) { return {-a.h, -a.l}; }

// C_j = beta C_j + alpha sum_i A_i Y[i][j] on FP64 vectors with the products
// and sums in float-float arithmetic (the mixed solver's FP64 root rotations:
// FP64-level results at the FP32 rate).  Same layout and launch as
// combine2_kernel.
template <int JC>
__global__ void __launch_bounds__(256) combine_ff_kernel(const EigK *ks, int nch, VSet A, VSet C,
                                                         const double2 *Y, double alpha, double beta) {
    __shared__ float4 Ys[JMAX][JC];     // (re.h, re.l, im.h, im.l)
    const int prob = blockIdx.y;
    const int k = prob / nch, ch = prob % nch;
    const EigK d = ks[k];
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = t < d.nvec;
    const int ma = A.count(), mc = C.count();
    const double2 *y = Y + (size_t)prob * LD * LD;
    for (int j0 = 0; j0 < mc; j0 += JC) {
        __syncthreads();
        for (int e = threadIdx.x; e < ma * JC; e += blockDim.x) {
            const int i = e / JC, jj = e % JC;
            const double2 yv = j0 + jj < mc ? y[i * LD + j0 + jj] : make_double2(0.0, 0.0);
            const FF re = ff_from(yv.x), im = ff_from(yv.y);
            Ys[i][jj] = make_float4(re.h, re.l, im.h, im.l);
        }
        __syncthreads();
        if (!live) continue;
        FF ar[JC], ai[JC];
#pragma unroll
        for (int jj = 0; jj < JC; ++jj) ar[jj] = ai[jj] = FF{0.f, 0.f};
        for (int i = 0; i < ma; ++i) {
            const double2 av = d.base[(long long)A.at(i, ch) * d.nvec + t];
            const FF xr = ff_from(av.x), xi = ff_from(av.y);
#pragma unroll
            for (int jj = 0; jj < JC; ++jj) {
                const float4 w = Ys[i][jj];
                const FF yr{w.x, w.y}, yi{w.z, w.w};
                ff_mac(ar[jj], xr, yr);          // re += xr yr - xi yi
                ff_mac(ar[jj], ff_neg(xi), yi);
                ff_mac(ai[jj], xr, yi);          // im += xr yi + xi yr
                ff_mac(ai[jj], xi, yr);
            }
        }
#pragma unroll
        for (int jj = 0; jj < JC; ++jj) {
            if (j0 + jj >= mc) break;
            double2 *c = d.base + (long long)C.at(j0 + jj, ch) * d.nvec + t;
            const double2 v = make_double2(alpha * ((double)ar[jj].h + (double)ar[jj].l),
                                           alpha * ((double)ai[jj].h + (double)ai[jj].l));
            *c = beta == 0.0 ? v : make_double2(beta * c->x + v.x, beta * c->y + v.y);
        }
    }
}

// C_j = beta C_j + alpha sum_i A_i Y[i][j]: one element t per thread, JC
// output columns at a time with their coefficients staged in shared memory.
template <int JC, bool F32>
__global__ void __launch_bounds__(256) combine2_kernel(const EigK *ks, int nch, VSet A, VSet C,
                                                       const double2 *Y, double alpha, double beta) {
    typedef typename std::conditional<F32, float2, double2>::type T2;
    typedef typename std::conditional<F32, float, double>::type T;
    __shared__ T2 Ys[JMAX][JC];
    const int prob = blockIdx.y;
    const int k = prob / nch, ch = prob % nch;
    const EigK d = ks[k];
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = t < d.nvec;
    const int ma = A.count(), mc = C.count();
    const double2 *y = Y + (size_t)prob * LD * LD;
    for (int j0 = 0; j0 < mc; j0 += JC) {
        __syncthreads();
        for (int e = threadIdx.x; e < ma * JC; e += blockDim.x) {
            const int i = e / JC, jj = e % JC;
            const double2 yv = j0 + jj < mc ? y[i * LD + j0 + jj] : make_double2(0.0, 0.0);
            Ys[i][jj] = mk((T)yv.x, (T)yv.y);
        }
        __syncthreads();
        if (!live) continue;
        T2 *vb = F32 ? reinterpret_cast<T2 *>(d.v32) : reinterpret_cast<T2 *>(d.base);
        T2 acc[JC];
#pragma unroll
        for (int jj = 0; jj < JC; ++jj) acc[jj] = czero<T2>();
        for (int i = 0; i < ma; ++i) {
            const T2 a = vb[(long long)A.at(i, ch) * d.nvec + t];
#pragma unroll
            for (int jj = 0; jj < JC; ++jj) cfma(acc[jj], a, Ys[i][jj]);
        }
#pragma unroll
        for (int jj = 0; jj < JC; ++jj) {
            if (j0 + jj >= mc) break;
            T2 *c = vb + (long long)C.at(j0 + jj, ch) * d.nvec + t;
            const T2 v = rscale((T)alpha, acc[jj]);
            *c = beta == 0.0 ? v : rscale((T)beta, *c) + v;
        }
    }
}

// [X|K]^H H [X|K] (and the S counterpart) when X holds Ritz vectors of the
// last Rayleigh-Ritz (X^H H X = diag(eps), X^H S X = I): rows i >= M come
// from the products KH = K^H H [X|K], KS = K^H S [X|K] (row i - M), the
// upper triangle is their conjugate.  GS may be null (no S matrix).
__global__ void assemble_rr_kernel(const double2 *KH, const double2 *KS, const double *eps, int M, int m,
                                   double2 *GH, double2 *GS) {
    const int k = blockIdx.y;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m * m) return;
    const int i = e / m, j = e % m;
    const size_t o = (size_t)k * LD * LD;
    double2 h, sv;
    if (i < M && j < M) {
        h = make_double2(i == j ? eps[k * M + i] : 0.0, 0.0);
        sv = make_double2(i == j ? 1.0 : 0.0, 0.0);
    } else if (i >= j) {
        h = KH[o + (i - M) * LD + j];
        sv = KS ? KS[o + (i - M) * LD + j] : make_double2(0.0, 0.0);
    } else {
        h = KH[o + (j - M) * LD + i];
        h.y = -h.y;
        sv = KS ? KS[o + (j - M) * LD + i] : make_double2(0.0, 0.0);
        sv.y = -sv.y;
    }
    if (i == j) { h.y = 0.0; sv.y = 0.0; }
    GH[o + i * LD + j] = h;
    if (GS) GS[o + i * LD + j] = sv;
}

// dead slots (mask 0) of an S-Gram matrix become identity rows and columns,
// so that its Cholesky factor exists and leaves them decoupled
__global__ void mask_sgram_kernel(double2 *G, const int *mask, int m) {
    const int prob = blockIdx.y;
    double2 *g = G + (size_t)prob * LD * LD;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m * m) return;
    const int i = e / m, j = e % m;
    const bool di = mask[prob * LD + i] == 0, dj = mask[prob * LD + j] == 0;
    if (di || dj) g[i * LD + j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
}

// C = op(A) B for small m x m matrices (leading dimension LD), one thread per
// output element; op = conjugate transpose when conjA.
__global__ void small_zgemm_kernel(const double2 *A, const double2 *B, double2 *C, int m, int conjA) {
    const int prob = blockIdx.y;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m * m) return;
    const int i = e / m, j = e % m;
    const double2 *a = A + (size_t)prob * LD * LD, *b = B + (size_t)prob * LD * LD;
    double2 s = make_double2(0.0, 0.0);
    for (int q = 0; q < m; ++q) {
        double2 av = conjA ? a[q * LD + i] : a[i * LD + q];
        if (conjA) av.y = -av.y;
        cfma(s, av, b[q * LD + j]);
    }
    C[(size_t)prob * LD * LD + i * LD + j] = s;
}

// dead-slot mask of a subspace: columns < ofs are the block's inputs (the
// first bsz live), columns >= ofs are Krylov slots with their alive flags
__global__ void alive_mask_kernel(const int *alive, int kd, int ofs, int M, int b, int nch, int m,
                                  int nprob, int *mask) {
    const int prob = blockIdx.x * blockDim.x + threadIdx.x;
    if (prob >= nprob) return;
    const int ch = prob % nch;
    const int bsz = nch == 1 ? M : min(b, M - ch * b);
    for (int c = 0; c < m; ++c)
        mask[prob * LD + c] = c < ofs ? (c < bsz ? 1 : 0) : alive[prob * kd + (c - ofs)];
}

__global__ void fill_int_kernel(int *p, int n, int v) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

__global__ void set_src_kernel(int *srcH, int *srcS, int nprob, int nch, int kH, int kS, int cs, int slot) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nprob) return;
    srcH[p] = kH + (p % nch) * cs + slot;
    srcS[p] = kS + (p % nch) * cs + slot;
}

// ---------------------------------------------------------------------------
// host driver
#define MB_LAUNCH_E(kid, ...)            \
    do {                                 \
        if (rc) break;                   \
        cudaEvent_t ev_;                 \
        prof_begin(h, s, kid, &ev_);     \
        __VA_ARGS__;                     \
        prof_end(h, s, kid, ev_);        \
        launched();                      \
    } while (0)

namespace {

// real symmetric Jacobi (host, small): z-modes of the initial guess
void host_jacobi_sym(int n, std::vector<double> &A, std::vector<double> &w, std::vector<double> &V) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                tot += A[(size_t)i * n + j] * A[(size_t)i * n + j];
                if (i != j) off += A[(size_t)i * n + j] * A[(size_t)i * n + j];
            }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                double th = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2 * apq);
                double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1));
                double c = 1 / std::sqrt(t * t + 1), s = t * c;
                for (int r = 0; r < n; ++r) {
                    double xp = A[(size_t)r * n + p], xq = A[(size_t)r * n + q];
                    A[(size_t)r * n + p] = c * xp - s * xq;
                    A[(size_t)r * n + q] = s * xp + c * xq;
                }
                for (int r = 0; r < n; ++r) {
                    double xp = A[(size_t)p * n + r], xq = A[(size_t)q * n + r];
                    A[(size_t)p * n + r] = c * xp - s * xq;
                    A[(size_t)q * n + r] = s * xp + c * xq;
                }
                for (int r = 0; r < n; ++r) {
                    double vp = V[(size_t)r * n + p], vq = V[(size_t)r * n + q];
                    V[(size_t)r * n + p] = c * vp - s * vq;
                    V[(size_t)r * n + q] = s * vp + c * vq;
                }
            }
    }
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
}

// Lowest M free-electron states (|k+G|^2/2 + z-mode n): pure plane wave times
// an S-normalized eigenvector of (D/2) c = e S c.  S-orthonormal by construction.
// The z modes of the free-electron start: eigenvectors c of (D/2) c = w S c,
// S-normalized (c = L^{-T} y with S = L L^T), ascending in w.  They do not
// depend on k, so they are computed once per handle.
static void zmodes(mb_handle *h) {
    if (!h->zmode_w.empty()) return;
    const int nb = h->nb, K = h->order, W = 2 * K - 1;
    std::vector<double> L((size_t)nb * nb, 0.0), D((size_t)nb * nb, 0.0);
    for (int j = 0; j < nb; ++j)
        for (int d = 0; d < K && j - d >= 0; ++d) L[(size_t)j * nb + (j - d)] = h->Lb[(size_t)j * K + d];
    for (int j = 0; j < nb; ++j)
        for (int dd = 0; dd < W; ++dd) {
            int jj = j + dd - (K - 1);
            if (jj >= 0 && jj < nb) D[(size_t)j * nb + jj] = 0.5 * h->Db[(size_t)j * W + dd];
        }
    // Linv by forward substitution
    std::vector<double> Li((size_t)nb * nb, 0.0);
    for (int c = 0; c < nb; ++c)
        for (int i = c; i < nb; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int q = c; q < i; ++q) s -= L[(size_t)i * nb + q] * Li[(size_t)q * nb + c];
            Li[(size_t)i * nb + c] = s / L[(size_t)i * nb + i];
        }
    std::vector<double> T1((size_t)nb * nb, 0.0), A((size_t)nb * nb, 0.0);
    for (int i = 0; i < nb; ++i)
        for (int j = 0; j < nb; ++j) {
            double s = 0;
            for (int q = 0; q < nb; ++q) s += Li[(size_t)i * nb + q] * D[(size_t)q * nb + j];
            T1[(size_t)i * nb + j] = s;
        }
    for (int i = 0; i < nb; ++i)
        for (int j = 0; j < nb; ++j) {
            double s = 0;
            for (int q = 0; q < nb; ++q) s += T1[(size_t)i * nb + q] * Li[(size_t)j * nb + q];
            A[(size_t)i * nb + j] = s;
        }
    std::vector<double> w, V;
    host_jacobi_sym(nb, A, w, V);
    std::vector<int> ord(nb);
    for (int i = 0; i < nb; ++i) ord[i] = i;
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return w[a] < w[b]; });
    h->zmode_w.resize(nb);
    h->zmode_c.assign((size_t)nb * nb, 0.0);   // [mode][j]
    for (int n = 0; n < nb; ++n) {
        h->zmode_w[n] = w[ord[n]];
        for (int j = 0; j < nb; ++j) {   // c_z = L^{-T} y
            double s = 0;
            for (int q = j; q < nb; ++q) s += Li[(size_t)q * nb + j] * V[(size_t)q * nb + ord[n]];
            h->zmode_c[(size_t)n * nb + j] = s;
        }
    }
}

// Lowest M free-electron states at k-point ik: plane wave G times z mode n,
// energy |k+G|^2/2 + w_n.
void free_electron_start(mb_handle *h, int ik, int M, std::vector<double2> &X) {
    zmodes(h);
    const int nb = h->nb;
    const KPoint &kp = h->kp[ik];
    std::vector<std::tuple<double, int, int>> cand;
    const int nmode = std::min(nb, M);
    cand.reserve((size_t)kp.ng * nmode);
    for (int g = 0; g < kp.ng; ++g)
        for (int n = 0; n < nmode; ++n) cand.emplace_back(0.5 * kp.q2[g] + h->zmode_w[n], g, n);
    std::partial_sort(cand.begin(), cand.begin() + std::min<size_t>(M, cand.size()), cand.end());
    X.assign((size_t)M * nb * kp.ldg, make_double2(0.0, 0.0));
    for (int c = 0; c < M; ++c) {
        const int g = std::get<1>(cand[c]), n = std::get<2>(cand[c]);
        for (int j = 0; j < nb; ++j) X[((size_t)c * nb + j) * kp.ldg + g] = make_double2(h->zmode_c[(size_t)n * nb + j], 0.0);
    }
}

struct Solver {
    mb_handle *h;
    cudaStream_t s;
    int nk, M, kd, b, nblk, mA, mB, nc;
    int Mconv;          // roots tested for convergence and returned (M includes guards)
    int prec;           // precision of the H applies that build Krylov vectors
    bool fp64_roots = false;   // finish phase: HX of the roots recomputed in FP64 every cycle
    // mixed precision: the Krylov Gram-Schmidt runs on FP32 copies (v32), and
    // the small Rayleigh-Ritz problems of cycles A and B use the S-Gram of
    // their basis (a pencil; FP32 in the bulk cycles, FP64 in the finish
    // phase), so that their result does not depend on how orthogonal the
    // Krylov vectors came out
    bool gs32 = false;
    // bulk cycles (lowp()): X, HX and SX live only in the FP32 copies, and
    // the chains' slot s of chain ch is at o32K + s*nc + ch (likewise SK, HK),
    // so that one slot of every chain is a contiguous block for the applies
    int o32X = 0, o32SX = 0, o32HX = 0, o32W = 0, o32K = 0, o32SK = 0, o32HK = 0, o32T = 0, o32T2 = 0, n32 = 0;
    double2 *d_Sg = nullptr, *d_Ub = nullptr, *d_Tb = nullptr;
    int *d_statb = nullptr;
    int oV, oHV, oSV, oVB, oHVB, oSVB, oQ, oHQ, oW, oSW, oT;
    int nvecs;
    std::vector<EigK> kd_host;
    EigK *d_k = nullptr;
    std::vector<void *> allocs;
    double2 *d_G = nullptr, *d_part = nullptr, *d_Y = nullptr, *d_Ysel = nullptr;
    double2 *d_U = nullptr, *d_G2 = nullptr, *d_T = nullptr;
    double *d_evals = nullptr, *d_eps = nullptr, *d_res = nullptr, *d_dots = nullptr, *d_theta = nullptr;
    int *d_seed = nullptr, *d_srcH = nullptr, *d_srcS = nullptr, *d_alive = nullptr, *d_status = nullptr;
    int *d_mask = nullptr;
    int *d_tcerr = nullptr;   // set by a tensor-core kernel whose bounded wait ran out
    size_t part_cap = 0;
    long long nmax = 0;
    int maxldg = 0;
    int applies = 0;
    int rc = MB_OK;

    ~Solver() {
        for (void *p : allocs) cudaFreeAsync(p, s);   // stream-ordered: no device-wide synchronization
    }
    int cuda(cudaError_t e) {
        if (e != cudaSuccess && rc == MB_OK) rc = cuda_fail(h, e);
        return rc;
    }
    int launched() { return cuda(cudaGetLastError()); }
    template <typename T> T *alloc(size_t n) {
        void *p = nullptr;
        if (rc) return nullptr;
        if (cuda(cudaMallocFromPoolAsync(&p, std::max<size_t>(n, 1) * sizeof(T), mb_pool(h->device), s))) return nullptr;
        allocs.push_back(p);
        return reinterpret_cast<T *>(p);
    }

    // G = A^H B per problem; lower: A^H B is Hermitian (A and B span the same
    // vectors in the same order), only j <= i is computed
    void gram(int nch, VSet A, VSet B, double2 *G, bool f32 = false, bool lower = false) {
        const int mbc = B.count();
        // narrowest column group that covers mbc in the fewest slots
        static const int widths[] = {1, 2, 3, 4, 5, 6, 7, 8, 12, 16};
        int gj = 16;
        long long best = 1ll << 40;
        for (int w : widths) {
            const long long slots = (long long)((mbc + w - 1) / w) * w;
            const long long cost = slots * 64 + (mbc + w - 1) / w;   // column slots, then fewer groups
            if (cost < best) { best = cost; gj = w; }
        }
        switch (gj) {
#define MB_GJ(W) case W: gram_t<W>(nch, A, B, G, f32, lower); break;
            MB_GJ(1) MB_GJ(2) MB_GJ(3) MB_GJ(4) MB_GJ(5) MB_GJ(6) MB_GJ(7) MB_GJ(8) MB_GJ(12) MB_GJ(16)
#undef MB_GJ
        }
    }
    template <int GJ> void gram_t(int nch, VSet A, VSet B, double2 *G, bool f32, bool lower) {
        const int nprob = nk * nch;
        const int ma = A.count(), mbc = B.count();
        if (f32 && mbc >= 4 && 2 * mbc <= 128 && ma <= GTC_NMAX && ma * mbc >= 64) {
            // tensor cores: two resident CTAs per SM over the whole grid
            const int ntile = std::max(16, (ma + 15) / 16 * 16);
            int nsplit = std::max(1, std::min(1024, (2 * h->num_sms + nprob - 1) / nprob));
            nsplit = std::min<long long>(nsplit, std::max<long long>(1, nmax / (2 * GTC_KC)));
            while ((size_t)nprob * nsplit * ma * mbc > part_cap && nsplit > 1) --nsplit;
            const size_t smem = gtc_smem_bytes(ntile);
            cuda(smem_limit_once((const void *)gram_tc32_kernel, h->device, h->smem_optin));
            MB_LAUNCH_E(KN_GRAM32, gram_tc32_kernel<<<dim3(nsplit, nprob), 128, smem, s>>>(d_k, nch, A, B, nsplit, ntile,
                                                                                        d_part, d_tcerr));
            MB_LAUNCH_E(KN_GRAM32,
                        gram_reduce_kernel<<<dim3((ma * mbc + 7) / 8, nprob), 256, 0, s>>>(d_part, nsplit, ma, mbc, G,
                                                                                           lower ? 1 : 0));
            return;
        }
        if (f32 && ma * mbc >= 64 && mbc >= 4) {
            // tile kernel: about two resident CTAs per SM over the whole grid
            const int tiles = ((ma + GT_MAX - 1) / GT_MAX) * ((mbc + GT_MAX - 1) / GT_MAX);
            int nsplit = std::max(1, std::min(1024, (2 * h->num_sms + nprob * tiles - 1) / (nprob * tiles)));
            nsplit = std::min<long long>(nsplit, std::max<long long>(1, nmax / (4 * GT_KC)));
            while ((size_t)nprob * nsplit * ma * mbc > part_cap && nsplit > 1) --nsplit;
            MB_LAUNCH_E(KN_GRAM32, gram_tile32_kernel<<<dim3(nsplit, nprob, tiles), 256, 0, s>>>(d_k, nch, A, B, nsplit,
                                                                                               d_part));
            MB_LAUNCH_E(KN_GRAM32,
                        gram_reduce_kernel<<<dim3((ma * mbc + 7) / 8, nprob), 256, 0, s>>>(d_part, nsplit, ma, mbc, G,
                                                                                           lower ? 1 : 0));
            return;
        }
        const int rowgroups = (ma + 7) / 8, colgroups = (mbc + GJ - 1) / GJ;
        const int per_split = nprob * rowgroups * colgroups;
        int nsplit = std::max(1, std::min(512, (8 * h->num_sms + per_split - 1) / per_split));
        nsplit = std::min<long long>(nsplit, std::max<long long>(1, nmax / 256));   // >= 256 elements per chunk
        while ((size_t)nprob * nsplit * ma * mbc > part_cap && nsplit > 1) --nsplit;
        if (f32)
            MB_LAUNCH_E(KN_GRAM32, (gram_rows_kernel<true, GJ><<<dim3(nsplit, nprob, rowgroups * colgroups), 256, 0, s>>>(
                                       d_k, nch, A, B, nsplit, colgroups, d_part, lower ? 1 : 0)));
        else
            MB_LAUNCH_E(KN_GRAM, (gram_rows_kernel<false, GJ><<<dim3(nsplit, nprob, rowgroups * colgroups), 256, 0, s>>>(
                                     d_k, nch, A, B, nsplit, colgroups, d_part, lower ? 1 : 0)));
        MB_LAUNCH_E(f32 ? KN_GRAM32 : KN_GRAM,
                    gram_reduce_kernel<<<dim3((ma * mbc + 7) / 8, nprob), 256, 0, s>>>(d_part, nsplit, ma, mbc, G,
                                                                                           lower ? 1 : 0));
    }
    void combine(int nch, VSet A, VSet C, const double2 *Y, double alpha, double beta, bool f32 = false) {
        if (f32) {
            combine_t<true>(nch, A, C, Y, alpha, beta);
        } else if (gs32 && C.count() > 8) {
            // mixed solver, FP64 vectors: the root rotations in float-float
            const dim3 grid((unsigned)((nmax + 255) / 256), nk * nch);
            MB_LAUNCH_E(KN_COMBINE, (combine_ff_kernel<12><<<grid, 256, 0, s>>>(d_k, nch, A, C, Y, alpha, beta)));
        } else {
            combine_t<false>(nch, A, C, Y, alpha, beta);
        }
    }
    template <bool F32> void combine_t(int nch, VSet A, VSet C, const double2 *Y, double alpha, double beta) {
        const dim3 grid((unsigned)((nmax + 255) / 256), nk * nch);
        const int mc = C.count();
        // column width with the least padding (12 divides the common 36)
        auto waste = [&](int jc) { return (mc + jc - 1) / jc * jc - mc; };
        if (mc == 1)
            MB_LAUNCH_E(F32 ? KN_COMBINE32 : KN_COMBINE, (combine2_kernel<1, F32><<<grid, 256, 0, s>>>(d_k, nch, A, C, Y, alpha, beta)));
        else if (mc <= 4)
            MB_LAUNCH_E(F32 ? KN_COMBINE32 : KN_COMBINE, (combine2_kernel<4, F32><<<grid, 256, 0, s>>>(d_k, nch, A, C, Y, alpha, beta)));
        else if (mc <= 8)
            MB_LAUNCH_E(F32 ? KN_COMBINE32 : KN_COMBINE, (combine2_kernel<8, F32><<<grid, 256, 0, s>>>(d_k, nch, A, C, Y, alpha, beta)));
        else if (waste(12) < waste(16))
            MB_LAUNCH_E(F32 ? KN_COMBINE32 : KN_COMBINE, (combine2_kernel<12, F32><<<grid, 256, 0, s>>>(d_k, nch, A, C, Y, alpha, beta)));
        else
            MB_LAUNCH_E(F32 ? KN_COMBINE32 : KN_COMBINE, (combine2_kernel<16, F32><<<grid, 256, 0, s>>>(d_k, nch, A, C, Y, alpha, beta)));
    }
    // U = L^{-H} of np problems (FP32 arithmetic in the bulk cycles)
    void cholinv(int np, int m, const double2 *G, double2 *U, int *status, bool f32) {
        if (f32) {
            const size_t smem = (size_t)m * m * sizeof(float2) + m * sizeof(float);
            cuda(smem_limit_once((const void *)cholinv_kernel<float>, h->device, h->smem_optin));
            MB_LAUNCH_E(KN_SMALL, cholinv_kernel<float><<<np, 128, smem, s>>>(G, m, U, status));
        } else {
            const size_t smem = (size_t)m * m * sizeof(double2) + m * sizeof(double);
            cuda(smem_limit_once((const void *)cholinv_kernel<double>, h->device, h->smem_optin));
            MB_LAUNCH_E(KN_SMALL, cholinv_kernel<double><<<np, 128, smem, s>>>(G, m, U, status));
        }
    }
    void small_gemm(const double2 *A, const double2 *B, double2 *C, int m, int conjA, int np = 0) {
        MB_LAUNCH_E(KN_SMALL, small_zgemm_kernel<<<dim3((m * m + 127) / 128, np > 0 ? np : nk), 128, 0, s>>>(
                                  A, B, C, m, conjA));
    }
    void copy(int nch, VSet S, VSet D, int mode) {
        const unsigned bx = (unsigned)std::min<long long>(64, (nmax + 255) / 256);
        MB_LAUNCH_E(KN_VEC, copy_kernel<<<dim3(bx, S.count(), nk * nch), 256, 0, s>>>(d_k, nch, S, D, mode));
    }
    // S X: the banded S_0 of Eqs. (7)-(8) and, for ultrasoft atoms, the
    // augmentation term sum q |beta><beta| X (§II.B.2)
    void bandS(int src, int dst, int nv, bool f32 = false) {
        if (rc) return;
        std::vector<int> iks(nk);
        std::vector<const void *> xs(nk);
        std::vector<void *> ys(nk);
        for (int k = 0; k < nk; ++k) {
            iks[k] = k;
            if (f32) {
                xs[k] = kd_host[k].v32 + (long long)src * kd_host[k].nvec;
                ys[k] = kd_host[k].v32 + (long long)dst * kd_host[k].nvec;
            } else {
                xs[k] = kd_host[k].base + (long long)src * kd_host[k].nvec;
                ys[k] = kd_host[k].base + (long long)dst * kd_host[k].nvec;
            }
        }
        const int prec = f32 ? MB_FP32 : MB_FP64;
        int r = banded_block_apply(h, false, nk, iks.data(), xs.data(), ys.data(), nv, prec, s);
        if (r == MB_OK && h->uspp) r = uspp_S_add(h, nk, iks.data(), xs.data(), ys.data(), nv, prec, s);
        if (r && rc == MB_OK) rc = r;
    }
    void coldot(int nch, VSet A, VSet B, double *out, bool f32 = false) {
        const dim3 grid(A.count(), nk * nch);
        if (f32) MB_LAUNCH_E(KN_SMALL, coldot_kernel<true><<<grid, 256, 0, s>>>(d_k, nch, A, B, out));
        else MB_LAUNCH_E(KN_SMALL, coldot_kernel<false><<<grid, 256, 0, s>>>(d_k, nch, A, B, out));
    }
    // Y = H X on the FP32 copies (bulk cycles): nv vectors from src32 to dst32
    void apply32(int src32, int dst32, int nv) {
        if (rc) return;
        std::vector<int> iks(nk);
        std::vector<const void *> xs(nk);
        std::vector<void *> ys(nk);
        for (int k = 0; k < nk; ++k) {
            iks[k] = k;
            xs[k] = kd_host[k].v32 + (long long)src32 * kd_host[k].nvec;
            ys[k] = kd_host[k].v32 + (long long)dst32 * kd_host[k].nvec;
        }
        int r = apply_H_batch(h, nk, iks.data(), xs.data(), ys.data(), nv, prec, s);
        if (r && rc == MB_OK) rc = r;
        applies += nv * nk;
    }
    void bandSolve(int per_g, int src, int dst, int nv, bool f32 = false) {
        const dim3 grid((maxldg + 63) / 64, 1, nk * nv);
        const void *Lb = f32 ? h->t32.Lrecip : h->t64.Lrecip;
        switch (h->order) {
#define MB_BL(KK)                                                                                                 \
    case KK:                                                                                                      \
        if (f32)                                                                                                  \
            MB_LAUNCH_E(KN_BANDED, (eig_banded_solve_kernel<KK, true><<<grid, 64, 0, s>>>(d_k, Lb, per_g, h->nb, src, dst, nv))); \
        else                                                                                                      \
            MB_LAUNCH_E(KN_BANDED, (eig_banded_solve_kernel<KK, false><<<grid, 64, 0, s>>>(d_k, Lb, per_g, h->nb, src, dst, nv))); \
        break;
            MB_BL(3) MB_BL(4) MB_BL(5) MB_BL(6) MB_BL(7) MB_BL(8)
#undef MB_BL
        }
    }
    int nc_stage() const { return std::max(M, nc); }
    void applyH(int src, int dst, int nv, int p) {
        if (rc) return;
        std::vector<int> iks(nk);
        std::vector<const void *> xs(nk);
        std::vector<void *> ys(nk);
        for (int k = 0; k < nk; ++k) {
            iks[k] = k;
            if (p == MB_FP64) {
                xs[k] = kd_host[k].base + (long long)src * kd_host[k].nvec;
                ys[k] = kd_host[k].base + (long long)dst * kd_host[k].nvec;
            } else {
                xs[k] = kd_host[k].stage;
                ys[k] = kd_host[k].stage + (long long)nc_stage() * kd_host[k].nvec;
            }
        }
        if (p != MB_FP64) copy(1, vs(src, nv), vs(0, nv), 1);
        if (rc) return;
        int r = apply_H_batch(h, nk, iks.data(), xs.data(), ys.data(), nv, p, s);
        if (r && rc == MB_OK) rc = r;
        if (p != MB_FP64) copy(1, vs(nc_stage(), nv), vs(dst, nv), 2);
        applies += nv * nk;
    }
    void residuals_and_seeds(int nch) {
        if (lowp()) {
            MB_LAUNCH_E(KN_VEC, residual32_kernel<<<dim3(256, nk), 256, 0, s>>>(d_k, M, o32HX, o32SX, o32T, d_eps));
            bandSolve(0, o32T, o32T2, M, true);
            coldot(1, vs(o32T, M), vs(o32T2, M), d_dots, true);
        } else {
            MB_LAUNCH_E(KN_VEC, residual_kernel<<<dim3(256, nk), 256, 0, s>>>(d_k, M, oV, oHV, oSV, oT, d_eps));
            bandSolve(0, oT, oT + M, M);
            coldot(1, vs(oT, M), vs(oT + M, M), d_dots);
        }
        int np = nk * nch;
        MB_LAUNCH_E(KN_SMALL, seed_kernel<<<(np + 63) / 64, 64, 0, s>>>(d_dots, M, Mconv, nk, nch, b, d_res, d_eps, d_seed,
                                                                        d_theta, d_srcH, d_srcS, oHV, oSV));
    }
    // H K[slot] of every chain into HK[slot]; reduced-precision applies go
    // straight from the chain slots through the FP32 stage
    void applyH_chain(int nch, int slot, int kV, int kH, int cs) {
        if (prec == MB_FP64) {
            copy(nch, vs(kV + slot, 1, cs), vs(oQ, 1, 1), 0);
            applyH(oQ, oHQ, nch, prec);
            copy(nch, vs(oHQ, 1, 1), vs(kH + slot, 1, cs), 0);
            return;
        }
        if (rc) return;
        std::vector<int> iks(nk);
        std::vector<const void *> xs(nk);
        std::vector<void *> ys(nk);
        for (int k = 0; k < nk; ++k) {
            iks[k] = k;
            xs[k] = kd_host[k].stage;
            ys[k] = kd_host[k].stage + (long long)nc_stage() * kd_host[k].nvec;
        }
        copy(nch, vs(kV + slot, 1, cs), vs(0, 1, 1), 1);
        if (rc) return;
        int r = apply_H_batch(h, nk, iks.data(), xs.data(), ys.data(), nch, prec, s);
        if (r && rc == MB_OK) rc = r;
        copy(nch, vs(nc_stage(), 1, 1), vs(kH + slot, 1, cs), 2);
        applies += nch * nk;
    }
    // classical Gram-Schmidt, twice, in the S inner product, of the chain
    // inputs W (one per chain) on the FP32 copies: all coefficients of a pass
    // come from the same (pre-update) vector.  The roots X are common to
    // every chain of a k-point, so their part is one product with a column
    // per chain.
    void gs32_passes(int nch, int i) {
        for (int pass = 0; pass < 2; ++pass) {
            gram(1, vs(o32SX, M), vs(o32W, nch), d_G2, true);                              // SX^H [W_0 .. W_nch-1]
            if (i > 0) gram(nch, vs(o32SK, i, 1, 0, 0, 0, nc), vs(o32W, 1, 1), d_G, true);  // SK_ch^H W_ch
            combine(1, vs(o32X, M), vs(o32W, nch), d_G2, -1.0, 1.0, true);
            if (i > 0) combine(nch, vs(o32K, i, 1, 0, 0, 0, nc), vs(o32W, 1, 1), d_G, -1.0, 1.0, true);
        }
    }
    void krylov(int nch, int kV, int kS, int kH, int cs) {
        int np = nk * nch;
        MB_LAUNCH_E(KN_SMALL, fill_int_kernel<<<(np * kd + 127) / 128, 128, 0, s>>>(d_alive, np * kd, 1));
        const unsigned rbx = (unsigned)std::min<long long>(1024, (nmax + 255) / 256);
        if (lowp()) {
            // bulk cycles: every step on the FP32 copies; the applies read
            // and write the chain slots in place
            for (int i = 0; i < kd && !rc; ++i) {
                if (i > 0) apply32(o32K + (i - 1) * nc, o32HK + (i - 1) * nc, nch);
                MB_LAUNCH_E(KN_VEC, krylov_residual32_kernel<<<dim3(rbx, np), 256, 0, s>>>(
                                        d_k, nch, i, d_seed, d_theta, o32HX, o32SX, o32HK, o32SK, nc, o32W));
                bandSolve(1, o32W, o32W, nch, true);
                gs32_passes(nch, i);
                bandS(o32W, o32SK + i * nc, nch, true);
                coldot(nch, vs(o32W, 1, 1), vs(o32SK + i * nc, 1, 1), d_dots, true);
                MB_LAUNCH_E(KN_VEC, normalize32_kernel<<<dim3(128, np), 256, 0, s>>>(d_k, nch, o32W, o32K, o32SK, nc, i,
                                                                                     d_dots, d_alive, kd));
            }
            apply32(o32K + (kd - 1) * nc, o32HK + (kd - 1) * nc, nch);
            return;
        }
        if (gs32) {
            copy(1, vs(oV, M), vs(o32X, M), 3);
            copy(1, vs(oSV, M), vs(o32SX, M), 3);
        }
        for (int i = 0; i < kd && !rc; ++i) {
            if (i > 0) {
                applyH_chain(nch, i - 1, kV, kH, cs);
                MB_LAUNCH_E(KN_SMALL, set_src_kernel<<<(np + 63) / 64, 64, 0, s>>>(d_srcH, d_srcS, np, nch, kH, kS, cs, i - 1));
            }
            MB_LAUNCH_E(KN_VEC, krylov_residual_kernel<<<dim3(rbx, np), 256, 0, s>>>(
                                    d_k, nch, d_srcH, d_srcS, d_theta, gs32 ? o32W : oW, gs32 ? 1 : 0));
            if (gs32) {
                bandSolve(1, o32W, o32W, nch, true);
                gs32_passes(nch, i);
                copy(nch, vs(o32W, 1, 1), vs(oW, 1, 1), 4);
            } else {
                bandSolve(1, oW, oW, nch);
                for (int pass = 0; pass < 2; ++pass) {
                    gram(1, vs(oSV, M), vs(oW, nch), d_G2);                    // SX^H [W_0 .. W_nch-1]
                    if (i > 0) gram(nch, vs(kS, i, cs), vs(oW, 1, 1), d_G);     // SK_ch^H W_ch
                    combine(1, vs(oV, M), vs(oW, nch), d_G2, -1.0, 1.0);
                    if (i > 0) combine(nch, vs(kV, i, cs), vs(oW, 1, 1), d_G, -1.0, 1.0);
                }
            }
            bandS(oW, oSW, nch);
            coldot(nch, vs(oW, 1, 1), vs(oSW, 1, 1), d_dots);
            const bool need32 = gs32 && i + 1 < kd;
            MB_LAUNCH_E(KN_VEC, normalize_kernel<<<dim3(128, np), 256, 0, s>>>(d_k, nch, oW, oSW, kV, kS, cs, i,
                                                                               d_dots, d_alive, kd,
                                                                               need32 ? o32K : -1, o32SK, nc));
        }
        applyH_chain(nch, kd - 1, kV, kH, cs);
    }
    void jacobi(int nch, int m, bool masked, int ofs, bool f32 = false) {
        if (f32) jacobi_t<float>(nch, m, masked, ofs, 1e-6);
        else jacobi_t<double>(nch, m, masked, ofs, 1e-13);
    }
    template <typename T> void jacobi_t(int nch, int m, bool masked, int ofs, double tol) {
        const size_t c2 = 2 * sizeof(T);
        const size_t stat = 32 * sizeof(double) + sizeof(int) + LD * sizeof(int) + 256;
        size_t smem2 = (size_t)2 * m * m * c2 + kJacobiScratchBytes;
        size_t smem1 = (size_t)m * m * c2 + kJacobiScratchBytes;
        size_t smemx = (size_t)m * m * (2 * sizeof(double2) + 2 * sizeof(float2)) + kJacobiScratchBytes;
        const bool vs = smem2 + stat <= (size_t)h->smem_optin;
        const bool mixed = std::is_same<T, double>::value && m <= JMIX_MAX && smemx + stat <= (size_t)h->smem_optin;
        int np = nk * nch;
        if (masked)
            MB_LAUNCH_E(KN_SMALL, alive_mask_kernel<<<(np + 63) / 64, 64, 0, s>>>(d_alive, kd, ofs, M, b, nch, m, np, d_mask));
        if (mixed) {
            cuda(smem_limit_once((const void *)jacobi_mixed_kernel, h->device, h->smem_optin));
            MB_LAUNCH_E(KN_JACOBI, (jacobi_mixed_kernel<<<np, kJacobiThreads, smemx, s>>>(d_G, m, masked ? d_mask : nullptr, LD, 0,
                                                                               d_evals, d_Y, 30, tol)));
        } else if (vs) {
            cuda(smem_limit_once((const void *)jacobi_kernel<true, T>, h->device, h->smem_optin));
            MB_LAUNCH_E(KN_JACOBI, (jacobi_kernel<true, T><<<np, kJacobiThreads, smem2, s>>>(d_G, m, masked ? d_mask : nullptr, LD, 0,
                                                                                  d_evals, d_Y, 30, tol)));
        } else {
            cuda(smem_limit_once((const void *)jacobi_kernel<false, T>, h->device, h->smem_optin));
            MB_LAUNCH_E(KN_JACOBI, (jacobi_kernel<false, T><<<np, kJacobiThreads, smem1, s>>>(d_G, m, masked ? d_mask : nullptr, LD, 0,
                                                                                   d_evals, d_Y, 30, tol)));
        }
    }
    // bulk cycles of the mixed solver (before the FP64 finish phase)
    bool lowp() const { return gs32 && !fp64_roots; }
    // Rayleigh-Ritz of the pencil (V^H H V, V^H S V) of nch problems of size m
    // per k-point: U = L^{-H} from V^H S V = L L^H (dead Krylov slots made
    // identity), Ritz pairs of U^H (V^H H V) U; returns the Ritz vectors'
    // coordinates in the V basis (U Y) and leaves the values in d_evals.
    const double2 *rr_pencil(int nch, VSet V, VSet HV, VSet SV, int m, int ofs, bool f32 = false) {
        if (f32 && m >= 2 && m <= 8) {
            pencil_grams32(nch, V, HV, SV, m);
        } else {
            gram(nch, V, HV, d_G, f32, true);
            gram(nch, V, SV, d_Sg, f32, true);
        }
        return pencil_solve(nch, m, ofs);
    }
    // V^H HV into d_G and V^H SV into d_Sg (lower triangles completed), FP32 copies
    void pencil_grams32(int nch, VSet V, VSet HV, VSet SV, int m) {
        const int nprob = nk * nch;
        int nsplit = std::max(1, std::min(32, (4 * h->num_sms + nprob - 1) / nprob));
        while ((size_t)2 * nprob * nsplit * m * m > part_cap && nsplit > 1) --nsplit;
        double2 *pH = d_part, *pS = d_part + (size_t)nprob * nsplit * m * m;
        const dim3 grid(nsplit, nprob);
        switch (m) {
#define MB_PG(MM) case MM: MB_LAUNCH_E(KN_GRAM32, (pencil_gram32_kernel<MM><<<grid, 128, 0, s>>>(d_k, nch, V, HV, SV, nsplit, pH, pS))); break;
            MB_PG(2) MB_PG(3) MB_PG(4) MB_PG(5) MB_PG(6) MB_PG(7) MB_PG(8)
#undef MB_PG
        }
        const dim3 gr((m * m + 7) / 8, nprob);
        MB_LAUNCH_E(KN_GRAM32, gram_reduce_kernel<<<gr, 256, 0, s>>>(pH, nsplit, m, m, d_G, 1));
        MB_LAUNCH_E(KN_GRAM32, gram_reduce_kernel<<<gr, 256, 0, s>>>(pS, nsplit, m, m, d_Sg, 1));
    }
    // the pencil (d_G, d_Sg) of nch problems per k-point
    const double2 *pencil_solve(int nch, int m, int ofs) {
        const int np = nk * nch;
        const dim3 gs((m * m + 127) / 128, np);
        MB_LAUNCH_E(KN_SMALL, alive_mask_kernel<<<(np + 63) / 64, 64, 0, s>>>(d_alive, kd, ofs, M, b, nch, m, np, d_mask));
        MB_LAUNCH_E(KN_SMALL, mask_sgram_kernel<<<gs, 128, 0, s>>>(d_Sg, d_mask, m));
        cholinv(np, m, d_Sg, d_Ub, d_statb, lowp());
        small_gemm(d_G, d_Ub, d_Tb, m, 0, np);    // (V^H H V) U
        small_gemm(d_Ub, d_Tb, d_G, m, 1, np);    // U^H (V^H H V) U
        jacobi(nch, m, true, ofs, lowp());
        small_gemm(d_Ub, d_Y, d_Tb, m, 0, np);    // U Y
        return d_Tb;
    }
    // X, HX <- [V|..](m) Y[:, :M] and SX = S X (S is banded: recomputing it is
    // cheaper than rotating it).  Bulk cycles (lowp): the rotation of the
    // FP32 copies V32 in FP32, and HX from a fresh FP32 apply instead of a
    // rotation (cheaper, and no less accurate than HK from FP32 applies).
    void rotate_set(const double2 *Y, int m, const VSet *V32 = nullptr) {
        if (lowp()) {
            combine(1, *V32, vs(o32T, M), Y, 1.0, 0.0, true);
            copy(1, vs(o32T, M), vs(o32X, M), 5);
            apply32(o32X, o32HX, M);
            bandS(o32X, o32SX, M, true);
            return;
        }
        combine(1, vs(oV, m), vs(oT, M), Y, 1.0, 0.0);
        combine(1, vs(oHV, m), vs(oT + M, M), Y, 1.0, 0.0);
        copy(1, vs(oT, M), vs(oV, M), 0);
        copy(1, vs(oT + M, M), vs(oHV, M), 0);
        bandS(oV, oSV, M);
    }
    // Rayleigh-Ritz on [X | K_A] (withK) or on X.  With K_A, X holds the Ritz
    // vectors of the last Rayleigh-Ritz, so only the Krylov rows of the
    // projected matrices are computed.
    void rr_full(bool withK) {
        int m = withK ? mA : M;
        if (withK && lowp()) {
            // bulk cycles: the Krylov rows from the FP32 copies
            gram(1, vs(o32K, kd, 0, 0, 0, 0, nc), vs(o32HX, M, 0, o32HK, kd, 0, 1, nc), d_G2, true);
            gram(1, vs(o32K, kd, 0, 0, 0, 0, nc), vs(o32SX, M, 0, o32SK, kd, 0, 1, nc), d_T, true);
        } else if (withK) {
            gram(1, vs(oV + M, kd), vs(oHV, m), d_G2);
            if (gs32) gram(1, vs(oV + M, kd), vs(oSV, m), d_T);
        }
        if (withK) {
            MB_LAUNCH_E(KN_SMALL, assemble_rr_kernel<<<dim3((m * m + 127) / 128, nk), 128, 0, s>>>(
                                      d_G2, gs32 ? d_T : nullptr, d_eps, M, m, d_G, gs32 ? d_Sg : nullptr));
            if (gs32) {
                const VSet v32 = vs(o32X, M, 0, o32K, kd, 0, 1, nc);
                rotate_set(pencil_solve(1, m, M), m, &v32);
            } else {
                jacobi(1, m, true, M);
                rotate_set(d_Y, m);
            }
        } else {
            gram(1, vs(oV, m), vs(oHV, m), d_G, false, true);
            jacobi(1, m, false, M);
            rotate_set(d_Y, m);
        }
        MB_LAUNCH_E(KN_SMALL, take_evals_kernel<<<(M * nk + 127) / 128, 128, 0, s>>>(d_evals, M, nk, d_eps));
    }
    // S-orthonormalization and Rayleigh-Ritz in one rotation: U = L^{-H} from
    // X^H S X = L L^H, Ritz pairs of U^H (X^H H X) U, then X <- X U Y.
    void orth_rr() {
        const bool f32 = lowp();
        if (f32) {
            gram(1, vs(o32X, M), vs(o32SX, M), d_G, true, true);
        } else {
            gram(1, vs(oV, M), vs(oSV, M), d_G, false, true);
        }
        cholinv(nk, M, d_G, d_U, d_status, f32);
        if (f32) gram(1, vs(o32X, M), vs(o32HX, M), d_G2, true, true);
        else gram(1, vs(oV, M), vs(oHV, M), d_G2, false, true);
        small_gemm(d_G2, d_U, d_T, M, 0);     // (X^H H X) U
        small_gemm(d_U, d_T, d_G, M, 1);      // U^H (X^H H X) U
        jacobi(1, M, false, M, lowp());
        small_gemm(d_U, d_Y, d_T, M, 0);      // U Y
        const VSet x32 = vs(o32X, M);
        rotate_set(d_T, M, &x32);
        MB_LAUNCH_E(KN_SMALL, take_evals_kernel<<<(M * nk + 127) / 128, 128, 0, s>>>(d_evals, M, nk, d_eps));
    }
    void cycle_B() {
        residuals_and_seeds(nblk);
        if (!lowp()) {
            copy(nblk, vs(oV, b, b), vs(oVB, b, mB), 0);
            copy(nblk, vs(oHV, b, b), vs(oHVB, b, mB), 0);
            if (gs32) copy(nblk, vs(oSV, b, b), vs(oSVB, b, mB), 0);
        }
        krylov(nblk, oVB + b, oSVB + b, oHVB + b, mB);
        const double2 *Yc = d_Y;
        // block ch: [X_b | K_ch] (in the bulk cycles from the FP32 copies)
        const VSet x32 = vs(o32X, b, b, o32K, kd, 1, 1, nc);
        const VSet hx32 = vs(o32HX, b, b, o32HK, kd, 1, 1, nc);
        if (lowp()) {
            Yc = rr_pencil(nblk, x32, hx32, vs(o32SX, b, b, o32SK, kd, 1, 1, nc), mB, b, true);
        } else if (gs32) {
            Yc = rr_pencil(nblk, vs(oVB, mB, mB), vs(oHVB, mB, mB), vs(oSVB, mB, mB), mB, b);
        } else {
            gram(nblk, vs(oVB, mB, mB), vs(oHVB, mB, mB), d_G, false, true);
            jacobi(nblk, mB, true, b);
        }
        int np = nk * nblk;
        MB_LAUNCH_E(KN_SMALL, select_kernel<<<(np + 31) / 32, 32, 0, s>>>(d_evals, Yc, mB, b, M, nblk, np, d_eps, d_Ysel));
        if (lowp()) {
            // the new X and HX of every block land in scratch (nblk*b vectors
            // each) first: the rotation reads the old X
            combine(nblk, x32, vs(o32T, b, b), d_Ysel, 1.0, 0.0, true);
            combine(nblk, hx32, vs(o32T2, b, b), d_Ysel, 1.0, 0.0, true);
            copy(1, vs(o32T, M), vs(o32X, M), 5);
            copy(1, vs(o32T2, M), vs(o32HX, M), 5);
            bandS(o32X, o32SX, M, true);
        } else {
            combine(nblk, vs(oVB, mB, mB), vs(oV, b, b), d_Ysel, 1.0, 0.0);
            combine(nblk, vs(oHVB, mB, mB), vs(oHV, b, b), d_Ysel, 1.0, 0.0);
            bandS(oV, oSV, M);
        }
    }
};

}  // namespace

namespace {
// The solve runs on a private non-blocking stream (capturable, unlike the
// legacy default stream) that first waits for the caller's stream.
// a mixed-precision warm start whose FP64 residuals are all below this (Ha)
// goes straight to the finish phase
constexpr double kWarmFinishResidual = 1e-4;

struct SolveStream {
    cudaStream_t s = nullptr;
    cudaError_t err = cudaSuccess;
    SolveStream(cudaStream_t caller) {
        err = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (err != cudaSuccess) return;
        cudaEvent_t ev;
        err = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (err != cudaSuccess) return;
        err = cudaEventRecord(ev, caller);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(s, ev, 0);
        cudaEventDestroy(ev);
    }
    ~SolveStream() {
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    }
};
}  // namespace

int eigsolve(mb_handle *h, int nbands, double tol, int prec, double *evals, void *evecs,
             const mb_solve_opts *so, mb_solve_info *info, cudaStream_t caller) {
    auto t0 = std::chrono::steady_clock::now();
    if (!evals || nbands < 1 || !(tol > 0.0)) return MB_EINVAL;
    if (prec != MB_FP64 && prec != MB_FP32 && prec != MB_BF16) return MB_EINVAL;
    if (cudaSetDevice(h->device) != cudaSuccess) return MB_ECUDA;
    SolveStream stream(caller);       // declared before the solver: its workspace is freed on it first
    if (stream.err != cudaSuccess) return cuda_fail(h, stream.err);
    cudaStream_t s = stream.s;
    Solver S;
    S.h = h;
    S.s = s;
    S.nk = (int)h->kp.size();
    int guard = so && so->guard != 0 ? std::max(0, so->guard) : std::max(2, (nbands + 7) / 8);
    S.Mconv = nbands;
    S.M = nbands + guard;
    S.kd = so && so->krylov_depth > 0 ? so->krylov_depth : kDefaultKrylovDepth;
    S.b = so && so->block > 0 ? so->block : kDefaultBlock;
    int max_cycles = so && so->max_cycles > 0 ? so->max_cycles : 200;
    if (S.b > S.M) S.b = S.M;
    S.nblk = (S.M + S.b - 1) / S.b;
    S.mA = S.M + S.kd;
    S.mB = S.b + S.kd;
    S.nc = std::max(1, S.nblk);
    if (S.mA > JMAX || S.mB > JMAX || S.M > LD) return MB_EUNSUPPORTED;
    if (S.nc_stage() > h->max_bands) return MB_EUNSUPPORTED;
    for (auto &k : h->kp)
        if ((long long)k.ng * h->nb < S.mA) return MB_EINVAL;
    if (cudaSetDevice(h->device) != cudaSuccess) return MB_ECUDA;
    int rc = ensure_precond(h);
    if (rc) return rc;
    // vector regions
    // [X | K_A] regions are sized so that the last block of cycle B, when M is
    // not a multiple of b, writes its unused columns into K_A (scratch then)
    const int mAr = std::max(S.mA, S.nblk * S.b);
    S.oV = 0;
    S.oHV = mAr;
    S.oSV = 2 * mAr;
    S.oVB = 3 * mAr;
    S.oHVB = S.oVB + S.nblk * S.mB;
    S.oSVB = S.oHVB + S.nblk * S.mB;
    S.oQ = S.oSVB + S.nblk * S.mB;
    S.oHQ = S.oQ + S.nc;
    S.oW = S.oHQ + S.nc;
    S.oSW = S.oW + S.nc;
    S.oT = S.oSW + S.nc;
    S.nvecs = S.oT + 3 * S.mA;
    // FP32 Gram-Schmidt workspace (mixed precision): X, SX, the chain inputs W,
    // then K and SK of every chain (chain ch, depth i at + ch*kd + i)
    S.gs32 = prec != MB_FP64;
    S.o32X = 0;
    S.o32SX = S.M;
    S.o32HX = 2 * S.M;
    S.o32W = 3 * S.M;
    S.o32K = S.o32W + S.nc;
    S.o32SK = S.o32K + S.nc * S.kd;
    S.o32HK = S.o32SK + S.nc * S.kd;
    S.o32T = S.o32HK + S.nc * S.kd;
    S.o32T2 = S.o32T + std::max(S.M, S.nblk * S.b);
    S.n32 = S.o32T2 + std::max(S.M, S.nblk * S.b);
    // per-k memory
    S.kd_host.resize(S.nk);
    size_t pofs = 0;
    for (int k = 0; k < S.nk; ++k) {
        EigK &e = S.kd_host[k];
        e.ldg = h->kp[k].ldg;
        e.ng = h->kp[k].ng;
        e.nvec = (long long)h->nb * e.ldg;
        e.base = S.alloc<double2>((size_t)S.nvecs * e.nvec);
        e.stage = S.alloc<float2>((size_t)2 * S.nc_stage() * e.nvec);
        e.v32 = S.gs32 ? S.alloc<float2>((size_t)S.n32 * e.nvec) : nullptr;
        e.pfac = (const double *)h->t64.Pfac + pofs;
        e.pfac32 = (const float *)h->t32.Pfac + pofs;
        pofs += (size_t)e.ldg * h->nb * h->order;
        if (S.rc) return S.rc;
        S.cuda(cudaMemsetAsync(e.base, 0, sizeof(double2) * (size_t)S.nvecs * e.nvec, s));
        S.nmax = std::max(S.nmax, e.nvec);
        S.maxldg = std::max(S.maxldg, e.ldg);
    }
    int nprob = S.nk * S.nc;
    S.d_k = S.alloc<EigK>(S.nk);
    S.d_G = S.alloc<double2>((size_t)nprob * LD * LD);
    S.d_Y = S.alloc<double2>((size_t)nprob * LD * LD);
    S.d_Ysel = S.alloc<double2>((size_t)nprob * LD * LD);
    S.d_U = S.alloc<double2>((size_t)S.nk * LD * LD);
    S.d_G2 = S.alloc<double2>((size_t)S.nk * LD * LD);
    S.d_T = S.alloc<double2>((size_t)S.nk * LD * LD);
    S.part_cap = (size_t)std::max(2 * h->num_sms, nprob) * JMAX * JMAX;
    S.d_part = S.alloc<double2>(S.part_cap);
    S.d_evals = S.alloc<double>((size_t)nprob * LD);
    S.d_eps = S.alloc<double>((size_t)S.nk * S.M);
    S.d_res = S.alloc<double>((size_t)S.nk * S.M);
    S.d_dots = S.alloc<double>((size_t)S.nk * std::max(S.M, S.nc));
    S.d_theta = S.alloc<double>(nprob);
    S.d_seed = S.alloc<int>(nprob);
    S.d_srcH = S.alloc<int>(nprob);
    S.d_srcS = S.alloc<int>(nprob);
    S.d_alive = S.alloc<int>((size_t)nprob * S.kd);
    S.d_mask = S.alloc<int>((size_t)nprob * LD);
    S.d_status = S.alloc<int>(S.nk);
    S.d_tcerr = S.alloc<int>(1);
    if (S.gs32) {
        S.d_Sg = S.alloc<double2>((size_t)nprob * LD * LD);
        S.d_Ub = S.alloc<double2>((size_t)nprob * LD * LD);
        S.d_Tb = S.alloc<double2>((size_t)nprob * LD * LD);
        S.d_statb = S.alloc<int>(nprob);
    }
    if (S.rc) return S.rc;
    S.cuda(cudaMemcpyAsync(S.d_k, S.kd_host.data(), sizeof(EigK) * S.nk, cudaMemcpyHostToDevice, s));
    S.cuda(cudaMemsetAsync(S.d_Ysel, 0, sizeof(double2) * (size_t)nprob * LD * LD, s));
    S.cuda(cudaMemsetAsync(S.d_status, 0, sizeof(int) * S.nk, s));
    S.cuda(cudaMemsetAsync(S.d_tcerr, 0, sizeof(int), s));
    // initial trial vectors: the lowest free-electron states, or (warm
    // start) the caller's vectors in place of the first nbands of them
    const bool warm = so && so->warm_start && evecs;
    size_t woff = 0;
    for (int k = 0; k < S.nk && !S.rc; ++k) {
        std::vector<double2> X0;
        free_electron_start(h, k, S.M, X0);
        S.cuda(cudaMemcpyAsync(S.kd_host[k].base, X0.data(), sizeof(double2) * X0.size(), cudaMemcpyHostToDevice, s));
        const size_t nwarm = (size_t)nbands * h->nb * h->kp[k].ldg;
        if (warm)
            S.cuda(cudaMemcpyAsync(S.kd_host[k].base, reinterpret_cast<const double2 *>(evecs) + woff,
                                   sizeof(double2) * nwarm, cudaMemcpyDeviceToDevice, s));
        woff += nwarm;
        S.cuda(cudaStreamSynchronize(s));
    }
    S.prec = prec;
    // the apply scratch is sized up front for every batch this solve issues,
    // so that nothing allocates while a grand cycle is being captured
    {
        size_t need = 0;
        const int sizes[3] = {1, S.nc, S.nc_stage()};
        for (int pi = 0; pi < 2; ++pi)
            for (int bi = 0; bi < 3; ++bi) {
                need = std::max(need, apply_scratch_bytes(h, S.nk, sizes[bi], pi == 0 ? MB_FP64 : MB_FP32));
                if (h->uspp) need = std::max(need, uspp_scratch_bytes(h, S.nk, sizes[bi], pi == 0 ? MB_FP64 : MB_FP32));
            }
        S.cuda(cudaStreamSynchronize(s));
        if (S.rc == MB_OK) {
            int r2 = ensure_scratch(h, need, s);
            if (r2) return r2;
        }
    }
    bool started = false;
    if (S.lowp() && warm) {
        // a warm start already near convergence skips the FP32 bulk cycles
        // (whose rounding would first undo its accuracy): the start vectors'
        // FP64 residuals decide
        S.fp64_roots = true;
        S.applyH(S.oV, S.oHV, S.M, MB_FP64);
        S.bandS(S.oV, S.oSV, S.M);
        S.orth_rr();
        S.residuals_and_seeds(1);
        std::vector<double> r0((size_t)S.nk * S.M);
        S.cuda(cudaMemcpyAsync(r0.data(), S.d_res, sizeof(double) * r0.size(), cudaMemcpyDeviceToHost, s));
        S.cuda(cudaStreamSynchronize(s));
        double mx = 0.0;
        for (int k = 0; k < S.nk; ++k)
            for (int i = 0; i < S.Mconv; ++i) {
                const double r = r0[(size_t)k * S.M + i];
                mx = std::max(mx, r == r ? r : 1e300);
            }
        if (mx < kWarmFinishResidual) started = true;
        else S.fp64_roots = false;
    }
    if (!started) {
        if (S.lowp()) {
            // mixed precision: the bulk cycles start from FP32 copies of the
            // (S-orthonormal) start vectors
            S.copy(1, vs(S.oV, S.M), vs(S.o32X, S.M), 3);
            S.apply32(S.o32X, S.o32HX, S.M);
            S.bandS(S.o32X, S.o32SX, S.M, true);
            S.orth_rr();
        } else {
            S.applyH(S.oV, S.oHV, S.M, S.prec);
            S.bandS(S.oV, S.oSV, S.M);
            // the caller's vectors next to free-electron guards, or free-electron
            // states that the ultrasoft S does not keep orthonormal: S-orthonormalize
            if (warm || h->uspp) S.orth_rr();
            else S.rr_full(false);
        }
        S.residuals_and_seeds(1);
    }
    std::vector<double> res((size_t)S.nk * S.M);
    double last = 1e300, prev = 1e300, maxres = 1e300, bulk_best = 1e300;
    int bulk_idle = 0;
    int cycles = 0;
    bool converged = false;
    // One grand cycle: A (Krylov space of the worst root + Rayleigh-Ritz on
    // all roots), B (per-block Krylov spaces, Rayleigh-Ritz, maximum-overlap
    // selection), S-orthonormalization + Rayleigh-Ritz, residuals and seeds.
    auto cycle_body = [&]() {
        S.krylov(1, S.oV + S.M, S.oSV + S.M, S.oHV + S.M, 0);
        S.rr_full(true);
        S.cycle_B();
        // Krylov vectors may come from reduced-precision applies: in the
        // finish phase the roots' HX is recomputed in FP64 first, so the
        // Rayleigh-Ritz values and the residual test below are FP64
        if (S.fp64_roots) S.applyH(S.oV, S.oHV, S.M, MB_FP64);
        S.orth_rr();
        S.residuals_and_seeds(1);
    };
    // From the second cycle of each apply precision on, a cycle is one CUDA
    // graph launch (captured once); the host only reads the residuals.
    const bool use_graphs = !h->profiling;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    int applies_per_cycle[2] = {0, 0};
    int cur_gi = -1, plain_left = 0;
    auto conv_max = [&]() {
        double mx = 0.0;
        for (int k = 0; k < S.nk; ++k)
            for (int i = 0; i < S.Mconv; ++i) {
                double r = res[(size_t)k * S.M + i];
                mx = std::max(mx, r == r ? r : 1e300);
            }
        return mx;
    };
    int finish_cycles = 0;
    for (cycles = 1; cycles <= max_cycles && !S.rc; ++cycles) {
        const int gi = (S.prec == MB_FP64 || S.fp64_roots) ? 1 : 0;
        finish_cycles += gi;
        if (gi != cur_gi) {
            cur_gi = gi;
            plain_left = 1;
        }
        if (!use_graphs || plain_left > 0) {
            cycle_body();
            --plain_left;
        } else {
            if (!gexec[gi]) {
                cudaGraph_t graph = nullptr;
                const int before = S.applies;
                S.cuda(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
                cycle_body();
                applies_per_cycle[gi] = S.applies - before;
                S.applies = before;
                cudaError_t e = cudaStreamEndCapture(s, &graph);
                S.cuda(e);
                if (S.rc == MB_OK) S.cuda(cudaGraphInstantiate(&gexec[gi], graph, 0));
                if (graph) cudaGraphDestroy(graph);
            }
            if (S.rc == MB_OK) S.cuda(cudaGraphLaunch(gexec[gi], s));
            S.applies += applies_per_cycle[gi];
        }
        S.cuda(cudaMemcpyAsync(res.data(), S.d_res, sizeof(double) * res.size(), cudaMemcpyDeviceToHost, s));
        int tcerr = 0, tcerr_apply = 0;
        S.cuda(cudaMemcpyAsync(&tcerr, S.d_tcerr, sizeof(int), cudaMemcpyDeviceToHost, s));
        if (h->d_tcerr)        // the projector contractions of MB_BF16 applies
            S.cuda(cudaMemcpyAsync(&tcerr_apply, h->d_tcerr, sizeof(int), cudaMemcpyDeviceToHost, s));
        S.cuda(cudaStreamSynchronize(s));
        if (S.rc) break;
        if (tcerr || tcerr_apply) {   // a tensor-core kernel's bounded wait ran out: its products are not valid
            S.rc = MB_ETIMEOUT;
            break;
        }
        maxres = conv_max();
        if (S.prec != MB_FP64 && !S.fp64_roots) {
            // stalled: two bulk cycles in a row without a 30 % gain on the best
            // residual so far (the FP32 arithmetic of the bulk cycles has a
            // floor, and its residuals need not decrease monotonically there)
            if (maxres < 0.7 * bulk_best) {
                bulk_best = maxres;
                bulk_idle = 0;
            } else {
                ++bulk_idle;
            }
            // a stall counts only near the FP32 floor (~1e-5 of the spectrum's
            // width): far above it the largest residual belongs to roots still
            // converging, which the cheaper bulk cycles handle as well; past
            // half the cycle budget the finish phase starts regardless
            bool stalled = (cycles > 3 && maxres < 1e-3 && (maxres > 0.7 * prev || bulk_idle >= 2)) ||
                           cycles >= max_cycles / 2;
            if (maxres < 30.0 * tol || stalled) {
                // finish phase: the roots get FP64 HX from here on
                S.fp64_roots = true;
                S.copy(1, vs(S.o32X, S.M), vs(S.oV, S.M), 4);
                S.applyH(S.oV, S.oHV, S.M, MB_FP64);
                S.bandS(S.oV, S.oSV, S.M);
                S.orth_rr();
                S.residuals_and_seeds(1);
                S.cuda(cudaMemcpyAsync(res.data(), S.d_res, sizeof(double) * res.size(), cudaMemcpyDeviceToHost, s));
                S.cuda(cudaStreamSynchronize(s));
                maxres = conv_max();
            }
        }
        prev = last;
        last = maxres;
        if ((S.prec == MB_FP64 || S.fp64_roots) && maxres < tol) {
            converged = true;
            break;
        }
    }
    for (auto &g : gexec)
        if (g) cudaGraphExecDestroy(g);
    if (S.rc) return S.rc;
    if (S.lowp()) S.copy(1, vs(S.o32X, S.M), vs(S.oV, S.M), 4);   // stopped in the bulk phase
    std::vector<double> eps((size_t)S.nk * S.M);
    S.cuda(cudaMemcpyAsync(eps.data(), S.d_eps, sizeof(double) * eps.size(), cudaMemcpyDeviceToHost, s));
    if (evecs) {
        char *dst = reinterpret_cast<char *>(evecs);
        for (int k = 0; k < S.nk; ++k) {
            size_t bytes = sizeof(double2) * (size_t)S.Mconv * S.kd_host[k].nvec;
            S.cuda(cudaMemcpyAsync(dst, S.kd_host[k].base, bytes, cudaMemcpyDeviceToDevice, s));
            dst += bytes;
        }
    }
    S.cuda(cudaStreamSynchronize(s));
    if (S.rc) return S.rc;
    for (int k = 0; k < S.nk; ++k)
        std::memcpy(evals + (size_t)k * S.Mconv, eps.data() + (size_t)k * S.M, sizeof(double) * S.Mconv);
    if (info) {
        info->cycles = std::min(cycles, max_cycles);
        info->applies = S.applies;
        info->max_residual = maxres;
        info->finish_cycles = std::min(finish_cycles, max_cycles);
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return converged ? MB_OK : MB_ENOTCONV;
}

}  // namespace mb

// Self-test hook for the tensor-core Gram kernel: G = A^H B (FP64 host
// output, row-major ma x mb interleaved complex) for ma + mb FP32 complex
// vectors of length n stored contiguously on the device (A first), split
// into nsplit chunks.
extern "C" int mb_debug_gram_tc32(const void *V, long long n, int ma, int mb, int nsplit, double *G, void *stream) {
    using namespace mb;
    if (!V || !G || n < 1 || ma < 1 || mb < 1 || 2 * mb > 128 || ma > GTC_NMAX || nsplit < 1 || nsplit > 4096)
        return MB_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    EigK hk{};
    hk.v32 = reinterpret_cast<float2 *>(const_cast<void *>(V));
    hk.nvec = n;
    const int ntile = std::max(16, (ma + 15) / 16 * 16);
    EigK *dk = nullptr;
    double2 *part = nullptr, *Gd = nullptr;
    int *err = nullptr;
    cudaError_t e = cudaMalloc(&dk, sizeof(EigK));
    if (e == cudaSuccess) e = cudaMalloc(&part, sizeof(double2) * (size_t)nsplit * ma * mb);
    if (e == cudaSuccess) e = cudaMalloc(&Gd, sizeof(double2) * LD * LD);
    if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyAsync(dk, &hk, sizeof(EigK), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
    const size_t smem = gtc_smem_bytes(ntile);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(gram_tc32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        gram_tc32_kernel<<<dim3(nsplit, 1), 128, smem, s>>>(dk, 1, vs(0, ma), vs(ma, mb), nsplit, ntile, part, err);
        gram_reduce_kernel<<<dim3((ma * mb + 7) / 8, 1), 256, 0, s>>>(part, nsplit, ma, mb, Gd, 0);
        e = cudaGetLastError();
    }
    std::vector<double2> hG((size_t)LD * LD);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(hG.data(), Gd, sizeof(double2) * LD * LD, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(dk);
    cudaFree(part);
    cudaFree(Gd);
    cudaFree(err);
    if (e != cudaSuccess) return MB_ECUDA;
    for (int i = 0; i < ma; ++i)
        for (int j = 0; j < mb; ++j) {
            G[2 * ((size_t)i * mb + j)] = hG[(size_t)i * LD + j].x;
            G[2 * ((size_t)i * mb + j) + 1] = hG[(size_t)i * LD + j].y;
        }
    return herr ? MB_ETIMEOUT : MB_OK;
}

// Self-test hook for the float-float rotation kernel: C = A Y for ma FP64
// complex device vectors A of length n (stored one after another) and a host
// ma x mc complex matrix Y (interleaved doubles, row i = coefficients of
// A_i); C: mc device vectors of length n, overwritten.
extern "C" int mb_debug_combine_ff(const void *A, const double *Y, long long n, int ma, int mc, void *C,
                                   void *stream) {
    using namespace mb;
    if (!A || !Y || !C || n < 1 || ma < 1 || mc < 1 || ma > JMAX || mc > LD) return MB_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    // one work array holding A then C, addressed through index sets
    double2 *base = nullptr, *Yd = nullptr;
    EigK *dk = nullptr;
    cudaError_t e = cudaMalloc(&base, sizeof(double2) * (size_t)(ma + mc) * n);
    if (e == cudaSuccess) e = cudaMalloc(&Yd, sizeof(double2) * LD * LD);
    if (e == cudaSuccess) e = cudaMalloc(&dk, sizeof(EigK));
    std::vector<double2> hY((size_t)LD * LD, make_double2(0.0, 0.0));
    for (int i = 0; i < ma; ++i)
        for (int j = 0; j < mc; ++j)
            hY[(size_t)i * LD + j] = make_double2(Y[2 * ((size_t)i * mc + j)], Y[2 * ((size_t)i * mc + j) + 1]);
    EigK hk{};
    hk.base = base;
    hk.nvec = n;
    if (e == cudaSuccess) e = cudaMemcpyAsync(base, A, sizeof(double2) * (size_t)ma * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(Yd, hY.data(), sizeof(double2) * LD * LD, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dk, &hk, sizeof(EigK), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        const dim3 grid((unsigned)((n + 255) / 256), 1);
        combine_ff_kernel<12><<<grid, 256, 0, s>>>(dk, 1, vs(0, ma), vs(ma, mc), Yd, 1.0, 0.0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(C, base + (size_t)ma * n, sizeof(double2) * (size_t)mc * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(base);
    cudaFree(Yd);
    cudaFree(dk);
    return e == cudaSuccess ? MB_OK : MB_ECUDA;
}
