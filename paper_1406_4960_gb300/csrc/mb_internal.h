// Internal state of an mb_handle and the kernel launch interfaces.
#pragma once

#include <cuda_runtime.h>

#include <complex>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/mb.h"

namespace mb {

using cdouble = std::complex<double>;

// Per-k-point host data.
struct KPoint {
    double k[2];
    int ng = 0, ldg = 0;
    std::vector<int> n1, n2;        // G = n1 b1 + n2 b2
    std::vector<int> goff;          // natural grid offset i1*N2 + i2 of each G
    std::vector<double> q2;         // |k+G|^2
    std::vector<double> qx, qy;     // k+G cartesian
    std::vector<cdouble> qproj;     // nterm x ldg in-plane projector factors
};

// entries of a padded row of the S band: 2 order - 1 rounded up to a multiple
// of 4, so that a row is a whole number of 16-byte loads in both precisions
constexpr int band_pad(int order) { return (2 * order - 1 + 3) / 4 * 4; }

// Device copies of one precision (R = double or float).
struct DevTables {
    void *Bq = nullptr;      // nq x order, B_{t+m}(z_q) of the full basis
    void *V = nullptr;       // nq x N1 x N2, w_q V / (N1 N2), bit-reversed layout
    void *Vn = nullptr;      // the same in natural layout
    void *tw = nullptr;      // Nmax/2 complex, exp(+2 pi i k / Nmax)
    void *Sband = nullptr;   // nb x (2 order - 1): S[j][j+d], d = -(order-1)..order-1
    void *SbandP = nullptr;  // the same with rows padded to band_pad(order) entries (zeros)
    void *Dband = nullptr;   // same layout for D = <B'|B'>
    void *Lband = nullptr;   // nb x order: Cholesky L[j][j-d], d = 0..order-1
    void *Lrecip = nullptr;  // the same with 1 / L[j][j] at d = 0 (eigensolver's solves)
    void *q2 = nullptr;      // all k, concatenated with kofs
    void *qproj = nullptr;   // all k: nterm x ldg each (in-plane factor of every term), offset qofs[k]
    void *zproj = nullptr;   // nterm x nb: z factor of every projector term
    void *zf = nullptr;      // nzf x nb: the distinct rows of zproj
    void *E = nullptr;       // nkb diagonal strengths, then nkb partner couplings
    void *Pfac = nullptr;    // preconditioner factors: all k, ldg x nb x order each
    void *Vt = nullptr;      // nq x N2 x N1, w_q V / (N1 N2), i1 fastest (FP32 compact-plane kernel)
    void *Q = nullptr;       // ultrasoft q: nkb diagonal, then nkb partner couplings (the layout of E)
    void *Eid = nullptr;     // strengths 1 (diagonal) and 0 (couplings): the overlaps <beta_p|x> themselves
};

struct Scratch {
    size_t bytes = 0;
    void *ptr = nullptr;
};

}  // namespace mb

struct mb_handle {
    int device = 0;
    double a1[2], a2[2], b1[2], b2[2], Ac = 0;
    double ecut = 0;
    int order = 0, nquad = 0, nint = 0, nb = 0, nq = 0;
    int n1 = 0, n2 = 0, l1 = 0, l2 = 0;
    int nterm = 0;
    int max_bands = 0;
    int smem_optin = 227 * 1024;   // opt-in shared memory per block
    int num_sms = 152;
    double precond_shift = 1.0;
    std::vector<double> breaks, tau;
    std::vector<double> zq, wq;
    std::vector<double> Bq;          // nq x order
    std::vector<double> Sb, Db, Lb;  // band storage as in DevTables
    // local pseudopotential terms (Eq. (10)) grouped by profile: lgrp[3 g ..] =
    // kind (0 Gaussian, 1 core term), width (a, or R_c), height R_z; the
    // atoms of group g are lion[3 i ..] = (weight A or Z, x, y) for i in
    // lstart[g] .. lstart[g+1]
    std::vector<double> lgrp, lion;
    std::vector<int> lstart;
    double *d_vloc = nullptr;        // nq x N1 x N2 natural order, V(r, z_q) (Ha), on the device
    // Kleinman-Bylander projectors as sums of separable terms: projector p
    // (nkb of them) is u_p = sum_{t in terms(p)} zproj[t](j) qproj[t](G); a
    // 1s or p projector has one term, a 2s projector two.  Strengths: the
    // diagonal Ekb[p] and one coupling Ecoup[p] to projector partner[p]
    // (the 1s-2s pair of an atom; -1 for none).
    int nkb = 0;
    std::vector<double> zproj, Ekb, Ecoup;
    // ultrasoft augmentation (§II.B.2): q of every projector and of its
    // partner coupling (the layout of Ekb / Ecoup); the atoms whose
    // augmentation charges are nonzero: first projector, count, position, r_Q
    bool uspp = false;
    std::vector<double> Qkb, Qcoup;
    struct AugAtom { int p0, np; double x, y, z, rQ; };
    std::vector<AugAtom> aug;
    std::vector<int> tproj, partner, pstart, plist;   // term -> projector; terms of projector p
    // distinct z factors of the terms: zfun (nzf x nb), pgroup[t] = f, and
    // the terms of factor f in zlist[zstart[f] .. zstart[f+1])
    int nzf = 0;
    std::vector<double> zfun;
    std::vector<int> pgroup, zstart, zlist;
    // device copy: pgroup (nterm) | zstart (nzf+1) | zlist (nterm) | tproj (nterm)
    //              | partner (nkb) | pstart (nkb+1) | plist (nterm)
    int *d_zidx = nullptr;
    std::vector<mb::KPoint> kp;
    std::vector<int> kofs, qofs;     // offsets of per-k arrays (in elements)
    int total_ldg = 0;
    int *d_goff = nullptr;           // all k (int), offset kofs
    int *d_rows = nullptr;           // occupied grid rows of every k, offset rows_ofs[k]
    void *d_projB = nullptr;         // BF16 projector tables for the tensor-core contractions
    void *d_tcerr = nullptr;         // status word of the tensor-core kernels' bounded waits
    std::vector<int> pb0_ofs, pb1_ofs, pb0_ld, pb1_ld;
    std::vector<int> rows_ofs, nrows;
    // compact planes of the FP32 plane kernel, per k-point: occupied grid
    // rows n1min .. n1min + nocc - 1, and the disc-free positions of those rows
    int *d_cpos = nullptr;           // all k (int), offset kofs: (n1 - n1min)(N2 + 1) + (n2 mod N2)
    int *d_zpos = nullptr;           // all k, offset zofs[k], nzero[k] entries
    std::vector<int> nocc, zofs, nzero;
    std::vector<unsigned long long> rowmask;
    mb::DevTables t64, t32;
    bool pfac_ready = false;
    // z modes of the eigensolver's free-electron start (k-independent, cached)
    std::vector<double> zmode_w, zmode_c;
    mb::Scratch scratch;
    void *d_desc = nullptr;          // descriptor arrays for batched launches
    // second stream of the apply: the projector overlaps run there beside the
    // plane kernel (fork and join by events, capturable into graphs)
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // the handle's own stream: its tables are allocated, uploaded and freed
    // there (stream-ordered, from the library's pool), so setting up or
    // destroying a handle never waits for other work on the device
    cudaStream_t hs = nullptr;
    cudaEvent_t scratch_ev = nullptr;      // recorded after the last apply that used the scratch
    int *d_queue = nullptr;                // work-queue counters of the persistent plane kernel (2 ints)
    size_t desc_bytes = 0;
    std::string last_cuda_error;
    // plane-kernel launch shapes picked by mb_autotune: (k-points per batch,
    // bands, FP64?) -> (largest bands per CTA of the radix-2 / register-FFT
    // kernels, resident-CTA waves, compact-plane kernel instance id or -1)
    struct Tuned { int bt = 1; int waves = 0; int p32 = -1; int persist = 0; };
    std::map<std::tuple<int, int, int>, Tuned> tuned;
    std::string tune_report;         // the last mb_autotune's candidates and times
    // launch accounting (always on) and optional per-kernel event timing
    long long launches = 0;
    int profiling = 0;               // 0 off, 1 every kernel, 2 the plane kernel only
    struct ProfEvent { int kernel; cudaEvent_t a, b; };
    std::vector<ProfEvent> prof_pending;
    std::vector<cudaEvent_t> prof_pool;
    double prof_ms[16] = {0};
    long long prof_count[16] = {0};
};

namespace mb {

// setup.cpp
int build_host_tables(mb_handle *h, const mb_cell *cell, const double *kpts, int nk,
                      double ecut, const double *breaks, int nbreaks, int order,
                      const mb_atom *atoms, int natoms, const mb_opts *opts);
void precond_factors(const mb_handle *h, int ik, double shift, std::vector<double> &out);

// apply.cu
int upload_tables(mb_handle *h);
int upload_potential(mb_handle *h);
// vloc.cu
int vloc_build(mb_handle *h);             // d_vloc from the atoms' analytic terms, then the derived tables
int vloc_derive_tables(mb_handle *h);     // d_vloc -> t64.V/Vn, t32.V/Vn/Vt
size_t vloc_build_scratch_bytes(const mb_handle *h);
int vloc_tabulate(mb_handle *h, int mode, double *out, cudaStream_t s, const std::vector<double> *lgrp = nullptr,
                  const std::vector<double> *lion = nullptr, const std::vector<int> *lstart = nullptr);
// 0: V(r, z_q); 1: core charge density (of the given groups instead of the atoms', when passed)
// apply.cu: the ultrasoft overlap term Y += sum q_pq beta_p (beta_q^H X) (§II.B.2)
// S_0 X (inv = false) or S_0^-1 X (inv = true) for the blocks X[i] -> Y[i] of
// k-points iks[i] (nbands vectors at stride nb * ldg, X[i] != Y[i]); one launch
// per kMaxK k-points
int banded_block_apply(mb_handle *h, bool inv, int nsel, const int *iks, const void *const *X, void *const *Y,
                       int nbands, int prec, cudaStream_t s);
bool banded_block_supported(const mb_handle *h, int prec, bool inv);
int uspp_S_add(mb_handle *h, int nsel, const int *iks, const void *const *X, void *const *Y, int nbands, int prec,
               cudaStream_t s);
size_t uspp_scratch_bytes(const mb_handle *h, int nk, int nbands, int prec);
// apply.cu: <beta_p|x_b> of FP64 blocks (the layout of mb_eigsolve's evecs) into F (host,
// nk x nbands x nkb complex as interleaved doubles)
int uspp_overlaps(mb_handle *h, const void *evecs, int nbands, double *F, cudaStream_t s);
int ensure_precond(mb_handle *h);
void free_tables(mb_handle *h);
int ensure_scratch(mb_handle *h, size_t bytes, cudaStream_t s);
// the library's stream-ordered memory pool on a device (freed memory is kept
// for reuse up to a threshold instead of being returned at every sync)
cudaMemPool_t mb_pool(int device);
// device tables of a handle: allocate + upload on the handle's stream, free there
int dev_upload(mb_handle *h, void **dst, const void *src, size_t bytes);
void dev_free(mb_handle *h, void **p);
// the device half of mb_setup, for host tables already built
int setup_device(mb_handle *h);
int apply_H_batch(mb_handle *h, int nsel, const int *iks, const void *const *X,
                  void *const *Y, int nbands, int prec, cudaStream_t s);
int apply_banded_batch(mb_handle *h, int which, int nsel, const int *iks, const void *const *X,
                       void *const *Y, int nbands, int prec, cudaStream_t s);
size_t apply_scratch_bytes(const mb_handle *h, int nk, int nbands, int prec);
size_t apply_H_scratch_need(const mb_handle *h, int ik, int nbands, int prec);
int apply_H_on_scratch(mb_handle *h, int ik, const void *X, void *Y, int nbands, int prec, cudaStream_t s,
                       void *scratch);

enum { BAND_S = 0, BAND_SINV = 1, BAND_PREC = 2 };

// eigensolver defaults: Krylov depth and roots per block of the second grand
// cycle (one root per block: every root gets its own Krylov space, which
// needed the fewest FP64 operations to 1e-6 Ha on the slab and graphene cells)
constexpr int kDefaultKrylovDepth = 5;
constexpr int kDefaultBlock = 1;

// kernel ids for launch accounting / profiling
enum { KN_PLANE = 0, KN_EPILOGUE, KN_PROJ, KN_COEF, KN_BACKPROJ, KN_BANDED, KN_GRAM, KN_COMBINE,
       KN_JACOBI, KN_SMALL, KN_VEC, KN_GRAM32, KN_COMBINE32, KN_COUNT };
extern const char *const kKernelNames[KN_COUNT];
void prof_begin(mb_handle *h, cudaStream_t s, int kernel, cudaEvent_t *a);
void prof_end(mb_handle *h, cudaStream_t s, int kernel, cudaEvent_t a);
int prof_collect(mb_handle *h);

int cuda_fail(mb_handle *h, cudaError_t e);
// returns cuda_fail(h, e) from the enclosing function when a CUDA call fails
#define MB_CUDA(call)                                  \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_fail(h, e_); \
    } while (0)
int upload_proj_tables(mb_handle *h);
cudaError_t smem_limit_once(const void *func, int device, int bytes);

}  // namespace mb
