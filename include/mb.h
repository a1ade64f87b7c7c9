/* mb.h -- C ABI of the GB300 mixed-basis (2D plane wave x B-spline) library.
 *
 * The library applies the Kohn-Sham Hamiltonian H and the overlap S of the
 * mixed basis of Ren, Hsue and Chang (arXiv:1406.4960) to blocks of trial
 * vectors on one CUDA device, and solves H c = eps S c for the lowest roots
 * with the generalized Lanczos-Krylov iteration of their §II.C.
 *
 * Basis (§II.B.1, Eq. (6)):  <r|k+G; j> = A^{-1/2} exp(i(k+G).r_par) B_j(z)
 * with G in the disc |k+G|^2/2 <= Ecut and B_j the order-kappa B-splines of
 * §II.A on a clamped knot sequence, the first and last spline dropped (zero
 * boundary values).  Units: Hartree and bohr.
 *
 * Coefficient blocks.  A block of `nbands` vectors at k-point ik is a device
 * array of complex numbers, interleaved (re, im), laid out
 *     X[band][j][g]      band < nbands, j < nb, g < ldg
 * with g fastest.  Only g < ng(ik) are basis functions; the padding columns
 * ng <= g < ldg are ignored on input and written as zero on output.  The
 * element type is double2 for MB_FP64 and float2 for MB_FP32 / MB_BF16.
 * The G order inside the disc is the library's; mb_gvectors() reports it.
 * All device pointers are owned by the caller; the handle owns its tables.
 *
 * Errors.  Every call returns MB_OK (0) or an MB_E* code; nothing aborts.
 * Calls on one handle must not overlap (one host thread per handle).
 * Streams are passed as `void*` holding a cudaStream_t (NULL = the legacy
 * default stream).  Device pointers must be 16-byte aligned.
 */
#ifndef MB_H
#define MB_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mb_handle mb_handle;

enum {
    MB_OK = 0,
    MB_EINVAL = 1,      /* bad argument: sizes, ik, knots, grid too small for the disc */
    MB_ENOMEM = 2,      /* device or host allocation failed */
    MB_ENOTCONV = 3,    /* eigensolver did not reach tol within max_cycles */
    MB_ETIMEOUT = 4,    /* a bounded device-side wait expired */
    MB_ECUDA = 5,       /* a CUDA runtime call failed (see mb_last_cuda_error) */
    MB_EUNSUPPORTED = 6 /* valid request that the library does not implement */
};

/* Arithmetic of an apply.  MB_FP64: every step in double.  MB_FP32: B-spline
 * evaluation, FFTs, potential product, banded terms and projector
 * contraction in float.  MB_BF16: as MB_FP32, but the two projector
 * contractions run on the tensor cores with bf16 operands and float
 * accumulation. */
typedef enum { MB_FP64 = 0, MB_FP32 = 1, MB_BF16 = 2 } mb_prec;

/* In-plane lattice vectors (bohr). */
typedef struct { double a1[2]; double a2[2]; } mb_cell;

/* One atom of the surface unit cell.
 * Local pseudopotential (§II.B.1, Eq. (10)):
 *     -Z erf(|r - pos| / Rcore) / |r - pos|  +  A * exp(-|r - pos|^2 / (2 w^2))
 * (Z in units of e, Rcore and w in bohr, A in Ha; Z = 0 or A = 0 drops the
 * term).  The core term is the Coulomb potential of a Gaussian core charge;
 * its in-plane g = 0 component diverges like 2 pi Z / (A_c g) and that
 * z-independent constant is dropped, keeping
 *     +(2 pi Z / A_c) [dz erf(dz / Rcore) + (Rcore / sqrt(pi)) exp(-dz^2 / Rcore^2)],
 * dz = z - pos[2] (a constant shifts every eigenvalue by itself; in a neutral
 * cell the electrons' Hartree term cancels it).
 * Ultrasoft augmentation (§II.B.2; used when any q is nonzero): the overlap
 * becomes S = S_0 + sum q_pq |beta_p><beta_q| over the atom's projectors,
 * q[0..3] for 1s, p_x, p_y, p_z, q2s for 2s and q12 for the 1s-2s pair (the
 * pairs whose augmentation charge Q_{nl,n'l'}(r) Y_LM with L = min|l - l'|
 * integrates to nonzero in the real p basis), with the synthetic charge
 * shape Q_pq(r) = q_pq exp(-r^2/rQ^2) / (pi^(3/2) rQ^3) (rQ > 0 in bohr).
 * mb_scf makes the strengths self-consistent, D_pq = E_pq + int V_eff Q_pq,
 * and augments the density; mb_apply_S includes the term; mb_apply_Sinv
 * returns MB_EUNSUPPORTED for such a handle.
 * Kleinman-Bylander projectors (Eq. (14)), GTH Gaussian radial parts with
 * alpha = 1 / (2 rc^2) for every channel: nproj = 0 (none), 4 (1s, p_x, p_y,
 * p_z) or 5 (the same and the second s channel, beta ~ r^2 exp(-alpha r^2),
 * whose projection is Z_{1,00} Q_{2,00} + Z_{2,00} Q_{1,00}), each normalized
 * to unit norm.  Strengths in Ha: E[0..3] for 1s, p_x, p_y, p_z (a physical p
 * channel has E[1] = E[2] = E[3]), E2s for 2s and E12 for the 1s-2s coupling
 * (the off-diagonal element of GTH's h matrix; used when nproj = 5). */
typedef struct {
    double pos[3];
    double A;
    double w;
    int nproj;
    double E[4];
    double rc;
    double E2s;
    double E12;
    double Z;
    double Rcore;
    double q[4];
    double q2s;
    double q12;
    double rQ;
} mb_atom;

typedef struct {
    int n1, n2;        /* in-plane FFT grid; powers of two in [4, 256], each
                          at least 2*max|n_i| + 1 over the discs of all k */
    int nquad;         /* Gauss-Legendre points per knot interval (0: order) */
    int device;        /* CUDA device ordinal */
    int max_bands;     /* largest block passed to the apply calls (0: 128);
                          sizes the handle's scratch */
    double precond_shift; /* c of the eigensolver's (T(G) + c S)^-1 (0: 1 Ha) */
} mb_opts;

/* Build the basis and every device table for `nk` k-points.
 *   cell     in-plane lattice
 *   kpts     nk x 2 cartesian in-plane wave vectors (1/bohr), host
 *   ecut     plane-wave cutoff on |k+G|^2/2 (Ha)
 *   breaks   nbreaks strictly increasing z breakpoints (bohr), host; the
 *            knot sequence is clamped (end breakpoints repeated `order` times),
 *            so there are n_int = nbreaks - 1 intervals and
 *            nb = n_int + order - 3 retained B-splines
 *   order    B-spline order kappa in [3, 8]; n_int >= order
 *   atoms    natoms atoms (host); may be NULL when natoms == 0
 *   opts     grid, quadrature and device (host, required)
 * Cites: §II.A (knots, Eqs. (1)-(3)), §II.B.1 (Eqs. (6)-(17)).
 * Errors: MB_EINVAL, MB_ENOMEM, MB_ECUDA.  *out is NULL on failure. */
int mb_setup(const mb_cell *cell, const double *kpts, int nk, double ecut,
             const double *breaks, int nbreaks, int order,
             const mb_atom *atoms, int natoms, const mb_opts *opts,
             mb_handle **out);

/* Release everything the handle owns.  NULL is ignored.  The work queued on
 * the handle's calls must have completed (synchronize the streams passed to
 * it first; mb_eigsolve returns with its own work done).  Device memory of the
 * handle -- tables and apply scratch -- is allocated and freed stream-ordered
 * from the library's memory pool on the handle's own streams, so neither
 * mb_setup nor mb_destroy waits for other work on the device; the pool keeps
 * up to 16 GiB of freed memory reserved for the next handle. */
void mb_destroy(mb_handle *h);

/* Sizes at k-point ik: disc size ng, retained B-splines nb, padded stride
 * ldg (a multiple of 32).  Any output pointer may be NULL. */
int mb_sizes(const mb_handle *h, int ik, int *ng, int *nb, int *ldg);

/* Integer coordinates (n1, n2) of G = n1 b1 + n2 b2 for each g < ng in the
 * library's order: idx[2*g], idx[2*g+1].  Host buffer of 2*ng ints. */
int mb_gvectors(const mb_handle *h, int ik, int *idx);

/* Number of z quadrature planes (n_int * nquad) and, if the pointers are not
 * NULL, their abscissae and weights (host buffers of that length). */
int mb_zplanes(const mb_handle *h, int *nq, double *zq, double *wq);

/* Replace the local potential by a caller-given real table
 * V[q][i1][i2] = V(r_par = i1/n1 a1 + i2/n2 a2, z_q) in Ha on the quadrature
 * planes (host, nq*n1*n2 doubles) -- the general local potential of
 * §II.B.1, Eqs. (19)-(20).  Projectors are unchanged.  Waits for all work on
 * the device first (queued applies may still read the old table). */
int mb_set_local_potential(mb_handle *h, const double *V);

/* The local potential the applies use, in mb_set_local_potential's layout
 * (host buffer of nq*n1*n2 doubles).  mb_setup builds it on the device from
 * the atoms' terms: V(r_par, z_q) = Re sum_m c(m, z_q) exp(i g_m . r_par)
 * over the grid frequencies m in [-n/2, n/2) per axis, c the sum over atoms
 * of each term's in-plane component times exp(-i g_m . pos_par) -- Eq. (13)
 * for the Gaussian, the Coulomb integral of §II.B.1 of the Gaussian core
 * charge for the core term (see mb_atom).  Blocks until the copy is done.
 * Errors: MB_EINVAL (NULL arguments), MB_ECUDA. */
int mb_local_potential(mb_handle *h, double *V);

/* Y = H X at k-point ik (§II.B.1: kinetic Eq. (9), local potential through
 * in-plane FFTs on the quadrature planes, Kleinman-Bylander Eq. (17)).
 * X and Y are distinct device blocks of nbands (1 <= nbands <= max_bands)
 * in the element type of `prec`.  Asynchronous on `stream`. */
int mb_apply_H(mb_handle *h, int ik, const void *X, void *Y, int nbands,
               int prec, void *stream);

/* Y = H X for several k-points in one pass: X[i], Y[i] are the blocks of
 * k-point iks[i] (host arrays of nsel device pointers). */
int mb_apply_H_batch(mb_handle *h, int nsel, const int *iks,
                     const void *const *X, void *const *Y, int nbands,
                     int prec, void *stream);

/* ---- H apply without device allocation --------------------------------
 * The paper has no counterpart to this call; it exists for callers of this
 * library that must not allocate device memory while they run -- for example
 * code whose device memory is a fixed budget handed out by its own pool, or a
 * pipeline that cannot afford the device-wide synchronization that cudaMalloc
 * and cudaFree may cause.  mb_apply_H grows a scratch buffer owned by the
 * handle on demand (cudaMalloc); this variant computes the same Y = H X for
 * one k-point with its scratch in an array of MB_NOALLOC_SCRATCH_BYTES
 * compiled into the library instead.  It calls no cudaMalloc, cudaFree or
 * other allocating routine; the caller still passes X and Y (device, layout
 * and element type as for mb_apply_H), and the handle must already exist.
 *
 *   - The array is a file-scope __device__ object: every GPU on which the
 *     library's device code is loaded holds it until the process exits.
 *   - Each call made outside stream capture looks the array's address up on
 *     the handle's device (cudaGetSymbolAddress); a call inside a capture
 *     uses the address of the last uncaptured call on that device, so make
 *     the first call on a device before any stream capture (a first call
 *     inside a capture returns MB_EINVAL).
 *   - Every call, from every handle, shares the one array and leaves its
 *     contents behind.  Nothing in it has to start at zero (each element is
 *     written before it is read), but calls whose work overlaps on the GPU --
 *     different streams, or several host threads -- race on it: serialize them.
 *   - Returns MB_EINVAL when the request needs more scratch than the array
 *     holds (it fits, for example, a 32-band FP32 apply of a 179-G, 120-spline
 *     slab k-point), and the other MB_E* codes of mb_apply_H. */
#define MB_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
int mb_apply_H_noalloc(mb_handle *h, int ik, const void *X, void *Y, int nbands,
                       int prec, void *stream);

/* Y = S X (§II.B.1, Eqs. (7)-(8): S is G-diagonal and banded in j). */
int mb_apply_S(mb_handle *h, int ik, const void *X, void *Y, int nbands,
               int prec, void *stream);

/* Y = S^-1 X from the banded Cholesky factor of the G-independent S_z. */
int mb_apply_Sinv(mb_handle *h, int ik, const void *X, void *Y, int nbands,
                  int prec, void *stream);

/* S X and S^-1 X for several k-points in one launch: X[i], Y[i] are the
 * blocks of k-point iks[i] (host arrays of nsel distinct device pointers;
 * X[i] and Y[i] must not overlap).  Each (k-point, band, 32-column) tile of
 * X -- for S, a run of 32 rows of it and its halo -- is brought into shared
 * memory by TMA bulk copies; if their bounded wait expires the tile's output
 * is not written and mb_status reports MB_ETIMEOUT. */
int mb_apply_S_batch(mb_handle *h, int nsel, const int *iks, const void *const *X,
                     void *const *Y, int nbands, int prec, void *stream);
int mb_apply_Sinv_batch(mb_handle *h, int nsel, const int *iks, const void *const *X,
                        void *const *Y, int nbands, int prec, void *stream);

/* Synchronizes the handle's device and reports whether a bounded device-side
 * wait in an asynchronous call of this handle ran out since the last check
 * (MB_ETIMEOUT: the outputs of that call are not valid) or not (MB_OK);
 * clears the record. */
int mb_status(mb_handle *h);

typedef struct {
    int cycles;           /* grand cycles used (§II.C) */
    int applies;          /* vectors multiplied by H */
    double max_residual;  /* max_i ||H x_i - eps_i S x_i||_{S^-1} at exit */
    double seconds;       /* wall time of the call */
    int finish_cycles;    /* of `cycles`, those run with FP64 root applies (all
                             of them for MB_FP64; the finish phase otherwise) */
} mb_solve_info;

typedef struct {
    int krylov_depth;     /* k of K = span{v, A v, ..., A^k v} (0: 5) */
    int block;            /* roots per block in the second grand cycle (0: 1) */
    int max_cycles;       /* (0: 200) */
    int polish;           /* reserved (0) */
    int guard;            /* extra roots carried above the requested ones
                             (0: max(2, ceil(nbands/8)); negative: none) */
    int warm_start;       /* nonzero: evecs holds start vectors for the nbands
                             roots (any basis of a nearby subspace, e.g. the
                             roots of a previous potential); they replace the
                             lowest free-electron states of the cold start */
} mb_solve_opts;

/* Lowest `nbands` roots of H c = eps S c at every k-point (§II.C).
 *   prec   MB_FP64: every step in double ("plain").  MB_FP32 / MB_BF16:
 *          bulk cycles with every vector step in FP32 (applies in that
 *          precision, Gram products on the tensor cores, small dense
 *          problems in FP32 or FP64), then finish cycles with FP64 roots
 *          until the FP64 residual < tol.
 *   tol    residual tolerance ||H x - eps S x||_{S^-1} (Ha)
 *   evals  host, nk*nbands doubles, ascending per k
 *   evecs  optional device pointer (NULL: not returned): nk blocks of
 *          nbands double2 vectors, block ik at offset sum_{i<ik} nbands*nb*ldg(i)
 *   sopts  optional (NULL: defaults); info optional.
 * Returns MB_ENOTCONV (evals still written) if max_cycles is reached,
 * MB_ETIMEOUT if a tensor-core kernel's bounded device wait expired (its
 * products are then not valid and the solve stops). */
int mb_eigsolve(mb_handle *h, int nbands, double tol, int prec, double *evals,
                void *evecs, const mb_solve_opts *sopts, mb_solve_info *info,
                void *stream);

/* ---- the self-consistent loop (§II.B.1 and §III.A) ---------------------
 * Fields on the quadrature planes are device arrays of nq*n1*n2 doubles in
 * mb_set_local_potential's layout, f[q][i1][i2] at r_par = i1/n1 a1 + i2/n2 a2.
 *
 * Electron density rho = sum_{k,n} f_nk |phi_nk|^2 of the coefficient blocks
 * evecs (device, the layout of mb_eigsolve's evecs: nk blocks of nbands
 * vectors [band][j][ldg]) with occupations occ (host, nk*nbands, spin and
 * k-point weight included); phi is the basis expansion of Eq. (6) with
 * A = A_c.  FP64; deterministic (partials summed in a fixed order).  The
 * caller's stream is synchronized before return (occ is read from the host).
 * Errors: MB_EINVAL (NULL pointers, nbands < 1), MB_EUNSUPPORTED (a grid
 * whose FP64 plane does not fit in shared memory), MB_ECUDA. */
int mb_density(mb_handle *h, const void *evecs, int nbands, const double *occ, double *rho, void *stream);

/* Coulomb potential of an electron density, V_H(r) = int rho(r')/|r - r'|,
 * through the 2D transform of 1/r (the Coulomb integral of §II.B.1): per
 * in-plane component g, V(z, g) = int dz' rho(z', g) (2 pi/g) exp(-g|z - z'|),
 * the z integral by the planes' Gauss rule; at g = 0 the z-independent
 * divergence (2 pi/g) x net charge is dropped, keeping
 * -2 pi int dz' rho(z', 0) |z - z'| (with the atoms' core terms, which drop
 * theirs, a neutral cell loses nothing).  rho and vh: device fields.  The
 * stream is synchronized before return.  Errors as mb_density's. */
int mb_hartree(mb_handle *h, const double *rho, double *vh, void *stream);

/* LDA exchange-correlation potential v_xc and energy per electron exc
 * (optional, may be NULL) of a density: exchange of the uniform gas and the
 * Ceperley-Alder correlation as parametrized by Perdew and Zunger (Phys. Rev.
 * B 23, 5048 (1981)), spin-unpolarized, evaluated at max(rho, 1e-10 bohr^-3)
 * (in the vacuum the density falls below what FP64 sums and converged
 * eigenvectors resolve; there the potential is the small constant of the
 * floor).  Device fields; asynchronous on the stream.  Errors: MB_EINVAL
 * (NULL rho or vxc), MB_ECUDA. */
int mb_xc_lda(mb_handle *h, const double *rho, double *vxc, double *exc, void *stream);

typedef struct {
    int nbands;           /* roots per k-point (room above nelec/2 for the smearing) */
    double nelec;         /* electrons per cell (<= 0: the atoms' sum of Z, a neutral cell) */
    double sigma;         /* Fermi-Dirac width (Ha), > 0 */
    double mix_weight;    /* W of the Kerker mixing (0: 0.5) */
    double g_max;         /* Kerker cutoff wave vector (1/bohr) (0: 1) */
    int pulay_depth;      /* steps Pulay combines, at most 8 (0: 4; 1: Kerker alone) */
    double tol;           /* stop when max |change of V_H + V_xc| < tol (Ha) */
    int max_iter;         /* eigensolves at most (0: 60) */
    double eig_tol;       /* residual tolerance of the eigensolves (0: tol / 10); while the
                             potential still changes by dv, an iteration solves to
                             max(eig_tol, min(dv / 10, 1e-3)) */
    int prec;             /* MB_FP64 or MB_FP32 (mixed-precision eigensolves) */
    const double *kweights; /* host, nk weights summing to 1 (NULL: uniform) */
} mb_scf_opts;

typedef struct {
    int iterations;       /* eigensolves run */
    double dv;            /* last max |change of V_H + V_xc| (Ha) */
    double mu;            /* Fermi level of the last occupations (Ha) */
    double nelec;         /* electrons in the final input density */
    int eig_cycles;       /* grand cycles over all eigensolves */
    double seconds, seconds_eig, seconds_density, seconds_potential;
} mb_scf_info;

/* Self-consistent field (§II.B.1, §III.A).  Starting from the atoms' Gaussian
 * core charges as the electron density, each iteration adds V_scf = V_H + V_xc
 * of the input density to the atoms' local potential, solves for the lowest
 * nbands roots (mb_eigsolve), fills them with Fermi-Dirac occupations and
 * mixes the output density into the next input: the paper's Kerker form
 * W g^2/(g^2 + g_max^2) on g != 0 (the g = 0 profile, which that factor
 * would freeze, scaled by the factor of the grid's first nonzero shell: the
 * mixing stays local in z and keeps the electron count) from the Pulay
 * combination of the last pulay_depth steps that minimizes the residual.  Stops when V_scf changes by
 * less than tol (§III.A's criterion).  evals: host nk*nbands, the roots of
 * the final potential; rho_out: optional device field, the final input
 * density.  The handle's local potential holds the final total potential on
 * return (and, with ultrasoft atoms, its projector strengths the final D);
 * its later applies and eigensolves use them.  Errors: MB_EINVAL (nbands < 1,
 * sigma or tol not positive, a precision other than MB_FP64 / MB_FP32, no
 * electrons or more than 2 nbands of them, weights not summing to 1),
 * MB_ENOTCONV when max_iter is reached (evals still written), the errors of
 * mb_eigsolve and mb_density. */
int mb_scf(mb_handle *h, const mb_scf_opts *opts, double *evals, double *rho_out, mb_scf_info *info);

/* ---- launch-shape autotuner -------------------------------------------
 * Times the plane kernel's candidate launch shapes for an apply of `nbands`
 * bands at all k-points of the handle, on scratch blocks it allocates, and
 * keeps the fastest for later applies and eigensolves of that shape.  The
 * candidates: in FP32, every compiled instance of the compact-plane kernel
 * that can run the batch (they differ in threads and bands per CTA, CTAs per
 * SM and where the window of X rows lives), each as a static grid and as a
 * persistent launch fed by a device work queue; the register-FFT / radix-2
 * kernels with 1-4 bands per CTA; each with the built-in run count and with
 * explicit wave targets.  Set-up time call (allocates; not during stream
 * capture).  best_bt: bands per CTA of a register-FFT / radix-2 choice, or
 * -1 - id for compact-plane instance `id` (mb_plane_kernel_name names it).
 * best_waves = 0 means the built-in wave model chose the run length (CTA
 * count rounded to whole waves of resident CTAs); > 0, a target of that many
 * CTAs per resident slot.  Outputs may be NULL. */
int mb_autotune(mb_handle *h, int nbands, int prec, int *best_bt, int *best_waves,
                double *best_ms);

/* Name of the plane-kernel instance that an apply of `nbands` bands at
 * k-points 0 .. nk-1 (at most 64) in precision `prec` launches with the
 * handle's current tuning, written to buf (host, len bytes, truncated and
 * NUL-terminated). */
int mb_plane_kernel_name(const mb_handle *h, int nk, int nbands, int prec, char *buf, int len);

/* The candidates the last mb_autotune of this handle timed, one line each
 * (kernel instance, bands per CTA, wave target, ms per apply), written to buf
 * (host, len bytes, truncated and NUL-terminated). */
int mb_autotune_report(const mb_handle *h, char *buf, int len);

/* The compact-plane kernel instances (FP32 and BF16 applies) that can run an
 * apply of k-points 0 .. nk-1: their ids are written to ids (host, at most
 * `max`); returns how many there are (0 for MB_FP64), or -MB_EINVAL. */
int mb_plane_kernel_candidates(const mb_handle *h, int nk, int nbands, int prec, int *ids, int max);

/* Fix the plane-kernel choice for applies of that shape instead of timing
 * it: id >= 0 a compact-plane instance from mb_plane_kernel_candidates,
 * -1 the default choice, -2 the register-FFT / radix-2 kernels; waves as
 * mb_autotune reports it (0: the built-in run count); persistent != 0: the
 * compact-plane kernel's persistent launch, one CTA per resident slot taking
 * (k-point, band tile, interval run) items from a device work queue.
 * MB_EINVAL for an id that cannot run the batch. */
int mb_plane_kernel_select(mb_handle *h, int nk, int nbands, int prec, int id, int waves,
                           int persistent);

/* ---- continuous-batching solve server ---------------------------------
 * Serves mb_eigsolve requests of mixed sizes on one device.  Submitted
 * requests queue; `slots` worker threads admit them whenever a slot is idle
 * and the request's device footprint (basis tables, apply scratch, Krylov
 * workspace -- computed exactly from a host-side set-up of its basis) fits in
 * what is left of `hbm_budget_bytes`, first fit over the queue.  Each
 * admitted request keeps its own handle and stream, so requests that arrive
 * while others run are admitted as memory frees up and their work overlaps
 * on the device.  Results do not depend on the mix (private state, fixed
 * reduction orders).  The request's arrays are copied at submission. */
typedef struct mb_server mb_server;
typedef struct {
    mb_cell cell;
    const double *kpts;   /* nk x 2 */
    int nk;
    double ecut;
    const double *breaks;
    int nbreaks;
    int order;
    const mb_atom *atoms;
    int natoms;
    mb_opts opts;         /* device is overridden by the server's */
    int nbands;
    double tol;
    int prec;
} mb_request;

int mb_server_create(int device, int slots, double hbm_budget_bytes, mb_server **out);
/* MB_ENOMEM if the request could never fit the budget. */
int mb_server_submit(mb_server *srv, const mb_request *req, long long *ticket);
/* Blocks until the request completes (timeout_s <= 0: no limit; otherwise
 * MB_ETIMEOUT after that many seconds, the request still pending).  evals:
 * host nk*nbands doubles; latency_s: submission to completion; phases: host
 * array of 3 (queue wait, set-up of the request's handle, solve and
 * teardown), seconds, summing to latency_s.  Outputs may be NULL.  Returns
 * the request's own status (that of mb_setup / mb_eigsolve). */
int mb_server_wait(mb_server *srv, long long ticket, double *evals, mb_solve_info *info,
                   double *latency_s, double *phases, double timeout_s);
int mb_server_stats(mb_server *srv, int *queued, int *running, int *peak_running,
                    double *bytes_in_use, double *peak_bytes);
/* Finishes every queued and running request, then frees the server. */
void mb_server_destroy(mb_server *srv);

/* ---- instrumentation ------------------------------------------------
 * Every kernel the library launches is counted per handle.  With profiling
 * on (mb_set_profiling: 0 off, 1 every kernel, 2 the plane kernel only, whose
 * two events per apply leave the rest of the step undisturbed), each
 * profiled launch is also bracketed by CUDA events on its own stream; the
 * per-kernel totals accumulate until mb_profile_reset.  Kernel ids:
 * 0 plane, 1 epilogue, 2 proj, 3 coef, 4 backproj, 5 banded, 6 gram,
 * 7 combine, 8 jacobi, 9 small, 10 vec, 11 gram32, 12 combine32 (the FP32
 * Gram-Schmidt products of the mixed-precision eigensolver); mb_kernel_name
 * gives the names. */
int mb_set_profiling(mb_handle *h, int on);
int mb_profile_read(mb_handle *h, int kernel, double *ms_total, long long *count);
int mb_profile_reset(mb_handle *h);
long long mb_launch_count(const mb_handle *h);
const char *mb_kernel_name(int kernel);

/* Message for an error code (static storage). */
const char *mb_strerror(int code);

/* The last CUDA error string seen by this handle (static storage, or ""). */
const char *mb_last_cuda_error(const mb_handle *h);

#ifdef __cplusplus
}
#endif
#endif /* MB_H */
