"""The self-consistent loop of §II.B.1 and §III.A, plain FP64.

Test infrastructure only: tests, the package's smoke check and the
benchmark's CPU baseline use it; the library never does.

* Electron density on the quadrature planes (Eq. (6) basis):
      rho(r_par, z_q) = sum_{k,n} f_nk |phi_nk(r_par, z_q)|^2,
      phi = A_c^(-1/2) sum_{G,j} c_{Gj} exp(i (k+G).r_par) B_j(z);
  the k phase drops out of |phi|^2, so on the N1 x N2 grid each band is an
  inverse FFT of sum_j B_j(z_q) c_{Gj} placed at (n1 mod N1, n2 mod N2).
* Coulomb potential of the electrons by the 2D transform of 1/r (the
  Coulomb integral of §II.B.1), on the planes' in-plane components
  rho(z, g) = (1/(N1 N2)) sum_r rho(r, z) exp(-i g.r):
      V_H(z, g) = int dz' rho(z', g) (2 pi / g) exp(-g |z - z'|)      (g != 0)
      V_H(z, 0) = -2 pi int dz' rho(z', 0) |z - z'|
  (at g = 0 the term (2 pi / g) x net charge is dropped, the same reading as
  for the core term: with the core terms' it cancels in a neutral cell).
  The z integral is the Gauss rule of the planes.
* Exchange-correlation: LDA, spin-unpolarized, exchange of the uniform gas
  and the Ceperley-Alder correlation as parametrized by Perdew and Zunger
  (Phys. Rev. B 23, 5048 (1981)), the form the paper cites, evaluated at
  max(rho, RHO_FLOOR): in the vacuum the density falls to values (1e-16 and
  below) that neither FP64 sums nor converged eigenvectors resolve, and the
  cube root of that noise would dominate any change of V_xc; below the floor
  the potential is the small constant v_xc(RHO_FLOOR) (continuous in rho).
* Mixing (§III.A): the paper's Kerker form
      rho_new(z, g) = rho_in(z, g) + W g^2 / (g^2 + g_max^2) (rho_out - rho_in)(z, g)
  on g != 0.  The printed factor is 0 at g = 0, which would freeze the
  planar-average profile rho(z, 0); that profile is mixed with the factor's
  value on the grid's first nonzero shell, W g_1^2 / (g_1^2 + g_max^2), g_1
  the shortest nonzero grid vector.  The mixing stays local in z (each
  component's profile is scaled), so the electron count is kept exactly and
  nothing is smeared into the vacuum, where the LDA potential is most
  sensitive to small densities.  Pulay / RMM-DIIS over the last 4 steps: the
  input densities and residuals R = rho_out - rho_in are combined with
  coefficients summing to 1 that minimize |sum a_i R_i|, and the Kerker step
  is taken from that combination.  Inner product of two (z, g) fields:
  sum_q w_q sum_g Re(conj(a) b).
* Occupations: Fermi-Dirac of width sigma, two electrons per state, k-point
  weights w_k; the chemical potential by bisection on the electron count.
* Convergence (§III.A): the change of V_scf = V_H + V_xc between successive
  iterations, max over the planes' grid points, below tol.
* Ultrasoft atoms (§II.B.2, Eq. for E_nlm,n'l'm'): the strengths of every
  iteration are D_pq = E0_pq + int V_eff Q_pq d^3r with V_eff = V_H + V_xc +
  V_LOC (the tabulated total local potential), i.e. with Q_pq = q_pq g
  (hamiltonian.py), D_pq = E0_pq + q_pq int V_eff g, the integral the grid
  sum sum_q w_q sum_r V g A_c / (N1 N2); the eigenproblem is H c = eps S c
  with the ultrasoft S; and the density is augmented inside the cores,
      rho += sum_atoms g(r) sum_n f_n sum_pq q_pq <phi_n|beta_p><beta_q|phi_n>,
  which keeps the electron count: int rho = sum_n f_n <phi_n|S|phi_n>.
"""
from __future__ import annotations

import math

import numpy as np

from . import eigen as E
from . import hamiltonian as Hm

# Perdew-Zunger (1981) parametrization of the Ceperley-Alder correlation
# energy per electron of the unpolarized gas, in Hartree
PZ_GAMMA, PZ_BETA1, PZ_BETA2 = -0.1423, 1.0529, 0.3334
PZ_A, PZ_B, PZ_C, PZ_D = 0.0311, -0.048, 0.0020, -0.0116
RHO_FLOOR = 1e-10   # bohr^-3: the LDA is evaluated at max(rho, RHO_FLOOR)


def grid_freqs(model):
    """Cartesian g_m and |g_m| for the grid index (u, v), m = wrap(u, v)."""
    N1, N2 = model.grid
    m1 = Hm.wrap(np.arange(N1), N1)
    m2 = Hm.wrap(np.arange(N2), N2)
    g = m1[:, None, None] * model.b1[None, None, :] + m2[None, :, None] * model.b2[None, None, :]
    return g, np.sqrt(np.sum(g * g, axis=-1))


def density(models, coefs, occ):
    """rho(r_par, z_q), shape (nq, N1, N2).

    models: one Model per k-point; coefs[k]: (nbands, nb, ng) coefficients
    c[n, j, G]; occ[k][n]: occupation f_nk (spin and k weight included)."""
    m0 = models[0]
    N1, N2 = m0.grid
    nq = len(m0.zb.zq)
    rho = np.zeros((nq, N1, N2))
    for m, C, f in zip(models, coefs, occ):
        u = m.gidx[:, 0] % N1
        v = m.gidx[:, 1] % N2
        for n in range(C.shape[0]):
            if f[n] == 0.0:
                continue
            psi_q = m.zb.B @ C[n]                       # (nq, ng): sum_j B_j(z_q) c_{Gj}
            grid = np.zeros((nq, N1, N2), dtype=np.complex128)
            grid[:, u, v] = psi_q
            phi = (N1 * N2) * np.fft.ifft2(grid, axes=(1, 2))
            rho += f[n] * np.abs(phi) ** 2 / m.Ac
    return rho


def to_g(field):
    """In-plane components (1/(N1 N2)) sum_r f(r) exp(-i g.r) per plane."""
    return np.fft.fft2(field, axes=(1, 2)) / (field.shape[1] * field.shape[2])


def to_r(comp):
    """The real field with in-plane components `comp` (inverse of to_g)."""
    return (comp.shape[1] * comp.shape[2]) * np.fft.ifft2(comp, axes=(1, 2)).real


def hartree_g(model, rho_g):
    """V_H(z_q, g) from rho(z_q, g) by the Coulomb integral, z integral by the
    planes' Gauss rule (module docstring)."""
    zq, wq = model.zb.zq, model.zb.wq
    _, gn = grid_freqs(model)
    dz = np.abs(zq[:, None] - zq[None, :])               # |z_q - z_q'|
    out = np.zeros_like(rho_g)
    N1, N2 = model.grid
    for u in range(N1):
        for v in range(N2):
            g = gn[u, v]
            K = -2.0 * math.pi * dz if g == 0.0 else (2.0 * math.pi / g) * np.exp(-g * dz)
            out[:, u, v] = K @ (wq * rho_g[:, u, v])
    return out


def xc_pz(rho):
    """(v_xc, eps_xc) per point of a density array (Hartree): LDA exchange
    and the Perdew-Zunger correlation of max(rho, RHO_FLOOR)."""
    n = np.maximum(np.asarray(rho, dtype=np.float64), RHO_FLOOR)
    rs = (3.0 / (4.0 * math.pi * n)) ** (1.0 / 3.0)
    ex = -0.75 * (3.0 * n / math.pi) ** (1.0 / 3.0)
    vx = (4.0 / 3.0) * ex
    ec = np.empty_like(n)
    vc = np.empty_like(n)
    hi = rs >= 1.0
    sr = np.sqrt(rs[hi])
    den = 1.0 + PZ_BETA1 * sr + PZ_BETA2 * rs[hi]
    ec[hi] = PZ_GAMMA / den
    vc[hi] = ec[hi] * (1.0 + (7.0 / 6.0) * PZ_BETA1 * sr + (4.0 / 3.0) * PZ_BETA2 * rs[hi]) / den
    lo = ~hi
    r = rs[lo]
    lr = np.log(r)
    ec[lo] = PZ_A * lr + PZ_B + PZ_C * r * lr + PZ_D * r
    vc[lo] = PZ_A * lr + (PZ_B - PZ_A / 3.0) + (2.0 / 3.0) * PZ_C * r * lr + (2.0 * PZ_D - PZ_C) * r / 3.0
    v = vx + vc
    e = ex + ec
    return v, e


def occupations(evals, kweights, nelec, sigma):
    """Fermi-Dirac occupations f_nk = 2 w_k / (1 + exp((eps - mu)/sigma)) with
    sum f = nelec; mu by bisection.  Returns (f, mu)."""
    ev = np.asarray(evals, dtype=np.float64)
    wk = np.asarray(kweights, dtype=np.float64)[:, None]

    def count(mu):
        x = np.clip((ev - mu) / sigma, -700.0, 700.0)
        return float(np.sum(2.0 * wk / (1.0 + np.exp(x))))

    lo, hi = ev.min() - 40.0 * sigma, ev.max() + 40.0 * sigma
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if count(mid) < nelec:
            lo = mid
        else:
            hi = mid
    mu = 0.5 * (lo + hi)
    x = np.clip((ev - mu) / sigma, -700.0, 700.0)
    return 2.0 * wk / (1.0 + np.exp(x)), mu


def core_density(model):
    """The atoms' Gaussian core charges rho_c on the grid (the start density):
    components (Z/A_c) exp(-g^2 R_c^2/4) exp(-dz^2/R_c^2) / (sqrt(pi) R_c) exp(-i g.R_par)."""
    g, gn = grid_freqs(model)
    c = np.zeros((len(model.zb.zq),) + gn.shape, dtype=np.complex128)
    for at in model.atoms:
        if getattr(at, "Z", 0.0) == 0.0:
            continue
        Rc = at.Rcore
        dz = model.zb.zq - at.pos[2]
        prof = np.exp(-(dz / Rc) ** 2) / (math.sqrt(math.pi) * Rc)
        phase = np.exp(-1j * (g[..., 0] * at.pos[0] + g[..., 1] * at.pos[1]))
        c += (at.Z / model.Ac) * prof[:, None, None] * (np.exp(-0.25 * (gn * Rc) ** 2) * phase)[None]
    return to_r(c)


def atom_gaussian(model, at, R=None):
    """The normalized Gaussian exp(-|r - R|^2/R^2) / (pi^(3/2) R^3) of an atom
    on the grid (radius R, default the atom's augmentation radius rQ)."""
    R = at.rQ if R is None else R
    g, gn = grid_freqs(model)
    dz = model.zb.zq - at.pos[2]
    prof = np.exp(-(dz / R) ** 2) / (math.sqrt(math.pi) * R)
    phase = np.exp(-1j * (g[..., 0] * at.pos[0] + g[..., 1] * at.pos[1]))
    return to_r((1.0 / model.Ac) * prof[:, None, None] * (np.exp(-0.25 * (gn * R) ** 2) * phase)[None])


def grid_integral(model, f):
    """int f d^3r on the planes' grid: sum_q w_q sum_r f A_c / (N1 N2)."""
    N1, N2 = model.grid
    return float(np.sum(model.zb.wq[:, None, None] * f) * model.Ac / (N1 * N2))


def _proj_atoms(model):
    """(atom, first projector index, count) of every atom with projectors."""
    out, o = [], 0
    for at in model.atoms:
        if at.nproj:
            out.append((at, o, at.nproj))
            o += at.nproj
    return out


def uspp_strengths(model, veff):
    """D = E0 + q (int V_eff g) per atom block (§II.B.2)."""
    E0 = Hm._block_diag([Hm._atom_block(at, list(at.E), at.e2s, at.e12) for at in model.atoms if at.nproj])
    Q = model.uspp_q()
    D = E0.copy()
    for at, o, n in _proj_atoms(model):
        if np.any(Q[o:o + n, o:o + n] != 0.0):
            D[o:o + n, o:o + n] += Q[o:o + n, o:o + n] * grid_integral(model, veff * atom_gaussian(model, at))
    return D


def augmentation(models, coefs, occ):
    """sum_atoms g(r) w_atom, w_atom = sum_{k,n} f sum_pq q_pq conj(F_p) F_q,
    F_p = <beta_p|phi> = u_p^H c."""
    m0 = models[0]
    Q = m0.uspp_q()
    atoms = _proj_atoms(m0)
    w = np.zeros(len(atoms))
    for m, C, f in zip(models, coefs, occ):
        _, U = m.kb_projectors()
        F = np.einsum("pjg,njg->np", np.conj(U), C)            # F[n, p]
        for i, (at, o, n) in enumerate(atoms):
            Fa = F[:, o:o + n]
            w[i] += float(np.real(np.einsum("n,np,pq,nq->", f, np.conj(Fa), Q[o:o + n, o:o + n], Fa)))
    rho = np.zeros((len(m0.zb.zq),) + m0.grid)
    for i, (at, o, n) in enumerate(atoms):
        if w[i] != 0.0:
            rho += w[i] * atom_gaussian(m0, at)
    return rho


class Mixer:
    """Kerker + Pulay (RMM-DIIS) over the last `depth` steps (§III.A)."""

    def __init__(self, model, W, gmax, depth=4):
        self.w = model.zb.wq
        _, gn = grid_freqs(model)
        g2 = gn * gn
        g1 = np.min(g2[g2 > 0.0])
        self.K = np.where(g2 > 0.0, W * g2 / (g2 + gmax * gmax), W * g1 / (g1 + gmax * gmax))
        self.depth = depth
        self.hist = []            # (rho_in_g, R_g)

    def kerker(self, R):
        """The Kerker step's factor on every component (module docstring)."""
        return self.K[None, :, :] * R

    def dot(self, a, b):
        return float(np.sum(self.w[:, None, None] * np.real(np.conj(a) * b)))

    def step(self, rho_in, rho_out):
        """New input density (real space) from this step's input and output."""
        ri, ro = to_g(rho_in), to_g(rho_out)
        self.hist.append((ri, ro - ri))
        self.hist = self.hist[-self.depth:]
        m = len(self.hist)
        A = np.zeros((m + 1, m + 1))
        for i in range(m):
            for j in range(m):
                A[i, j] = self.dot(self.hist[i][1], self.hist[j][1])
        A[:m, m] = A[m, :m] = 1.0
        rhs = np.zeros(m + 1)
        rhs[m] = 1.0
        a = np.linalg.lstsq(A, rhs, rcond=None)[0][:m]
        rho_opt = sum(a[i] * self.hist[i][0] for i in range(m))
        R_opt = sum(a[i] * self.hist[i][1] for i in range(m))
        return to_r(rho_opt + self.kerker(R_opt))


def scf(w, nbands, nelec, sigma=0.01, W=0.5, gmax=1.0, tol=1e-7, max_iter=60, kweights=None):
    """Plain SCF on a workload: dense generalized eigensolves per k-point.
    Returns dict(evals (nk, nbands), rho, vscf, iterations, dv)."""
    nk = w.nk
    kw = np.full(nk, 1.0 / nk) if kweights is None else np.asarray(kweights, dtype=np.float64)
    base = [Hm.model_from_workload(w, ik) for ik in range(nk)]
    rho_in = core_density(base[0])
    mixer = Mixer(base[0], W, gmax)
    vprev = None
    dv = math.inf
    it = 0
    uspp = base[0].uspp
    for it in range(1, max_iter + 1):
        vh = to_r(hartree_g(base[0], to_g(rho_in)))
        vxc, _ = xc_pz(rho_in)
        vscf = vh + vxc
        dv = math.inf if vprev is None else float(np.abs(vscf - vprev).max())
        vprev = vscf
        D = None
        if uspp:
            D = uspp_strengths(base[0], Hm.model_from_workload(w, 0, table=vscf).local_table())
        models = [Hm.model_from_workload(w, ik, table=vscf, strengths=D) for ik in range(nk)]
        evals, coefs = [], []
        for m in models:
            ev, C = E.generalized_lowest(m.dense_H(), m.dense_S(), nbands, vectors=True)
            evals.append(ev)
            coefs.append(C.T.reshape(nbands, m.nb, m.ng))
        evals = np.array(evals)
        if dv < tol:
            break
        f, _ = occupations(evals, kw, nelec, sigma)
        rho_out = density(models, coefs, f)
        if uspp:
            rho_out = rho_out + augmentation(models, coefs, f)
        rho_in = mixer.step(rho_in, rho_out)
    return {"evals": evals, "rho": rho_in, "vscf": vscf, "iterations": it, "dv": dv, "strengths": D}
