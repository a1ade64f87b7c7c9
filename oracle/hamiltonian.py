"""Matrix elements of S and H in the mixed basis (§II.B.1), FP64.

Basis (Eq. (6)): <r|k+G; j> = A^{-1/2} exp(i(k+G).r_par) B_j(z), with G in
the cutoff disc |k+G|^2/2 <= Ecut (Hartree) and j over the retained
B-splines.  A coefficient block is X[band][j][G] (G fastest); the flattened
basis index is j*N_G + g.

Elements, in Hartree (the paper's Rydberg -nabla^2 becomes -nabla^2/2):
* overlap, Eqs. (7)-(8):     S = delta_GG' <B_i|B_i'>
* kinetic, Eq. (9):          T = delta_GG' [ 1/2 <B_i'|B_i''> + 1/2 |k+G|^2 <B_i|B_i'> ]
* local Gaussian part of the pseudopotential, Eqs. (10)-(13):
      V = sum_atoms I(i; a, R_z; i') exp(-i dG.R_par) (A/A_c)(pi/a) exp(-|dG|^2/4a)
  with I by the z quadrature and dG wrapped onto the in-plane FFT grid (the
  grid on which the potential is tabulated; see ``wrap``);
* the core term -Z erf(r/R_c)/r of Eq. (10): the Coulomb potential of the
  Gaussian core charge rho_c, taken through the 2D transform of 1/r as in the
  Coulomb integral of §II.B.1; its in-plane components depend on z and g
  together (``core_term``), so its elements are
      <i|V_core|i'>(dG) = sum_q w_q B_i(z_q) B_i'(z_q) V_core(z_q, dG)
  (the general local-potential form, Eqs. (19)-(20));
* a general local potential given by its in-plane Fourier components per z,
  Eqs. (19)-(20): <i|V|i'>(dG) = int B_i B_i' V(z, dG) dz;
* Kleinman-Bylander projectors, Eqs. (14)-(17) and the Z.Q factorization that
  follows them: s (n=1), a real p_x, p_y, p_z set, and optionally the second
  s channel (n=2, beta ~ r^2 exp(-alpha r^2)) whose projection is the sum
  Z_{1,00} Q_{2,00} + Z_{2,00} Q_{1,00} (r^2 split into its in-plane and z
  parts).  The strengths form a Hermitian matrix per atom: E_{nl} on the
  diagonal and an optional 1s-2s coupling (the general E_{nl,n'l'} of GTH).
* ultrasoft pseudopotentials (§II.B.2): the overlap becomes
      S = S_0 + sum_pq q_pq u_p u_q^H,  q_pq = int Q_pq(r) d^3r,
  and the strengths E_pq are the self-consistent ones of the loop (``scf``).
  With the paper's restriction Q_pq(r) = Q_{nl,n'l'}(r) Y_LM, L = min |l - l'|,
  only pairs whose L = 0 part survives integrate to nonzero q: in the real
  p_x, p_y, p_z basis those are (s, s), (2s, 2s), (1s, 2s) and (p_i, p_i),
  the pattern of the KB strengths.  The radial parts are synthetic (no
  Vanderbilt files are at hand): Q_pq(r) = q_pq g(r), g the normalized
  Gaussian exp(-r^2/r_Q^2) / (pi^(3/2) r_Q^3) of the atom;

Readings:
* Gaussian local term A exp(-|r-R|^2/(2 w^2)), i.e. a = 1/(2 w^2);
* projector radius r_c means alpha = 1/(2 r_c^2);
* the p channel uses real x, y, z angular factors: any unitary mix of the m
  components gives the same sum_m |beta_m><beta_m|.  The in-plane transform of
  x exp(-alpha r^2) carries a factor i that the printed Q_{1,1+-1} omits; it is
  a constant phase per projector and cancels in |beta><beta|;
* C normalizes each projector to int |beta|^2 d^3r = 1;
* one Gaussian radius per atom: alpha_0 = alpha_1 = 1 / (2 r_c^2);
* dG is wrapped to the grid frequency range [-N/2, N/2) per axis, which is what
  a product on an N1 x N2 grid computes; the unwrapped element differs by terms
  of size exp(-g_Nyquist^2 / 4a);
* the core term's sign is the one Eq. (10) prints (attractive for Z > 0); the
  Coulomb integral's rho carries the electron's sign convention;
* the core term at g = 0: (2 pi/g) times the cell's net core charge diverges
  as g -> 0 and does not depend on z; it is dropped (in a neutral cell it
  cancels against the electrons' Hartree term, and a constant only shifts
  every eigenvalue by itself).  The z-dependent remainder,
  +(2 pi/A_c) int dz' rho_c(z') |z - z'|, is kept;
* the core term is tabulated on the grid as a real potential, so a coefficient
  enters as (c(m) + conj(c(-m))) / 2, with -m wrapped; this is c(m) itself for
  every m but those on the Nyquist row or column, where -m wraps onto m.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf, erfc, erfcx

from .bspline import ZBasis


def reciprocal(a1, a2):
    A = np.array([a1, a2], dtype=np.float64)
    B = 2.0 * np.pi * np.linalg.inv(A).T
    return B[0], B[1]


def wrap(n, N):
    """Integer frequency n mapped into [-N/2, N/2)."""
    return ((np.asarray(n) + N // 2) % N) - N // 2


def core_term(g, dz, Z, Rc, Ac):
    """In-plane Fourier component of the core term -Z erf(r/R_c)/r of Eq. (10)
    at in-plane wavevector magnitude g and height dz above the atom, per unit
    cell area (the convention of Eq. (13)).

    The core term is the potential of the Gaussian core charge
    rho_c(r) = Z exp(-r^2/R_c^2) / (pi^(3/2) R_c^3); with the 2D transform of
    1/r (the Coulomb integral of §II.B.1) its component at g is
        -(2 pi / g) int dz' rho_c(z', g) exp(-g |dz - z'|),
        rho_c(z', g) = (Z / A_c) exp(-g^2 R_c^2 / 4) exp(-z'^2 / R_c^2) / (sqrt(pi) R_c),
    which integrates in closed form to
        -(Z / A_c) (pi / g) [T(dz) + T(-dz)],  T(z) = exp(g z) erfc(g R_c / 2 + z / R_c).
    Where the erfc argument x is >= 0, T is written exp(-g^2 R_c^2/4 - z^2/R_c^2) erfcx(x)
    (g z - x^2 = -g^2 R_c^2 / 4 - z^2 / R_c^2), which cannot overflow.
    g = 0: the divergent constant is dropped (module docstring) and
        +(2 pi Z / A_c) [dz erf(dz / R_c) + (R_c / sqrt(pi)) exp(-dz^2 / R_c^2)]
    is kept."""
    g, dz = np.broadcast_arrays(np.asarray(g, dtype=np.float64), np.asarray(dz, dtype=np.float64))
    out = np.empty(g.shape)
    zero = g == 0.0
    z0 = dz[zero]
    out[zero] = (2.0 * math.pi * Z / Ac) * (z0 * erf(z0 / Rc) + Rc / math.sqrt(math.pi) * np.exp(-(z0 / Rc) ** 2))
    gp, zp = g[~zero], dz[~zero]

    def T(z):
        x = 0.5 * gp * Rc + z / Rc
        t = np.empty(x.shape)
        pos = x >= 0.0
        t[pos] = np.exp(-0.25 * (gp[pos] * Rc) ** 2 - (z[pos] / Rc) ** 2) * erfcx(x[pos])
        t[~pos] = np.exp(gp[~pos] * z[~pos]) * erfc(x[~pos])
        return t

    out[~zero] = -(Z / Ac) * (math.pi / gp) * (T(zp) + T(-zp))
    return out


class Model:
    """One k-point of the slab problem with all matrix-element ingredients."""

    def __init__(self, a1, a2, k, ecut, breaks, order, atoms, grid, nquad=None,
                 local_components=None, table=None, strengths=None):
        self.a1 = np.asarray(a1, dtype=np.float64)
        self.a2 = np.asarray(a2, dtype=np.float64)
        self.k = np.asarray(k, dtype=np.float64)
        self.ecut = float(ecut)
        self.grid = (int(grid[0]), int(grid[1]))
        self.zb = ZBasis(breaks, order, nquad)
        self.nb = self.zb.nb
        self.b1, self.b2 = reciprocal(self.a1, self.a2)
        self.Ac = abs(self.a1[0] * self.a2[1] - self.a1[1] * self.a2[0])
        self.atoms = list(atoms)
        self.local_components = list(local_components or [])
        # an extra local potential tabulated on the grid, V(r_par, z_q) of shape
        # (nq, N1, N2) (the general local potential of Eqs. (19)-(20); the SCF
        # loop puts V_H + V_xc here)
        self.table = None if table is None else np.asarray(table, dtype=np.float64)
        # strengths E_pq replacing the atoms' (the self-consistent D of the
        # ultrasoft loop), same layout as kb_projectors' E
        self.strengths = None if strengths is None else np.asarray(strengths, dtype=np.float64)
        self._sphere()
        self.S = self.zb.overlap()
        self.D = self.zb.stiffness()

    # ---- basis set (Eq. (6)) -------------------------------------------
    def _sphere(self):
        r = math.sqrt(2.0 * self.ecut)
        bmin = min(np.linalg.norm(self.b1), np.linalg.norm(self.b2))
        # |n_i| is bounded by (r + |k|) * |a_i| / (2 pi)
        lim1 = int(math.ceil((r + np.linalg.norm(self.k)) * np.linalg.norm(self.a1) / (2 * math.pi))) + 1
        lim2 = int(math.ceil((r + np.linalg.norm(self.k)) * np.linalg.norm(self.a2) / (2 * math.pi))) + 1
        idx = []
        for n1 in range(-lim1, lim1 + 1):
            for n2 in range(-lim2, lim2 + 1):
                q = self.k + n1 * self.b1 + n2 * self.b2
                if 0.5 * (q[0] * q[0] + q[1] * q[1]) <= self.ecut:
                    idx.append((n1, n2))
        del bmin
        self.gidx = np.array(idx, dtype=np.int64).reshape(-1, 2)
        self.ng = len(self.gidx)
        self.q = self.k[None, :] + self.gidx[:, :1] * self.b1[None, :] + self.gidx[:, 1:] * self.b2[None, :]
        self.q2 = np.sum(self.q * self.q, axis=1)

    @property
    def nbasis(self):
        return self.nb * self.ng

    def _dG_wrapped(self):
        """Wrapped integer differences G - G' and their cartesian vectors."""
        d1 = wrap(self.gidx[:, None, 0] - self.gidx[None, :, 0], self.grid[0])
        d2 = wrap(self.gidx[:, None, 1] - self.gidx[None, :, 1], self.grid[1])
        g = d1[..., None] * self.b1 + d2[..., None] * self.b2
        return d1, d2, g

    # ---- local potential (Eqs. (10)-(13), (19)-(20)) -------------------
    def local_terms(self):
        """List of (I (nb x nb), F (ng x ng)) with V = sum_terms I (x) F, i.e.
        V[(G,i),(G',i')] = sum I[i,i'] F[G,G'].

        Atoms sharing the same Gaussian (A, a) and height R_z share I; their
        in-plane factors are summed (the distributive law on Eq. (12))."""
        terms = []
        if self.atoms:
            d1, d2, g = self._dG_wrapped()
            g2 = np.sum(g * g, axis=-1)
            groups = {}
            for at in self.atoms:
                if at.A == 0.0:
                    continue
                a = 1.0 / (2.0 * at.w * at.w)
                key = (at.A, a, at.pos[2])
                phase = np.exp(-1j * (g[..., 0] * at.pos[0] + g[..., 1] * at.pos[1]))
                F = (at.A / self.Ac) * (math.pi / a) * np.exp(-g2 / (4.0 * a)) * phase
                groups[key] = groups.get(key, 0) + F
            for (A, a, Rz), F in groups.items():
                I = self.zb.weighted(np.exp(-a * (self.zb.zq - Rz) ** 2))
                terms.append((I, F))
        if self.local_components:
            d1 = wrap(self.gidx[:, None, 0] - self.gidx[None, :, 0], self.grid[0])
            d2 = wrap(self.gidx[:, None, 1] - self.gidx[None, :, 1], self.grid[1])
            for (m1, m2, fz) in self.local_components:
                F = ((d1 == wrap(m1, self.grid[0])) & (d2 == wrap(m2, self.grid[1]))).astype(np.complex128)
                I = self.zb.weighted(np.array([fz(z) for z in self.zb.zq]))
                terms.append((I, F))
        return terms

    def core_table(self):
        """Core-term components V_core(z_q, m) for every grid frequency m, shape
        (nq, N1, N2), index u standing for m = wrap(u): the atoms' sum of
        ``core_term`` times exp(-i g_m . R_par), as coefficients of a real
        table on the grid.  None when no atom has a core term."""
        ions = [at for at in self.atoms if getattr(at, "Z", 0.0) != 0.0]
        if not ions:
            return None
        N1, N2 = self.grid
        m1 = wrap(np.arange(N1), N1)
        m2 = wrap(np.arange(N2), N2)
        g = m1[:, None, None] * self.b1[None, None, :] + m2[None, :, None] * self.b2[None, None, :]
        gn = np.sqrt(np.sum(g * g, axis=-1))
        tab = np.zeros((len(self.zb.zq), N1, N2), dtype=np.complex128)
        for at in ions:
            if not at.Rcore > 0.0:
                raise ValueError("a core term needs Rcore > 0")
            phase = np.exp(-1j * (g[..., 0] * at.pos[0] + g[..., 1] * at.pos[1]))
            prof = core_term(gn[None, :, :], (self.zb.zq - at.pos[2])[:, None, None], at.Z, at.Rcore, self.Ac)
            tab += prof * phase[None, :, :]
        neg = tab[:, (-np.arange(N1)) % N1][:, :, (-np.arange(N2)) % N2]
        return 0.5 * (tab + np.conj(neg))

    def local_table(self):
        """The local potential V(r_par, z_q), shape (nq, N1, N2), on the grid
        r_par = (i1/N1) a1 + (i2/N2) a2: the sum over grid frequencies m of
        the Gaussian components (Eq. (13)) and the core components, each
        times exp(i g_m . r_par), by numpy's inverse FFT, plus the extra
        table when there is one."""
        N1, N2 = self.grid
        m1 = wrap(np.arange(N1), N1)
        m2 = wrap(np.arange(N2), N2)
        g = m1[:, None, None] * self.b1[None, None, :] + m2[None, :, None] * self.b2[None, None, :]
        g2 = np.sum(g * g, axis=-1)
        c = np.zeros((len(self.zb.zq), N1, N2), dtype=np.complex128)
        for at in self.atoms:
            if at.A == 0.0:
                continue
            a = 1.0 / (2.0 * at.w * at.w)
            phase = np.exp(-1j * (g[..., 0] * at.pos[0] + g[..., 1] * at.pos[1]))
            F = (at.A / self.Ac) * (math.pi / a) * np.exp(-g2 / (4.0 * a)) * phase
            c += np.exp(-a * (self.zb.zq - at.pos[2]) ** 2)[:, None, None] * F[None, :, :]
        Vc = self.core_table()
        if Vc is not None:
            c += Vc
        V = (N1 * N2) * np.fft.ifft2(c, axes=(1, 2)).real
        return V if self.table is None else V + self.table

    def nonsep_table(self):
        """Components on every grid frequency of the local terms that depend
        on z and g together: the core term and the extra table (its
        coefficients (1/(N1 N2)) sum_r V(r) exp(-i g_m . r) by numpy's FFT).
        None when there are neither."""
        Vc = self.core_table()
        if self.table is not None:
            N1, N2 = self.grid
            T = np.fft.fft2(self.table, axes=(1, 2)) / (N1 * N2)
            Vc = T if Vc is None else Vc + T
        return Vc

    def _core_index(self):
        """Flat grid index (u * N2 + v) of the wrapped G - G' of every pair."""
        d1, d2, _ = self._dG_wrapped()
        return (d1 % self.grid[0]) * self.grid[1] + (d2 % self.grid[1])

    # ---- Kleinman-Bylander projectors (Eqs. (14)-(17), Z.Q factors) ----
    def kb_projectors(self):
        """(E (nproj, nproj), U (nproj, nb, ng)) with V_NL = sum_pq E_pq u_p u_q^H.

        Per atom the projectors are 1s, p_x, p_y, p_z and (nproj == 5) 2s; E
        is block diagonal over atoms, diagonal but for the 1s-2s coupling."""
        Es, Us, blocks = [], [], []
        for at in self.atoms:
            if at.nproj == 0:
                continue
            alpha = 1.0 / (2.0 * at.rc * at.rc)
            Rz = at.pos[2]
            dz = self.zb.zq - Rz
            gz = np.exp(-alpha * dz * dz)
            Z0 = self.zb.B.T @ (self.zb.wq * gz)            # Z_{1,00}, Z_{1,1+-1}
            Z1 = self.zb.B.T @ (self.zb.wq * dz * gz)       # Z_{1,10}
            Z2 = self.zb.B.T @ (self.zb.wq * dz * dz * gz)  # Z_{2,00}
            Qs = (math.pi / alpha) * np.exp(-self.q2 / (4.0 * alpha))
            Qx = 1j * (self.q[:, 0] / (2.0 * alpha)) * Qs
            Qy = 1j * (self.q[:, 1] / (2.0 * alpha)) * Qs
            Q2 = (1.0 / alpha - self.q2 / (4.0 * alpha * alpha)) * Qs   # Q_{2,00}
            Cs = (2.0 * alpha / math.pi) ** 0.75
            Cp = 2.0 * math.sqrt(alpha) * Cs
            # int (r^2)^2 exp(-2 alpha r^2) d^3r = 4 pi (15/16) sqrt(pi) (2 alpha)^{-7/2}
            C2 = (4.0 * math.pi * 15.0 / 16.0 * math.sqrt(math.pi) * (2.0 * alpha) ** -3.5) ** -0.5
            phase = np.exp(-1j * (self.q[:, 0] * at.pos[0] + self.q[:, 1] * at.pos[1]))
            fs = [Cs * np.outer(Z0, Qs), Cp * np.outer(Z0, Qx),
                  Cp * np.outer(Z0, Qy), Cp * np.outer(Z1, Qs),
                  C2 * (np.outer(Z0, Q2) + np.outer(Z2, Qs))]
            if at.nproj not in (4, 5):
                raise ValueError("nproj must be 0, 4 or 5")
            for p in range(at.nproj):
                Us.append(phase[None, :] * np.conj(fs[p]) / math.sqrt(self.Ac))
            blocks.append(_atom_block(at, list(at.E), at.e2s, at.e12))
        if not Us:
            return np.zeros((0, 0)), np.zeros((0, self.nb, self.ng), dtype=np.complex128)
        E = _block_diag(blocks)
        if self.strengths is not None:
            E = self.strengths
        return E, np.array(Us)

    def uspp_q(self):
        """q_pq of the ultrasoft overlap (§II.B.2), kb_projectors' layout."""
        return _block_diag([_atom_block(at, list(getattr(at, "q", (0.0,) * 4)), getattr(at, "q2s", 0.0),
                                        getattr(at, "q12", 0.0)) for at in self.atoms if at.nproj])

    @property
    def uspp(self):
        Q = self.uspp_q()
        return Q.size > 0 and bool(np.any(Q != 0.0))

    # ---- dense matrices -------------------------------------------------
    def dense_S(self):
        S = np.kron(self.S, np.eye(self.ng)).astype(np.complex128)
        if self.uspp:
            _, U = self.kb_projectors()
            Uf = U.reshape(U.shape[0], -1).T
            S += Uf @ self.uspp_q() @ Uf.conj().T
        return S

    def dense_H(self):
        n = self.nbasis
        H = np.zeros((n, n), dtype=np.complex128)
        # kinetic: block diagonal in G
        for g in range(self.ng):
            T = 0.5 * self.D + 0.5 * self.q2[g] * self.S
            ix = np.arange(self.nb) * self.ng + g
            H[np.ix_(ix, ix)] += T
        for I, F in self.local_terms():
            H += np.kron(I, F)
        Vc = self.nonsep_table()
        if Vc is not None:
            # one z matrix per distinct wrapped dG: I_m = sum_q w_q B B V_core(z_q, m)
            ms, inv = np.unique(self._core_index(), return_inverse=True)
            Vq = Vc.reshape(Vc.shape[0], -1)[:, ms]
            Im = np.einsum("q,qi,qm,qj->mij", self.zb.wq, self.zb.B, Vq, self.zb.B)
            blk = Im[inv.reshape(self.ng, self.ng)]                  # [g, g', i, i']
            H += blk.transpose(2, 0, 3, 1).reshape(n, n)
        E, U = self.kb_projectors()
        if len(E):
            Uf = U.reshape(len(E), -1).T
            H += Uf @ E @ Uf.conj().T
        return H

    # ---- matrix-free apply (the same elements, contracted directly) ----
    def apply_S(self, X):
        X = np.asarray(X, dtype=np.complex128)
        Y = np.einsum("ij,bjg->big", self.S, X)
        if self.uspp:
            _, U = self.kb_projectors()
            Fp = np.einsum("pjg,bjg->pb", np.conj(U), X)
            Y += np.einsum("pjg,pb->bjg", U, self.uspp_q() @ Fp)
        return Y

    def apply_H(self, X):
        X = np.asarray(X, dtype=np.complex128)
        Y = 0.5 * np.einsum("ij,bjg->big", self.D, X)
        Y += 0.5 * self.q2[None, None, :] * np.einsum("ij,bjg->big", self.S, X)
        for I, F in self.local_terms():
            Y += np.einsum("ij,bjh,gh->big", I, X, F, optimize=True)
        Vc = self.nonsep_table()
        if Vc is not None:
            # per plane: psi_q(G') = sum_i' B_i'(z_q) X(i', G'), then the
            # in-plane sum over G' with V_core(z_q, G - G'), then sum_q w_q B_i(z_q)
            idx = self._core_index()
            psi = np.einsum("qj,bjg->qbg", self.zb.B, X)
            Vf = Vc.reshape(Vc.shape[0], -1)
            out = np.empty_like(psi)
            for q in range(psi.shape[0]):
                out[q] = psi[q] @ Vf[q][idx].T
            Y += np.einsum("q,qi,qbg->big", self.zb.wq, self.zb.B, out)
        E, U = self.kb_projectors()
        if len(E):
            Fp = np.einsum("pjg,bjg->pb", np.conj(U), X)      # u_q^H X
            Y += np.einsum("pjg,pb->bjg", U, E @ Fp)           # sum_pq u_p E_pq (u_q^H X)
        return Y

    def apply_H_entries(self, X, entries):
        """Selected entries Y[b, i, g] of H X, each one a row of H times X."""
        X = np.asarray(X, dtype=np.complex128)
        terms = self.local_terms()
        E, U = self.kb_projectors()
        Fp = np.einsum("pjg,bjg->pb", np.conj(U), X) if len(E) else None
        Vc = self.nonsep_table()
        if Vc is not None:
            idx = self._core_index()
            psi = np.einsum("qj,bjg->qbg", self.zb.B, X)
            Vf = Vc.reshape(Vc.shape[0], -1)
        out = np.zeros(len(entries), dtype=np.complex128)
        for n, (b, i, g) in enumerate(entries):
            T = 0.5 * self.D[i] + 0.5 * self.q2[g] * self.S[i]
            v = T @ X[b, :, g]
            for I, F in terms:
                v += I[i] @ X[b] @ F[g]
            if Vc is not None:
                v += np.sum(self.zb.wq * self.zb.B[:, i] * np.sum(Vf[:, idx[g]] * psi[:, b, :], axis=1))
            if Fp is not None:
                v += U[:, i, g] @ (E @ Fp[:, b])
            out[n] = v
        return out


def _atom_block(at, diag, d2s, d12):
    """One atom's block: diag over 1s, p_x, p_y, p_z (and 2s), the 1s-2s
    coupling off the diagonal."""
    b = np.diag(np.array(list(diag) + ([d2s] if at.nproj == 5 else []), dtype=float))
    if at.nproj == 5:
        b[0, 4] = b[4, 0] = d12
    return b


def _block_diag(blocks):
    n = sum(b.shape[0] for b in blocks)
    M = np.zeros((n, n))
    o = 0
    for b in blocks:
        M[o:o + b.shape[0], o:o + b.shape[0]] = b
        o += b.shape[0]
    return M


def model_from_workload(w, ik=0, local_components=None, with_atoms=True, table=None, strengths=None):
    """Oracle model for k-point `ik` of a workload description."""
    return Model(w.a1, w.a2, w.kpts[ik], w.ecut, w.breaks, w.order,
                 w.atoms if with_atoms else [], w.grid, w.nquad,
                 local_components=local_components, table=table, strengths=strengths)
