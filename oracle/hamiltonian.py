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
* a general local potential given by its in-plane Fourier components per z,
  Eqs. (19)-(20): <i|V|i'>(dG) = int B_i B_i' V(z, dG) dz;
* Kleinman-Bylander projectors, Eqs. (14)-(17) and the Z.Q factorization that
  follows them: s (n=1), a real p_x, p_y, p_z set, and optionally the second
  s channel (n=2, beta ~ r^2 exp(-alpha r^2)) whose projection is the sum
  Z_{1,00} Q_{2,00} + Z_{2,00} Q_{1,00} (r^2 split into its in-plane and z
  parts).  The strengths form a Hermitian matrix per atom: E_{nl} on the
  diagonal and an optional 1s-2s coupling (the general E_{nl,n'l'} of GTH).

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
  of size exp(-g_Nyquist^2 / 4a).
"""
from __future__ import annotations

import math

import numpy as np

from .bspline import ZBasis


def reciprocal(a1, a2):
    A = np.array([a1, a2], dtype=np.float64)
    B = 2.0 * np.pi * np.linalg.inv(A).T
    return B[0], B[1]


def wrap(n, N):
    """Integer frequency n mapped into [-N/2, N/2)."""
    return ((np.asarray(n) + N // 2) % N) - N // 2


class Model:
    """One k-point of the slab problem with all matrix-element ingredients."""

    def __init__(self, a1, a2, k, ecut, breaks, order, atoms, grid, nquad=None,
                 local_components=None):
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
            Eb = np.diag(np.array(list(at.E) + ([at.e2s] if at.nproj == 5 else []), dtype=float))
            if at.nproj == 5:
                Eb[0, 4] = Eb[4, 0] = at.e12
            blocks.append(Eb)
        if not Us:
            return np.zeros((0, 0)), np.zeros((0, self.nb, self.ng), dtype=np.complex128)
        n = sum(b.shape[0] for b in blocks)
        E = np.zeros((n, n))
        o = 0
        for b in blocks:
            E[o:o + b.shape[0], o:o + b.shape[0]] = b
            o += b.shape[0]
        return E, np.array(Us)

    # ---- dense matrices -------------------------------------------------
    def dense_S(self):
        return np.kron(self.S, np.eye(self.ng)).astype(np.complex128)

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
        E, U = self.kb_projectors()
        if len(E):
            Uf = U.reshape(len(E), -1).T
            H += Uf @ E @ Uf.conj().T
        return H

    # ---- matrix-free apply (the same elements, contracted directly) ----
    def apply_S(self, X):
        X = np.asarray(X, dtype=np.complex128)
        return np.einsum("ij,bjg->big", self.S, X)

    def apply_H(self, X):
        X = np.asarray(X, dtype=np.complex128)
        Y = 0.5 * np.einsum("ij,bjg->big", self.D, X)
        Y += 0.5 * self.q2[None, None, :] * np.einsum("ij,bjg->big", self.S, X)
        for I, F in self.local_terms():
            Y += np.einsum("ij,bjh,gh->big", I, X, F, optimize=True)
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
        out = np.zeros(len(entries), dtype=np.complex128)
        for n, (b, i, g) in enumerate(entries):
            T = 0.5 * self.D[i] + 0.5 * self.q2[g] * self.S[i]
            v = T @ X[b, :, g]
            for I, F in terms:
                v += I[i] @ X[b] @ F[g]
            if Fp is not None:
                v += U[:, i, g] @ (E @ Fp[:, b])
            out[n] = v
        return out


def model_from_workload(w, ik=0, local_components=None, with_atoms=True):
    """Oracle model for k-point `ik` of a workload description."""
    return Model(w.a1, w.a2, w.kpts[ik], w.ecut, w.breaks, w.order,
                 w.atoms if with_atoms else [], w.grid, w.nquad,
                 local_components=local_components)
