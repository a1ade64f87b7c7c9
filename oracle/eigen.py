"""Generalized eigenproblem H c = eps S c (§II.C), FP64 oracle.

* ``jacobi_herm``       cyclic complex Jacobi (``jacobi.c``, plain C) -- the
                        diagonalizer the paper uses for every subspace matrix.
* ``generalized_lowest`` the definition of the result: S = L L^H,
                        H~ = L^{-1} H L^{-H}, lowest eigenvalues of H~.  The
                        Hermitian step runs through ``jacobi_herm`` for small
                        orders and LAPACK (a library routine) above
                        ``JACOBI_MAX``; both are pinned against each other.
* ``lanczos_krylov``    the generalized Lanczos-Krylov iteration with its two
                        alternating grand cycles.

Readings of §II.C (the paper leaves them open):
* The Krylov operator for the generalized problem is A = P (H - theta S) for
  the seed vector's Ritz value theta, with P an SPD solve that is G-diagonal
  and banded in j.  P = S^{-1} gives the Krylov space of S^{-1} H itself
  (shift-invariance); the default P = (T(G) + c S)^{-1} (kinetic operator of
  each plane wave plus a constant shift c) keeps the stiff z-kinetic spectrum
  of the B-spline basis from stalling the iteration.
* Krylov vectors are built Arnoldi-style (each new vector S-orthogonalized,
  classical Gram-Schmidt applied twice, against all current roots and the
  previous Krylov vectors) -- the same span as {v, Av, ..., A^k v}.
* Depth k = 4, block size 8 in the second cycle; the seed of each Krylov
  space is the trial vector with the largest residual.
* Root selection in a block: the b Ritz vectors with the largest
  sum_j |<y|S|x_j>|^2 over the block's inputs; a Ritz vector whose value lies
  below the block's lowest input value and whose overlap is below 1/2 is a
  new root: it replaces the selected vector with the highest value.
* Converged when every residual ||H x - eps S x||_{S^-1} < tol over the
  requested roots.  g = max(2, ceil(M/8)) guard roots above them are
  carried along (and seeded from the free-electron start) so that a root the
  trial set misses is captured instead of the iteration settling on a
  higher one.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

JACOBI_MAX = 600
_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None


def build_jacobi():
    """Compile jacobi.c into oracle/_build/libjacobi.so (plain gcc)."""
    out_dir = os.path.join(_HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, "libjacobi.so")
    src = os.path.join(_HERE, "jacobi.c")
    if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", so, src, "-lm"])
    return so


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build_jacobi())
        _lib.oracle_jacobi_herm.restype = ctypes.c_int
        _lib.oracle_jacobi_herm.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_double, ctypes.c_int]
    return _lib


def jacobi_herm(A, rel_tol=1e-15, max_sweeps=60, vectors=True):
    """Eigenvalues (ascending) and eigenvectors of a Hermitian matrix by
    cyclic Jacobi rotations."""
    A = np.array(A, dtype=np.complex128, order="C", copy=True)
    n = A.shape[0]
    w = np.zeros(n)
    V = np.zeros((n, n), dtype=np.complex128) if vectors else None
    rc = _load().oracle_jacobi_herm(n, A.ctypes.data, w.ctypes.data,
                                    V.ctypes.data if vectors else None, rel_tol, max_sweeps)
    if rc == -2:
        raise MemoryError("jacobi: allocation failed")
    return (w, V) if vectors else w


def hermitian_eig(A, vectors=True):
    if A.shape[0] <= JACOBI_MAX:
        return jacobi_herm(A, vectors=vectors)
    if vectors:
        return np.linalg.eigh(A)
    return np.linalg.eigvalsh(A)


def generalized_lowest(H, S, m=None, vectors=False):
    """Lowest m eigenpairs of H c = eps S c by Cholesky reduction."""
    L = np.linalg.cholesky(S)
    Li = np.linalg.inv(L)
    Ht = Li @ H @ Li.conj().T
    Ht = 0.5 * (Ht + Ht.conj().T)
    if vectors:
        w, Y = hermitian_eig(Ht, vectors=True)
        C = Li.conj().T @ Y
        m = len(w) if m is None else m
        return w[:m], C[:, :m]
    w = hermitian_eig(Ht, vectors=False)
    return w if m is None else w[:m]


# ---------------------------------------------------------------------------
# generalized Lanczos-Krylov (§II.C)
# ---------------------------------------------------------------------------
class BlockOps:
    """Operators on flat vectors (columns of an (n, m) array) for one model."""

    def __init__(self, model, precond="kinetic", shift=None):
        self.m = model
        nb, ng = model.nb, model.ng
        self.shape = (nb, ng)
        self.Sfac = np.linalg.cholesky(model.S)
        if precond == "overlap":
            self.P = None
        else:
            c = 1.0 if shift is None else shift
            self.Pfac = [np.linalg.cholesky(0.5 * model.D + (0.5 * model.q2[g] + c) * model.S)
                         for g in range(ng)]
            self.P = True

    def _blk(self, V):
        nb, ng = self.shape
        return V.T.reshape(V.shape[1], nb, ng)

    def _flat(self, Y):
        return Y.reshape(Y.shape[0], -1).T

    def H(self, V):
        return self._flat(self.m.apply_H(self._blk(V)))

    def S(self, V):
        return self._flat(self.m.apply_S(self._blk(V)))

    def Sinv(self, V):
        Y = self._blk(V).copy()
        L = self.Sfac
        for b in range(Y.shape[0]):
            Y[b] = np.linalg.solve(L.conj().T, np.linalg.solve(L, Y[b]))
        return self._flat(Y)

    def prec(self, V):
        if self.P is None:
            return self.Sinv(V)
        Y = self._blk(V).copy()
        for g, L in enumerate(self.Pfac):
            Y[:, :, g] = np.linalg.solve(L.conj().T, np.linalg.solve(L, Y[:, :, g].T)).T
        return self._flat(Y)


def _s_orth_against(w, Q, SQ):
    """Classical Gram-Schmidt, twice, of w against S-orthonormal columns Q."""
    for _ in range(2):
        if Q.shape[1]:
            w = w - Q @ (SQ.conj().T @ w)
    return w


def _krylov(ops, v, theta, Qbase, SQbase, depth):
    """Arnoldi-style basis of span{A v, ..., A^depth v}, A = P (H - theta S),
    S-orthonormal and S-orthogonal to Qbase."""
    Q, SQ = Qbase, SQbase
    new, newS = [], []
    cur = v
    for _ in range(depth):
        w = ops.prec(ops.H(cur[:, None]) - theta * ops.S(cur[:, None]))[:, 0]
        w = _s_orth_against(w, Q, SQ)
        sw = ops.S(w[:, None])[:, 0]
        nrm = np.sqrt(max(np.real(np.vdot(w, sw)), 0.0))
        if nrm < 1e-12:
            break
        w = w / nrm
        sw = sw / nrm
        new.append(w)
        newS.append(sw)
        Q = np.hstack([Q, w[:, None]])
        SQ = np.hstack([SQ, sw[:, None]])
        cur = w
    if not new:
        return np.zeros((v.shape[0], 0), dtype=v.dtype), np.zeros((v.shape[0], 0), dtype=v.dtype)
    return np.array(new).T, np.array(newS).T


def s_orthonormalize(ops, X):
    """Column-by-column Gram-Schmidt (twice) in the S inner product."""
    Q = np.zeros((X.shape[0], 0), dtype=np.complex128)
    SQ = Q.copy()
    for c in range(X.shape[1]):
        w = _s_orth_against(X[:, c].astype(np.complex128), Q, SQ)
        sw = ops.S(w[:, None])[:, 0]
        nrm = np.sqrt(max(np.real(np.vdot(w, sw)), 0.0))
        if nrm < 1e-12:
            continue
        Q = np.hstack([Q, (w / nrm)[:, None]])
        SQ = np.hstack([SQ, (sw / nrm)[:, None]])
    return Q, SQ


def _rayleigh_ritz(V, HV):
    Hs = V.conj().T @ HV
    Hs = 0.5 * (Hs + Hs.conj().T)
    return jacobi_herm(Hs)


def select_roots(w, Y, b, eps_in):
    """Maximum-overlap choice of b Ritz pairs in a block, plus new roots.

    <y_l|S|x_j> = Y[j, l] because the block's inputs are the first b columns of
    an S-orthonormal basis."""
    ov = np.sum(np.abs(Y[:b, :]) ** 2, axis=0)
    chosen = list(np.argsort(-ov, kind="stable")[:b])
    lowest_in = float(np.min(eps_in))
    for l in range(len(w)):
        if l in chosen:
            continue
        if w[l] < lowest_in and ov[l] < 0.5:
            worst = max(chosen, key=lambda c: w[c])
            if w[l] < w[worst]:
                chosen[chosen.index(worst)] = l
    chosen.sort(key=lambda c: w[c])
    return Y[:, chosen], w[chosen]


def residual_norms(ops, X, HX, SX, eps):
    R = HX - SX * eps[None, :]
    SiR = ops.Sinv(R)
    return np.sqrt(np.maximum(np.real(np.sum(np.conj(R) * SiR, axis=0)), 0.0))


def default_guard(nroots):
    return max(2, -(-nroots // 8))


def lanczos_krylov(ops, X0, nroots, depth=4, block=8, tol=1e-8, max_cycles=300,
                   history=None, guard=None):
    """Lowest `nroots` eigenpairs of H c = eps S c from trial vectors X0 (n, m0).

    `guard` extra roots are carried along (X0 needs nroots + guard columns)
    and only the lowest `nroots` are tested for convergence and returned.
    Returns (eps, X, info) with X S-orthonormal."""
    nconv = nroots
    nroots = nroots + (default_guard(nroots) if guard is None else guard)
    X, SX = s_orthonormalize(ops, X0)
    HX = ops.H(X)
    w, Y = _rayleigh_ritz(X, HX)
    X, SX, HX = X @ Y, SX @ Y, HX @ Y
    eps = w.copy()
    M = nroots
    X, SX, HX, eps = X[:, :M], SX[:, :M], HX[:, :M], eps[:M]
    res = residual_norms(ops, X, HX, SX, eps)
    cycles = 0
    for cycles in range(1, max_cycles + 1):
        # --- cycle A: all roots + one Krylov space, seeded at the worst
        # root among those that are tested for convergence
        i = int(np.argmax(res[:nconv]))
        K, SK = _krylov(ops, X[:, i], eps[i], X, SX, depth)
        V = np.hstack([X, K])
        SV = np.hstack([SX, SK])
        HV = np.hstack([HX, ops.H(K)]) if K.shape[1] else HX
        w, Y = _rayleigh_ritz(V, HV)
        X, SX, HX, eps = V @ Y[:, :M], SV @ Y[:, :M], HV @ Y[:, :M], w[:M].copy()
        # --- cycle B: blocks of roots, each with its own Krylov space.  The
        # blocks are independent: every Krylov space is S-orthogonalized
        # against the roots as they stand when the cycle starts.
        Xc, SXc, HXc, epsc = X.copy(), SX.copy(), HX.copy(), eps.copy()
        res_all = residual_norms(ops, Xc, HXc, SXc, epsc)
        for b0 in range(0, M, block):
            blk = list(range(b0, min(M, b0 + block)))
            seed = blk[int(np.argmax(res_all[blk]))]
            K, SK = _krylov(ops, Xc[:, seed], epsc[seed], Xc, SXc, depth)
            if K.shape[1] == 0:
                continue
            V = np.hstack([Xc[:, blk], K])
            SV = np.hstack([SXc[:, blk], SK])
            HV = np.hstack([HXc[:, blk], ops.H(K)])
            w, Y = _rayleigh_ritz(V, HV)
            Yc, wc = select_roots(w, Y, len(blk), epsc[blk])
            X[:, blk], SX[:, blk], HX[:, blk] = V @ Yc, SV @ Yc, HV @ Yc
            eps[blk] = wc
        # keep the set ordered and S-orthonormal for the next cycle A
        X, SX = s_orthonormalize(ops, X)
        HX = ops.H(X)
        w, Y = _rayleigh_ritz(X, HX)
        X, SX, HX, eps = X @ Y, SX @ Y, HX @ Y, w.copy()
        res = residual_norms(ops, X, HX, SX, eps)
        if history is not None:
            history.append((cycles, eps[:nconv].copy(), res[:nconv].copy()))
        if np.max(res[:nconv]) < tol:
            break
    return eps[:nconv], X[:, :nconv], {"cycles": cycles, "residuals": res[:nconv]}
