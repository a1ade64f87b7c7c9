"""Pins for the oracle's eigen-solvers (§II.C): the Jacobi diagonalizer against
LAPACK, the Cholesky-reduced generalized problem against scipy's generalized
solver, and the Lanczos-Krylov iteration against the dense definition."""
import dataclasses

import numpy as np
import pytest
import scipy.linalg as sl

from oracle import eigen as E
from oracle import hamiltonian as Hm
from paper_1406_4960_gb300 import workloads as W


@pytest.mark.parametrize("n", [1, 2, 5, 40, 130])
def test_jacobi_matches_lapack(n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = A + A.conj().T
    w, V = E.jacobi_herm(A)
    assert np.all(np.diff(w) >= 0)
    assert np.abs(w - np.linalg.eigvalsh(A)).max() < 1e-12 * max(1.0, np.abs(w).max())
    assert np.abs(V.conj().T @ V - np.eye(n)).max() < 1e-12
    assert np.abs(A @ V - V * w[None, :]).max() < 1e-11 * max(1.0, np.abs(w).max())


def test_jacobi_degenerate_and_diagonal():
    D = np.diag([3.0, 1.0, 1.0, -2.0]).astype(complex)
    w, V = E.jacobi_herm(D)
    assert np.allclose(w, [-2, 1, 1, 3])
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.standard_normal((6, 6)) + 1j * rng.standard_normal((6, 6)))
    A = Q @ np.diag([1, 1, 1, 2, 2, 5.0]) @ Q.conj().T
    w = E.jacobi_herm(A, vectors=False)
    assert np.abs(w - [1, 1, 1, 2, 2, 5]).max() < 1e-13


def test_generalized_reduction_matches_scipy():
    rng = np.random.default_rng(4)
    n = 50
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    H = A + A.conj().T
    B = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    S = B @ B.conj().T + n * np.eye(n)
    w = E.generalized_lowest(H, S, 10)
    assert np.abs(w - sl.eigh(H, S, eigvals_only=True)[:10]).max() < 1e-12
    w2, C = E.generalized_lowest(H, S, 10, vectors=True)
    assert np.abs(C.conj().T @ S @ C - np.eye(10)).max() < 1e-11
    assert np.abs(H @ C - S @ C * w2[None, :]).max() < 1e-10


def _free_electron_start(m, M):
    ez, cz = sl.eigh(0.5 * m.D, m.S)
    cand = sorted((0.5 * m.q2[g] + ez[n], g, n) for g in range(m.ng) for n in range(4))
    X0 = np.zeros((m.nbasis, M), dtype=complex)
    for c, (_, g, n) in enumerate(cand[:M]):
        v = np.zeros((m.nb, m.ng), dtype=complex)
        v[:, g] = cz[:, n]
        X0[:, c] = v.reshape(-1)
    return X0


def test_lanczos_krylov_matches_dense_tiny():
    w = W.tiny()
    m = Hm.model_from_workload(w)
    ref = E.generalized_lowest(m.dense_H(), m.dense_S(), w.nbands)
    ops = E.BlockOps(m)
    eps, X, info = E.lanczos_krylov(ops, _free_electron_start(m, w.nbands + E.default_guard(w.nbands)), w.nbands, tol=1e-8)
    assert info["residuals"].max() < 1e-8
    assert np.abs(eps - ref).max() < 1e-10
    SX = ops.S(X)
    assert np.abs(X.conj().T @ SX - np.eye(w.nbands)).max() < 1e-10


def test_lanczos_krylov_with_projectors_and_k():
    w = dataclasses.replace(W.scaled(W.slab(), ecut=3.0, n_int=21, nbands=6),
                            kpts=W.slab().kpts[2:3])
    m = Hm.model_from_workload(w)
    ref = E.generalized_lowest(m.dense_H(), m.dense_S(), 6)
    ops = E.BlockOps(m)
    eps, X, info = E.lanczos_krylov(ops, _free_electron_start(m, 6 + E.default_guard(6)), 6, block=3, tol=1e-8)
    assert np.abs(eps - ref).max() < 1e-10


def test_lanczos_krylov_overlap_operator_is_the_literal_krylov_space():
    """With P = S^{-1} the Krylov space is that of S^{-1} H; it still converges
    (slowly) on a small case."""
    w = dataclasses.replace(W.tiny(), ecut=4.0, breaks=W.uniform_breaks(-8, 8, 11))
    m = Hm.model_from_workload(w)
    ref = E.generalized_lowest(m.dense_H(), m.dense_S(), 4)
    ops = E.BlockOps(m, precond="overlap")
    eps, X, info = E.lanczos_krylov(ops, _free_electron_start(m, 4 + E.default_guard(4)), 4, depth=6, block=2,
                                    tol=1e-7, max_cycles=400)
    assert np.abs(eps - ref).max() < 1e-9
