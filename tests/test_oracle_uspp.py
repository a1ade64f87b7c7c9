"""Pins for the oracle's ultrasoft terms (§II.B.2): the overlap
S = S_0 + sum q |beta><beta|, the self-consistent strengths
D = E0 + int V_eff Q, and the augmented density, against exact identities
(the electron count of generalized-orthonormal states, the normalization of
the augmentation charge, a constant potential) and the self-consistency of a
converged loop."""
import dataclasses
import math

import numpy as np
import pytest

from oracle import eigen as E
from oracle import hamiltonian as Hm
from oracle import scf as F
from paper_1406_4960_gb300 import workloads as W


def _cell(q=(0.6, 0.3, 0.3, 0.3), nk=2, rQ=0.7, nproj=4, q2s=0.0, q12=0.0):
    a = 4.2
    atoms = [W.Atom((0.7, 1.1, -0.6), -0.5, 0.8, nproj, (0.4, -0.2, -0.2, -0.2), 0.9, e2s=-0.1, e12=0.05,
                    Z=1.0, Rcore=0.5, q=q, q2s=q2s, q12=q12, rQ=rQ),
             W.Atom((2.9, 3.0, 0.7), -0.5, 0.8, nproj, (0.4, -0.2, -0.2, -0.2), 0.9, e2s=-0.1, e12=0.05,
                    Z=1.0, Rcore=0.5, q=q, q2s=q2s, q12=q12, rQ=rQ)]
    k = np.array([[0.0, 0.0], [0.31, -0.2]][:nk])
    return W.Workload("uspp", (a, 0.0), (0.35 * a, 0.93 * a), k, 4.0, W.uniform_breaks(-7.0, 7.0, 15),
                      6, 6, (16, 16), atoms, 4)


def test_overlap_structure():
    """Hermitian and positive definite; q = 0 gives S_0; the added term has
    the rank of the nonzero q entries (one s channel per atom here)."""
    m = Hm.model_from_workload(_cell(q=(0.6, 0.0, 0.0, 0.0)))
    S, S0 = m.dense_S(), np.kron(m.S, np.eye(m.ng))
    assert np.abs(S - S.conj().T).max() < 1e-13
    assert np.linalg.eigvalsh(S).min() > 0
    sv = np.linalg.svd(S - S0, compute_uv=False)
    assert sv[1] > 1e-6 * sv[0] and sv[2] < 1e-12 * sv[0]        # two atoms: rank 2
    m0 = Hm.model_from_workload(_cell(q=(0.0, 0.0, 0.0, 0.0)))
    assert np.abs(m0.dense_S() - S0).max() == 0.0
    X = W.random_block(3, m.nb, m.ng, seed=4)
    Y = m.apply_S(X)
    Yd = (S @ X.reshape(3, -1).T).T.reshape(X.shape)
    assert np.abs(Y - Yd).max() < 1e-12 * np.abs(Yd).max()


def test_augmentation_gaussian_is_normalized():
    """int g = 1 up to the Gauss rule's resolution of the Gaussian along z
    (~3e-9 on 0.93-bohr intervals for r_Q = 0.7, exact at half the spacing)."""
    w = _cell()
    for n_int, tol in ((15, 1e-8), (30, 1e-13)):
        m = Hm.model_from_workload(dataclasses.replace(w, breaks=W.uniform_breaks(-7.0, 7.0, n_int)))
        for at in m.atoms:
            assert abs(F.grid_integral(m, F.atom_gaussian(m, at)) - 1.0) < tol


def test_strengths_of_a_constant_potential():
    """V_eff = c everywhere: D = E0 + c q (int g = 1)."""
    w = _cell(nproj=5, q2s=0.2, q12=0.1)
    m = Hm.model_from_workload(w)
    c = -0.37
    D = F.uspp_strengths(m, np.full((len(m.zb.zq),) + m.grid, c))
    E0, _ = m.kb_projectors()
    assert np.abs(D - (E0 + c * m.uspp_q())).max() < 1e-9


@pytest.mark.parametrize("nproj", [4, 5])
def test_augmented_density_counts_every_electron(nproj):
    """With H c = eps S c and c^H S c = 1 the smooth density and the
    augmentation together integrate to sum f (int g = 1)."""
    w = _cell(nproj=nproj, q2s=0.25 if nproj == 5 else 0.0, q12=0.08 if nproj == 5 else 0.0)
    ms = [Hm.model_from_workload(w, ik) for ik in range(w.nk)]
    coefs, occ = [], []
    for i, m in enumerate(ms):
        S = m.dense_S()
        ev, C = E.generalized_lowest(m.dense_H(), S, 3, vectors=True)
        assert np.abs(C.conj().T @ S @ C - np.eye(3)).max() < 1e-10
        coefs.append(C.T.reshape(3, m.nb, m.ng))
        occ.append(np.array([1.0, 0.6, 0.2]) * (i + 1))
    smooth = F.density(ms, coefs, occ)
    aug = F.augmentation(ms, coefs, occ)
    total = sum(float(np.sum(o)) for o in occ)
    assert abs(F.grid_integral(ms[0], smooth + aug) - total) < 1e-8
    assert F.grid_integral(ms[0], aug) > 0.01          # positive q: charge moved into the cores


def test_uspp_without_q_is_the_norm_conserving_loop():
    w = _cell(q=(0.0, 0.0, 0.0, 0.0))
    out = F.scf(w, nbands=4, nelec=2.0, sigma=0.02, W=0.5, gmax=1.0, tol=1e-7, max_iter=60)
    assert out["strengths"] is None and out["dv"] < 1e-7


def test_uspp_loop_is_self_consistent():
    """The converged loop's D and density reproduce its potential."""
    w = _cell()
    out = F.scf(w, nbands=4, nelec=2.0, sigma=0.02, W=0.5, gmax=1.0, tol=1e-8, max_iter=80)
    assert out["dv"] < 1e-8, out["iterations"]
    m0 = Hm.model_from_workload(w)
    D = F.uspp_strengths(m0, Hm.model_from_workload(w, 0, table=out["vscf"]).local_table())
    assert np.abs(D - out["strengths"]).max() < 1e-12
    ms = [Hm.model_from_workload(w, ik, table=out["vscf"], strengths=D) for ik in range(w.nk)]
    evs, coefs = [], []
    for m in ms:
        ev, C = E.generalized_lowest(m.dense_H(), m.dense_S(), 4, vectors=True)
        evs.append(ev)
        coefs.append(C.T.reshape(4, m.nb, m.ng))
    f, _ = F.occupations(np.array(evs), np.full(w.nk, 0.5), 2.0, 0.02)
    rho = F.density(ms, coefs, f) + F.augmentation(ms, coefs, f)
    assert abs(F.grid_integral(m0, rho) - 2.0) < 1e-8
    v = F.to_r(F.hartree_g(m0, F.to_g(rho))) + F.xc_pz(rho)[0]
    assert np.abs(v - out["vscf"]).max() < 1e-6
