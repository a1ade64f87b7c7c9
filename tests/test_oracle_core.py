"""Pins for the oracle's core term -Z erf(r/R_c)/r of the local pseudopotential
(§II.B.1, Eq. (10) and the Coulomb integral with the 2D transform of 1/r).
The closed form in ``core_term`` is checked against numerical integrals that
do not use it: the Coulomb integral of the Gaussian core charge done by
quadrature, the real-space potential transformed by a Hankel integral, the
g = 0 remainder by quadrature, and high-precision arithmetic where the
closed form is rewritten to avoid overflow."""
import dataclasses
import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle import eigen as E
from oracle import hamiltonian as Hm
from paper_1406_4960_gb300 import workloads as W

CASES = [(0.3, 0.0, 0.8), (0.9, 0.4, 0.8), (2.5, -1.3, 0.5), (1.7, 3.0, 1.1), (6.0, 0.2, 0.35), (0.05, 2.0, 0.7)]


def _rho_g(zp, g, Rc):
    """In-plane component of the Gaussian core charge, Z = A_c = 1."""
    return math.exp(-0.25 * (g * Rc) ** 2) * math.exp(-(zp / Rc) ** 2) / (math.sqrt(math.pi) * Rc)


@pytest.mark.parametrize("g,dz,Rc", CASES)
def test_core_term_is_the_coulomb_integral_of_the_core_charge(g, dz, Rc):
    """-(2 pi/g) int dz' rho_c(z', g) exp(-g |dz - z'|), by adaptive quadrature."""
    f = lambda zp: _rho_g(zp, g, Rc) * math.exp(-g * abs(dz - zp))
    lo, hi = -12 * Rc, 12 * Rc
    pts = [dz] if lo < dz < hi else None
    val, err = integrate.quad(f, lo, hi, points=pts, epsabs=1e-14, epsrel=1e-12, limit=400)
    want = -(2 * math.pi / g) * val
    got = Hm.core_term(g, dz, 1.0, Rc, 1.0)
    assert abs(got - want) <= 1e-10 * max(1.0, abs(want)), (got, want)


@pytest.mark.parametrize("g,dz,Rc", [(0.6, 0.5, 0.8), (1.4, -0.9, 0.6), (2.2, 1.6, 1.0)])
def test_core_term_is_the_inplane_transform_of_the_real_space_potential(g, dz, Rc):
    """From Eq. (10) directly: -erf(r/Rc)/r = -1/r + erfc(r/Rc)/r; the in-plane
    transform of 1/r is 2 pi exp(-g|z|)/g, and the short-ranged erfc part is a
    Hankel integral 2 pi int rho J0(g rho) erfc(r/Rc)/r d rho."""
    def h(rho):
        r = math.hypot(rho, dz)
        return 2 * math.pi * rho * special.j0(g * rho) * math.erfc(r / Rc) / r
    tail, _ = integrate.quad(h, 0.0, 12 * Rc, epsabs=1e-13, epsrel=1e-12, limit=400)
    want = -2 * math.pi * math.exp(-g * abs(dz)) / g + tail
    got = Hm.core_term(g, dz, 1.0, Rc, 1.0)
    assert abs(got - want) <= 1e-9 * max(1.0, abs(want)), (got, want)


@pytest.mark.parametrize("dz,Rc", [(0.0, 0.8), (0.7, 0.8), (-2.5, 0.5), (4.0, 1.2)])
def test_core_term_at_g0_is_the_sheet_remainder(dz, Rc):
    """g = 0 keeps +2 pi int dz' rho_c(z') |dz - z'| (Z = A_c = 1), and
    core_term(g) + 2 pi / g tends to it as g -> 0."""
    f = lambda zp: _rho_g(zp, 0.0, Rc) * abs(dz - zp)
    lo, hi = -12 * Rc, 12 * Rc
    val, _ = integrate.quad(f, lo, hi, points=[dz] if lo < dz < hi else None, epsabs=1e-14, limit=400)
    got = Hm.core_term(0.0, dz, 1.0, Rc, 1.0)
    assert abs(got - 2 * math.pi * val) <= 1e-11 * max(1.0, abs(got))
    for g in (1e-3, 1e-4):
        lim = Hm.core_term(g, dz, 1.0, Rc, 1.0) + 2 * math.pi / g
        assert abs(lim - got) < 20 * g * (1 + abs(dz)) ** 2


def test_core_term_far_from_the_atom_is_the_bare_sheet():
    """Far from the core charge the g = 0 part is the bare charged sheet
    2 pi Z |dz| / A_c, and the g > 0 parts are the bare -2 pi Z exp(-g|dz|)/(g A_c)."""
    Rc, Z, Ac = 0.6, 3.0, 7.5
    for dz in (-9.0, 8.0):
        assert abs(Hm.core_term(0.0, dz, Z, Rc, Ac) - 2 * math.pi * Z * abs(dz) / Ac) < 1e-12
        for g in (0.4, 1.3):
            bare = -2 * math.pi * Z * math.exp(-g * abs(dz)) / (g * Ac)
            # the smeared charge's correction factor exp(g^2 Rc^2/4)... is inside erfc: compare loosely
            assert abs(Hm.core_term(g, dz, Z, Rc, Ac) - bare) <= 1e-6 * abs(bare) + 1e-300


def test_core_term_overflow_free_branch_matches_high_precision():
    """Where the closed form's exp(g z) erfc(.) would overflow in doubles, the
    erfcx form agrees with 40-digit arithmetic."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    for g, dz, Rc in [(30.0, 5.0, 0.5), (55.0, -4.0, 0.4), (12.0, 20.0, 1.5), (80.0, 0.01, 0.3)]:
        gg, zz, R = mpmath.mpf(g), mpmath.mpf(dz), mpmath.mpf(Rc)
        T = lambda z: mpmath.e ** (gg * z) * mpmath.erfc(gg * R / 2 + z / R)
        want = -(mpmath.pi / gg) * (T(zz) + T(-zz))
        got = Hm.core_term(g, dz, 1.0, Rc, 1.0)
        assert abs(got - float(want)) <= 1e-13 * abs(float(want)) + 1e-300, (g, dz, Rc, got, want)


def _core_cell(seed=5, Z=1.5, Rc=0.7, with_kb=True):
    rng = np.random.default_rng(seed)
    a = 4.7
    atoms = []
    for z in (-1.1, 0.8):
        f = rng.random(2)
        atoms.append(W.Atom((float(f[0] * a), float(f[1] * a), z), -1.0, 0.9,
                            4 if with_kb else 0, (0.7, -0.4, -0.4, -0.4) if with_kb else (0, 0, 0, 0), 1.1,
                            Z=Z, Rcore=Rc))
    return W.Workload("core", (a, 0.0), (0.3 * a, 0.95 * a), np.array([[0.13, -0.07]]), 4.0,
                      W.uniform_breaks(-7.0, 7.0, 13), 6, 6, (16, 16), atoms, 6)


def test_dense_H_with_core_term_is_hermitian_and_matches_the_applies():
    w = _core_cell()
    m = Hm.model_from_workload(w)
    H = m.dense_H()
    assert np.abs(H - H.conj().T).max() < 1e-12 * np.abs(H).max()
    X = W.random_block(3, m.nb, m.ng, seed=2)
    Y = m.apply_H(X)
    Yd = (H @ X.reshape(3, -1).T).T.reshape(X.shape)
    assert np.abs(Y - Yd).max() < 1e-11 * np.abs(Yd).max()
    ent = [(0, 0, 0), (1, 3, m.ng - 1), (2, m.nb - 1, 5), (1, 7, 11)]
    got = m.apply_H_entries(X, ent)
    assert np.abs(got - np.array([Y[b, i, g] for b, i, g in ent])).max() < 1e-11 * np.abs(Yd).max()


def test_core_term_eigenvalues_invariant_under_inplane_translation():
    """Moving every atom by the same in-plane vector changes H by a diagonal
    phase exp(-i G.t): the spectrum stays put (a dropped sign or a transposed
    dG in the core elements would break it)."""
    w = _core_cell(with_kb=False)
    t = np.array([1.37, -0.61])
    w2 = dataclasses.replace(w, atoms=[dataclasses.replace(a, pos=(a.pos[0] + t[0], a.pos[1] + t[1], a.pos[2]))
                                       for a in w.atoms])
    e1 = E.generalized_lowest(Hm.model_from_workload(w).dense_H(), Hm.model_from_workload(w).dense_S(), 12)
    m2 = Hm.model_from_workload(w2)
    e2 = E.generalized_lowest(m2.dense_H(), m2.dense_S(), 12)
    assert np.abs(e1 - e2).max() < 1e-10


def test_core_table_is_the_real_table_of_the_components():
    """local_table's inverse FFT is real, and its forward FFT gives back the
    core components on every dG that a pair of plane waves couples."""
    w = _core_cell(with_kb=False)
    w = dataclasses.replace(w, atoms=[dataclasses.replace(a, A=0.0) for a in w.atoms])
    m = Hm.model_from_workload(w)
    V = m.local_table()
    c = np.fft.fft2(V, axes=(1, 2)) / (V.shape[1] * V.shape[2])
    Vc = m.core_table()
    assert np.abs(c - Vc).max() < 1e-12 * np.abs(Vc).max()


def test_core_term_of_a_neutralised_pair_has_no_sheet_field():
    """Two core charges +Z and -Z at the same height and in-plane position
    cancel exactly: the elements vanish (the g = 0 choice is per charge, so a
    neutral pair leaves no field)."""
    w = _core_cell(with_kb=False)
    a0 = dataclasses.replace(w.atoms[0], A=0.0)
    w = dataclasses.replace(w, atoms=[a0, dataclasses.replace(a0, Z=-a0.Z)])
    m = Hm.model_from_workload(w)
    assert np.abs(m.core_table()).max() < 1e-15


def test_core_potential_is_deepest_at_the_atom():
    """Z > 0 is attractive (Eq. (10)'s sign): with one core atom on a grid
    point, the tabulated potential is lowest on that point, on the plane
    nearest the atom, and it rises away from it in z (the kept g = 0 part
    grows like 2 pi Z |dz| / A_c)."""
    w = _core_cell(with_kb=False)
    a = 4.7
    at = dataclasses.replace(w.atoms[0], A=0.0, pos=(5 / 16 * a + 0.3 * a * 3 / 16, 0.95 * a * 3 / 16, 0.37))
    w = dataclasses.replace(w, atoms=[at])
    m = Hm.model_from_workload(w)
    V = m.local_table()
    q, i1, i2 = np.unravel_index(np.argmin(V), V.shape)
    assert (i1, i2) == (5, 3)
    assert q == np.argmin(np.abs(m.zb.zq - 0.37))
    col = V[:, 5, 3]
    assert np.all(np.diff(col[: q + 1]) <= 0) and np.all(np.diff(col[q:]) >= 0)
