"""Pins for the oracle's matrix elements (§II.B.1) against closed forms,
invariances and brute-force numerical integrals that do not go through the
oracle's own formulas."""
import dataclasses
import math

import numpy as np
import pytest
import scipy.linalg as sl

from oracle import eigen as E
from oracle import hamiltonian as Hm
from paper_1406_4960_gb300 import workloads as W


def _small(with_kb=True, ecut=5.0, n_int=15, k=(0.0, 0.0), a=4.7, zext=6.0, square=True, seed=11):
    rng = np.random.default_rng(seed)
    atoms = []
    for z in (-1.2, 0.9):
        f = rng.random(2)
        atoms.append(W.Atom((float(f[0] * a), float(f[1] * a), z), -2.0, 0.9,
                            4 if with_kb else 0, (0.7, -0.4, -0.4, -0.4) if with_kb else (0, 0, 0, 0), 1.1))
    a2 = (0.0, a) if square else (0.4 * a, 0.9 * a)
    return W.Workload("small", (a, 0.0), a2, np.array([k], dtype=np.float64), ecut,
                      W.uniform_breaks(-zext, zext, n_int), 6, 6, (16, 16), atoms, 6)


def _eigs(m, n=None):
    return E.generalized_lowest(m.dense_H(), m.dense_S(), n)


# --------------------------------------------------------------------------
def test_free_electron_hard_wall_closed_form():
    """V = 0: eps = |k+G|^2/2 + (n pi / L)^2 / 2, approached from above."""
    w = dataclasses.replace(W.tiny(), kpts=np.array([[0.21, -0.13]]))
    m = Hm.model_from_workload(w, with_atoms=False)
    got = _eigs(m, 20)
    L = w.breaks[-1] - w.breaks[0]
    exact = np.sort(np.array([0.5 * q2 + 0.5 * (n * math.pi / L) ** 2
                              for q2 in m.q2 for n in range(1, 30)]))[:20]
    assert np.all(got - exact > -1e-12)
    assert np.abs(got - exact).max() < 1e-8


def test_constant_potential_shifts_spectrum():
    w = _small(with_kb=True)
    V0 = 0.3711
    base = _eigs(Hm.model_from_workload(w), 12)
    shifted = _eigs(Hm.model_from_workload(w, local_components=[(0, 0, lambda z: V0)]), 12)
    assert np.abs(shifted - base - V0).max() < 1e-12


def test_harmonic_well_closed_form():
    """V = omega^2 z^2 / 2, in-plane constant: eps = |k+G|^2/2 + omega (n + 1/2)."""
    om = 1.0
    w = dataclasses.replace(W.tiny(), breaks=W.uniform_breaks(-10, 10, 77), ecut=3.0,
                            kpts=np.array([[0.3, 0.1]]))
    m = Hm.model_from_workload(w, with_atoms=False,
                               local_components=[(0, 0, lambda z: 0.5 * om * om * z * z)])
    got = _eigs(m, 10)
    exact = np.sort(np.array([0.5 * q2 + om * (n + 0.5) for q2 in m.q2 for n in range(12)]))[:10]
    assert np.abs(got - exact).max() < 1e-8


def test_separable_cosine_potential():
    """V = 2 V1 cos(b1 . r): eps = eps_z(n) + eps_xy(m), eps_xy from a plain
    plane-wave matrix over the same disc."""
    V1 = 0.45
    w = dataclasses.replace(W.tiny(), ecut=4.0, breaks=W.uniform_breaks(-6, 6, 15),
                            kpts=np.array([[0.17, 0.05]]))
    comps = [(1, 0, lambda z: V1), (-1, 0, lambda z: V1)]
    m = Hm.model_from_workload(w, with_atoms=False, local_components=comps)
    got = _eigs(m, 15)
    ez = sl.eigh(0.5 * m.D, m.S, eigvals_only=True)
    n = m.ng
    P = np.diag(0.5 * m.q2).astype(complex)
    for i in range(n):
        for j in range(n):
            d = m.gidx[i] - m.gidx[j]
            if abs(d[0]) == 1 and d[1] == 0:
                P[i, j] += V1
    exy = np.linalg.eigvalsh(P)
    exact = np.sort((ez[:, None] + exy[None, :]).ravel())[:15]
    assert np.abs(got - exact).max() < 1e-11


def test_gaussian_element_by_real_space_quadrature():
    """(1/A_c) int_cell exp(-i dG.r) sum_images A exp(-a|r-R|^2) d^2r by a plain
    Riemann sum (spectrally accurate for a periodic integrand) equals the
    element's in-plane factor (A/A_c)(pi/a) exp(-dG^2/4a) exp(-i dG.R)."""
    w = _small(with_kb=False, square=False)
    m = Hm.model_from_workload(w)
    at = w.atoms[0]
    m1 = Hm.Model(w.a1, w.a2, w.kpts[0], w.ecut, w.breaks, w.order, [at], (64, 64))
    (I, F), = m1.local_terms()
    a = 1.0 / (2 * at.w * at.w)
    n = 96
    a1, a2 = np.array(w.a1), np.array(w.a2)
    s = (np.arange(n) + 0.5) / n
    r = s[:, None, None] * a1 + s[None, :, None] * a2
    V = np.zeros((n, n))
    for i1 in range(-3, 4):
        for i2 in range(-3, 4):
            R = np.array(at.pos[:2]) + i1 * a1 + i2 * a2
            d = r - R
            V += at.A * np.exp(-a * np.sum(d * d, axis=-1))
    rng = np.random.default_rng(0)
    for _ in range(12):
        g, gp = rng.integers(0, m1.ng, 2)
        dG = m1.q[g] - m1.q[gp]
        num = np.mean(np.exp(-1j * (r @ dG)) * V)        # (1/A_c) int_cell = mean over the cell
        assert abs(num - F[g, gp]) < 1e-10
    # z factor: I(i; a, R_z; i') by an independent fine Simpson rule
    from oracle import bspline as bs
    zz = np.linspace(w.breaks[0], w.breaks[-1], 24001)
    Bz = np.array([m1.zb.values(z) for z in zz])
    f = Bz[:, 3] * Bz[:, 5] * np.exp(-a * (zz - at.pos[2]) ** 2)
    h = zz[1] - zz[0]
    simpson = h / 3 * (f[0] + f[-1] + 4 * f[1:-1:2].sum() + 2 * f[2:-1:2].sum())
    assert abs(simpson - I[3, 5]) < 2e-6 * abs(I[3, 5])   # Gauss with p=k is a discretization
    zb2 = bs.ZBasis(w.breaks, w.order, nquad=14)
    I14 = zb2.weighted(np.exp(-a * (zb2.zq - at.pos[2]) ** 2))
    assert abs(simpson - I14[3, 5]) < 1e-10


def test_wrapped_and_unwrapped_local_elements_agree_to_the_aliasing_bound():
    w = W.slab()
    m = Hm.model_from_workload(w, ik=1)
    d1, d2, g = m._dG_wrapped()
    gd = m.q[:, None, :] - m.q[None, :, :]
    wrapped = (d1 != m.gidx[:, None, 0] - m.gidx[None, :, 0]) | (d2 != m.gidx[:, None, 1] - m.gidx[None, :, 1])
    assert wrapped.any()   # this grid does alias some dG
    a = 1.0 / (2 * w.atoms[0].w ** 2)
    g2w = np.sum(g * g, -1)[wrapped]
    bound = (abs(w.atoms[0].A) * len(w.atoms) / m.Ac) * (math.pi / a) * np.exp(-g2w.min() / (4 * a))
    assert bound < 1e-9
    del gd


# --------------------------------------------------------------------------
def test_projector_transforms_by_numerical_integration():
    """Q_{1,00}, Q_x, Q_y closed forms vs a Riemann sum over a large box, and
    the normalization int |beta|^2 = 1 of s and p projectors."""
    alpha = 1.0 / (2 * 1.1 ** 2)
    L, n = 16.0, 400
    x = (np.arange(n) + 0.5) / n * 2 * L - L
    X, Y = np.meshgrid(x, x, indexing="ij")
    dA = (2 * L / n) ** 2
    gauss = np.exp(-alpha * (X * X + Y * Y))
    for q in ([0.0, 0.0], [0.7, -0.3], [1.9, 1.2]):
        ph = np.exp(1j * (q[0] * X + q[1] * Y))
        Qs_num = np.sum(ph * gauss) * dA
        Qx_num = np.sum(X * ph * gauss) * dA
        Qy_num = np.sum(Y * ph * gauss) * dA
        q2 = q[0] ** 2 + q[1] ** 2
        Qs = math.pi / alpha * math.exp(-q2 / (4 * alpha))
        assert abs(Qs_num - Qs) < 1e-10
        assert abs(Qx_num - 1j * q[0] / (2 * alpha) * Qs) < 1e-10
        assert abs(Qy_num - 1j * q[1] / (2 * alpha) * Qs) < 1e-10
    # normalization (separable 1D integrals)
    t = np.linspace(-20, 20, 400001)
    h = t[1] - t[0]
    g1 = np.sum(np.exp(-2 * alpha * t * t)) * h
    g1x2 = np.sum(t * t * np.exp(-2 * alpha * t * t)) * h
    Cs = (2 * alpha / math.pi) ** 0.75
    Cp = 2 * math.sqrt(alpha) * Cs
    assert abs(Cs ** 2 * g1 ** 3 - 1) < 1e-10
    assert abs(Cp ** 2 * g1x2 * g1 ** 2 - 1) < 1e-10


def test_projector_overlaps_by_direct_integration():
    """u_p(G, i) = A_c^{-1/2} int exp(-i(k+G).r) B_i(z) beta_p(r - R) d^3r, the
    in-plane part by a Riemann sum over a large box, the z part by a fine rule."""
    w = _small(with_kb=True, k=(0.23, -0.11))
    m = Hm.model_from_workload(w)
    Es, U = m.kb_projectors()
    at = w.atoms[1]
    alpha = 1.0 / (2 * at.rc ** 2)
    Cs = (2 * alpha / math.pi) ** 0.75
    Cp = 2 * math.sqrt(alpha) * Cs
    L, n = 14.0, 280
    x = (np.arange(n) + 0.5) / n * 2 * L - L
    X, Y = np.meshgrid(x, x, indexing="ij")
    dA = (2 * L / n) ** 2
    zz = np.linspace(w.breaks[0], w.breaks[-1], 12001)
    hz = zz[1] - zz[0]
    Bz = np.array([m.zb.values(z) for z in zz])
    rng = np.random.default_rng(1)
    for _ in range(6):
        g = int(rng.integers(0, m.ng))
        i = int(rng.integers(0, m.nb))
        q = m.q[g]
        ph = np.exp(-1j * (q[0] * (X + at.pos[0]) + q[1] * (Y + at.pos[1])))
        rad = np.exp(-alpha * (X * X + Y * Y))
        dz = zz - at.pos[2]
        gz = np.exp(-alpha * dz * dz) * Bz[:, i]
        wz = np.full_like(zz, hz)
        wz[0] = wz[-1] = hz / 2
        plane_s = np.sum(ph * rad) * dA
        plane_x = np.sum(ph * X * rad) * dA
        plane_y = np.sum(ph * Y * rad) * dA
        ints = [Cs * plane_s * (wz @ gz), Cp * plane_x * (wz @ gz), Cp * plane_y * (wz @ gz),
                Cp * plane_s * (wz @ (dz * gz))]
        for p in range(4):
            ref = ints[p] / math.sqrt(m.Ac)
            assert abs(U[4 + p, i, g] - ref) < 2e-6 * max(1e-3, abs(ref)), (p, U[4 + p, i, g], ref)


def test_hamiltonian_structure():
    w = _small(with_kb=True, k=(0.1, 0.2))
    m = Hm.model_from_workload(w)
    H = m.dense_H()
    assert np.abs(H - H.conj().T).max() < 1e-14
    Es, U = m.kb_projectors()
    Unl = U.reshape(len(Es), -1).T
    Hnl = Unl @ Es @ Unl.conj().T
    assert np.linalg.matrix_rank(Hnl, tol=1e-10 * np.abs(Hnl).max()) <= len(Es)
    w0 = dataclasses.replace(w, atoms=[dataclasses.replace(a, E=(0, 0, 0, 0)) for a in w.atoms])
    wl = dataclasses.replace(w, atoms=[dataclasses.replace(a, nproj=0) for a in w.atoms])
    assert np.abs(Hm.model_from_workload(w0).dense_H() - Hm.model_from_workload(wl).dense_H()).max() == 0.0
    X = W.random_block(3, m.nb, m.ng, 9)
    Y = m.apply_H(X)
    Yd = (H @ X.reshape(3, -1).T).T.reshape(X.shape)
    assert np.abs(Y - Yd).max() < 1e-12 * np.abs(Yd).max()
    ent = [(0, 1, 2), (2, m.nb - 1, m.ng - 1), (1, 7, 0)]
    assert np.abs(m.apply_H_entries(X, ent) - np.array([Y[e] for e in ent])).max() < 1e-12 * np.abs(Y).max()
    Sd = m.dense_S()
    assert np.abs(m.apply_S(X) - (Sd @ X.reshape(3, -1).T).T.reshape(X.shape)).max() < 1e-14


def test_translation_invariance():
    """Moving every atom by the same in-plane vector leaves the spectrum unchanged
    (pins the relative phase of the local and projector terms)."""
    w = _small(with_kb=True, k=(0.19, -0.07))
    t = np.array([1.37, -0.58])
    w2 = dataclasses.replace(w, atoms=[dataclasses.replace(a, pos=(a.pos[0] + t[0], a.pos[1] + t[1], a.pos[2]))
                                       for a in w.atoms])
    e1 = _eigs(Hm.model_from_workload(w), 14)
    e2 = _eigs(Hm.model_from_workload(w2), 14)
    assert np.abs(e1 - e2).max() < 1e-11


def test_time_reversal():
    w = _small(with_kb=True, k=(0.19, -0.07))
    wm = dataclasses.replace(w, kpts=-w.kpts)
    e1 = _eigs(Hm.model_from_workload(w), 14)
    e2 = _eigs(Hm.model_from_workload(wm), 14)
    assert np.abs(e1 - e2).max() < 1e-11


def test_rotation_by_90_degrees():
    """Square cell: rotating atoms and k by 90 degrees maps H to a unitarily
    equivalent matrix (pins p_x against p_y)."""
    w = _small(with_kb=True, k=(0.19, -0.07))
    rot = lambda v: (-v[1], v[0])
    atoms = [dataclasses.replace(a, pos=(*rot(a.pos[:2]), a.pos[2])) for a in w.atoms]
    w2 = dataclasses.replace(w, atoms=atoms, kpts=np.array([rot(w.kpts[0])]))
    e1 = _eigs(Hm.model_from_workload(w), 14)
    e2 = _eigs(Hm.model_from_workload(w2), 14)
    assert np.abs(e1 - e2).max() < 1e-11


def test_z_reflection():
    """z -> -z of the atoms on symmetric knots leaves the spectrum unchanged
    (pins the p_z factor Z_{1,10})."""
    w = _small(with_kb=True, k=(0.19, -0.07))
    atoms = [dataclasses.replace(a, pos=(a.pos[0], a.pos[1], -a.pos[2])) for a in w.atoms]
    w2 = dataclasses.replace(w, atoms=atoms)
    e1 = _eigs(Hm.model_from_workload(w), 14)
    e2 = _eigs(Hm.model_from_workload(w2), 14)
    assert np.abs(e1 - e2).max() < 1e-11


def test_p_channel_differs_from_s_only():
    """Sanity of the pins above: a p_z-only strength change moves the spectrum."""
    w = _small(with_kb=True, k=(0.19, -0.07))
    w2 = dataclasses.replace(w, atoms=[dataclasses.replace(a, E=(a.E[0], a.E[1], a.E[2], a.E[3] - 0.3))
                                       for a in w.atoms])
    e1 = _eigs(Hm.model_from_workload(w), 14)
    e2 = _eigs(Hm.model_from_workload(w2), 14)
    assert np.abs(e1 - e2).max() > 1e-4


# --------------------------------------------------------------------------
# second s channel (n = 2) and the 1s-2s coupling
def _small2s(e12=0.23, e2s=-0.35, **kw):
    w = _small(with_kb=True, **kw)
    atoms = [dataclasses.replace(a, nproj=5, e2s=e2s, e12=e12) for a in w.atoms]
    return dataclasses.replace(w, atoms=atoms)


def test_second_s_channel_transform_and_normalization():
    """Q_{2,00} closed form vs a Riemann sum of (x^2 + y^2) exp(-alpha r^2)
    e^{iq.r}, and int |beta_2s|^2 = 1 for beta_2s = C r^2 exp(-alpha r^2)
    from separable 1D integrals ((x^2+y^2+z^2)^2 expanded)."""
    alpha = 1.0 / (2 * 1.1 ** 2)
    L, n = 16.0, 400
    x = (np.arange(n) + 0.5) / n * 2 * L - L
    X, Y = np.meshgrid(x, x, indexing="ij")
    dA = (2 * L / n) ** 2
    r2 = X * X + Y * Y
    gauss = np.exp(-alpha * r2)
    for q in ([0.0, 0.0], [0.7, -0.3], [1.9, 1.2]):
        ph = np.exp(1j * (q[0] * X + q[1] * Y))
        num = np.sum(r2 * ph * gauss) * dA
        q2 = q[0] ** 2 + q[1] ** 2
        closed = (1 / alpha - q2 / (4 * alpha ** 2)) * math.pi / alpha * math.exp(-q2 / (4 * alpha))
        assert abs(num - closed) < 1e-9
    t = np.linspace(-20, 20, 400001)
    h = t[1] - t[0]
    gk = [np.sum(t ** k * np.exp(-2 * alpha * t * t)) * h for k in (0, 2, 4)]
    norm_int = 3 * gk[2] * gk[0] ** 2 + 6 * gk[1] ** 2 * gk[0]
    C2 = (4.0 * math.pi * 15.0 / 16.0 * math.sqrt(math.pi) * (2.0 * alpha) ** -3.5) ** -0.5
    assert abs(C2 ** 2 * norm_int - 1) < 1e-10


def test_second_s_projector_by_direct_integration():
    """u_2s(G, i) = A_c^{-1/2} int exp(-i(k+G).r) B_i(z) C r^2 exp(-alpha r^2) d^3r
    (r relative to the atom) by a Riemann sum in plane and a fine z rule."""
    w = _small2s(k=(0.23, -0.11))
    m = Hm.model_from_workload(w)
    Emat, U = m.kb_projectors()
    assert U.shape[0] == 10 and Emat.shape == (10, 10)
    at = w.atoms[1]
    alpha = 1.0 / (2 * at.rc ** 2)
    C2 = (4.0 * math.pi * 15.0 / 16.0 * math.sqrt(math.pi) * (2.0 * alpha) ** -3.5) ** -0.5
    L, n = 14.0, 280
    x = (np.arange(n) + 0.5) / n * 2 * L - L
    X, Y = np.meshgrid(x, x, indexing="ij")
    dA = (2 * L / n) ** 2
    zz = np.linspace(w.breaks[0], w.breaks[-1], 12001)
    hz = zz[1] - zz[0]
    Bz = np.array([m.zb.values(z) for z in zz])
    wz = np.full_like(zz, hz)
    wz[0] = wz[-1] = hz / 2
    rng = np.random.default_rng(2)
    for _ in range(6):
        g = int(rng.integers(0, m.ng))
        i = int(rng.integers(0, m.nb))
        q = m.q[g]
        ph = np.exp(-1j * (q[0] * (X + at.pos[0]) + q[1] * (Y + at.pos[1])))
        rho2 = X * X + Y * Y
        rad = np.exp(-alpha * rho2)
        dz = zz - at.pos[2]
        gz = np.exp(-alpha * dz * dz) * Bz[:, i]
        val = C2 * (np.sum(ph * rho2 * rad) * dA * (wz @ gz) + np.sum(ph * rad) * dA * (wz @ (dz * dz * gz)))
        ref = val / math.sqrt(m.Ac)
        assert abs(U[5 + 4, i, g] - ref) < 2e-6 * max(1e-3, abs(ref)), (U[9, i, g], ref)
    # the strengths: E_1s, E_p, E_2s on the diagonal, E_12 coupling 1s <-> 2s
    assert Emat[0, 4] == Emat[4, 0] == 0.23 and Emat[4, 4] == -0.35 and Emat[0, 0] == 0.7
    assert np.count_nonzero(Emat - np.diag(np.diag(Emat))) == 4


def test_second_s_channel_structure():
    w = _small2s(k=(0.1, 0.2))
    m = Hm.model_from_workload(w)
    H = m.dense_H()
    assert np.abs(H - H.conj().T).max() < 1e-14
    Emat, U = m.kb_projectors()
    Unl = U.reshape(len(Emat), -1).T
    Hnl = Unl @ Emat @ Unl.conj().T
    assert np.linalg.matrix_rank(Hnl, tol=1e-10 * np.abs(Hnl).max()) <= len(Emat)
    # all strengths zero == no projectors at all
    w0 = dataclasses.replace(w, atoms=[dataclasses.replace(a, E=(0, 0, 0, 0), e2s=0.0, e12=0.0) for a in w.atoms])
    wl = dataclasses.replace(w, atoms=[dataclasses.replace(a, nproj=0) for a in w.atoms])
    assert np.abs(Hm.model_from_workload(w0).dense_H() - Hm.model_from_workload(wl).dense_H()).max() < 1e-15
    # with E_2s = E_12 = 0 the fifth projector drops out
    w4 = dataclasses.replace(w, atoms=[dataclasses.replace(a, nproj=4) for a in w.atoms])
    wz = dataclasses.replace(w, atoms=[dataclasses.replace(a, e2s=0.0, e12=0.0) for a in w.atoms])
    assert np.abs(Hm.model_from_workload(w4).dense_H() - Hm.model_from_workload(wz).dense_H()).max() < 1e-14
    # matrix-free apply and single entries against the dense matrix
    X = W.random_block(3, m.nb, m.ng, 9)
    Y = m.apply_H(X)
    Yd = (H @ X.reshape(3, -1).T).T.reshape(X.shape)
    assert np.abs(Y - Yd).max() < 1e-12 * np.abs(Yd).max()
    ent = [(0, 1, 2), (2, m.nb - 1, m.ng - 1)]
    assert np.abs(m.apply_H_entries(X, ent) - np.array([Y[e] for e in ent])).max() < 1e-12 * np.abs(Y).max()
    # the coupling moves the spectrum; translation, time reversal and z reflection do not
    e1 = _eigs(m, 14)
    wc = dataclasses.replace(w, atoms=[dataclasses.replace(a, e12=0.0) for a in w.atoms])
    assert np.abs(_eigs(Hm.model_from_workload(wc), 14) - e1).max() > 1e-5
    t = np.array([1.37, -0.58])
    wt = dataclasses.replace(w, atoms=[dataclasses.replace(a, pos=(a.pos[0] + t[0], a.pos[1] + t[1], a.pos[2]))
                                       for a in w.atoms])
    assert np.abs(_eigs(Hm.model_from_workload(wt), 14) - e1).max() < 1e-11
    wm = dataclasses.replace(w, kpts=-w.kpts)
    assert np.abs(_eigs(Hm.model_from_workload(wm), 14) - e1).max() < 1e-11
    wr = dataclasses.replace(w, atoms=[dataclasses.replace(a, pos=(a.pos[0], a.pos[1], -a.pos[2])) for a in w.atoms])
    assert np.abs(_eigs(Hm.model_from_workload(wr), 14) - e1).max() < 1e-11
