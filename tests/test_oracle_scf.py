"""Pins for the oracle's self-consistent loop (§II.B.1, §III.A): the density
against direct evaluation at grid points and its normalization, the Hartree
potential against the closed-form potential of a Gaussian charge, the LDA
against the derivative identity and the textbook limits, the occupations,
the Kerker-Pulay mixer, and self-consistency of the converged loop."""
import dataclasses
import math

import numpy as np
import pytest
from scipy import optimize

from oracle import eigen as E
from oracle import hamiltonian as Hm
from oracle import scf as F
from paper_1406_4960_gb300 import workloads as W


def _cell(nk=1, Z=1.0, ecut=4.0, n_int=15, grid=(16, 16), A=-0.5):
    a = 4.2
    atoms = [W.Atom((0.7, 1.1, -0.6), A, 0.8, Z=Z, Rcore=0.5),
             W.Atom((2.9, 3.0, 0.7), A, 0.8, Z=Z, Rcore=0.5)]
    k = np.array([[0.0, 0.0], [0.31, -0.2], [-0.12, 0.4]][:nk])
    return W.Workload("scf", (a, 0.0), (0.35 * a, 0.93 * a), k, ecut, W.uniform_breaks(-7.0, 7.0, n_int),
                      6, 6, grid, atoms, 4)


def _integral(m, rho):
    N1, N2 = m.grid
    return float(np.sum(m.zb.wq[:, None, None] * rho) * m.Ac / (N1 * N2))


def test_density_is_normalized_by_the_occupations():
    """c^H S c = 1 for each eigenvector, so the density integrates to sum f
    (Parseval on the grid and the exact S quadrature)."""
    w = _cell(nk=2)
    ms = [Hm.model_from_workload(w, ik) for ik in range(w.nk)]
    coefs, occ = [], []
    for i, m in enumerate(ms):
        ev, C = E.generalized_lowest(m.dense_H(), m.dense_S(), 3, vectors=True)
        coefs.append(C.T.reshape(3, m.nb, m.ng))
        occ.append(np.array([0.9, 0.4, 0.25]) * (i + 1))
    rho = F.density(ms, coefs, occ)
    assert abs(_integral(ms[0], rho) - sum(float(np.sum(o)) for o in occ)) < 1e-11


def test_density_of_two_plane_waves_at_grid_points():
    """One band a e^{i(k+G1).r} u(z) + b e^{i(k+G2).r} u(z): its density at a
    grid point r_i is |a e^{iG1.r} + b e^{iG2.r}|^2 |u(z)|^2 / A_c, evaluated
    directly (no transform)."""
    w = _cell()
    m = Hm.model_from_workload(w)
    rng = np.random.default_rng(4)
    cz = rng.standard_normal(m.nb)
    g1, g2 = 2, 7
    a, b = 0.8 + 0.3j, -0.4 + 0.5j
    C = np.zeros((1, m.nb, m.ng), dtype=np.complex128)
    C[0, :, g1] = a * cz
    C[0, :, g2] = b * cz
    rho = F.density([m], [C], [np.array([1.0])])
    N1, N2 = m.grid
    uz = m.zb.B @ cz
    G = m.gidx[:, 0:1] * m.b1 + m.gidx[:, 1:2] * m.b2
    for (i1, i2) in [(0, 0), (3, 11), (15, 7), (8, 8)]:
        r = (i1 / N1) * m.a1 + (i2 / N2) * m.a2
        amp = a * np.exp(1j * G[g1] @ r) + b * np.exp(1j * G[g2] @ r)
        want = np.abs(amp) ** 2 * uz ** 2 / m.Ac
        assert np.abs(rho[:, i1, i2] - want).max() < 1e-12 * max(1.0, want.max())


def _sheet_rho(m, Rc, R):
    g, gn = F.grid_freqs(m)
    dz = m.zb.zq - R[2]
    prof = np.exp(-(dz / Rc) ** 2) / (math.sqrt(math.pi) * Rc)
    phase = np.exp(-1j * (g[..., 0] * R[0] + g[..., 1] * R[1]))
    return (1.0 / m.Ac) * prof[:, None, None] * (np.exp(-0.25 * (gn * Rc) ** 2) * phase)[None], gn, g


@pytest.mark.parametrize("n_int", [40, 80])
def test_hartree_of_a_gaussian_charge_is_the_closed_form(n_int):
    """The Hartree potential of one Gaussian charge (unit Z) is minus the core
    term's closed form (same charge, opposite sign); the Gauss rule over the
    kink of exp(-g|z - z'|) converges like h^2."""
    w = dataclasses.replace(_cell(), breaks=W.uniform_breaks(-9.0, 9.0, n_int))
    m = Hm.model_from_workload(w)
    R = (1.3, 0.4, 0.3)
    Rc = 0.8
    rho_g, gn, g = _sheet_rho(m, Rc, R)
    V = F.hartree_g(m, rho_g)
    phase = np.exp(-1j * (g[..., 0] * R[0] + g[..., 1] * R[1]))
    want = -Hm.core_term(gn[None], (m.zb.zq - R[2])[:, None, None], 1.0, Rc, m.Ac) * phase[None]
    err = np.abs(V - want).max() / np.abs(want).max()
    assert err < {40: 3e-4, 80: 8e-5}[n_int], err


def test_hartree_error_falls_with_the_knot_spacing():
    errs = []
    for n_int in (30, 60, 120):
        w = dataclasses.replace(_cell(grid=(8, 8)), breaks=W.uniform_breaks(-9.0, 9.0, n_int))
        m = Hm.model_from_workload(w)
        rho_g, gn, g = _sheet_rho(m, 0.8, (0.0, 0.0, 0.2))
        V = F.hartree_g(m, rho_g)
        want = -Hm.core_term(gn[None], (m.zb.zq - 0.2)[:, None, None], 1.0, 0.8, m.Ac)
        errs.append(np.abs(V - want).max())
    assert errs[1] < errs[0] / 3 and errs[2] < errs[1] / 3, errs


def test_xc_potential_is_the_derivative_of_the_energy_density():
    """v_xc = d(rho eps_xc)/d rho on both sides of r_s = 1 (central differences)."""
    rs = np.array([0.05, 0.3, 0.9, 1.2, 3.0, 10.0, 60.0, 400.0])
    n = 3.0 / (4.0 * math.pi * rs ** 3)
    v, _ = F.xc_pz(n)
    h = 1e-5 * n
    ep = F.xc_pz(n + h)[1] * (n + h)
    em = F.xc_pz(n - h)[1] * (n - h)
    assert np.abs(v - (ep - em) / (2 * h)).max() < 1e-8 * np.abs(v).max()


def test_xc_limits_and_continuity():
    # exchange of the uniform gas: -3 k_F / (4 pi), k_F = (3 pi^2 n)^(1/3)
    n = np.array([1e-4, 0.01, 0.3, 5.0])
    kF = (3 * math.pi ** 2 * n) ** (1.0 / 3.0)
    rs = (3.0 / (4.0 * math.pi * n)) ** (1.0 / 3.0)
    _, e = F.xc_pz(n)
    ec = e + 3 * kF / (4 * math.pi)
    # correlation alone: the high-density coefficient of ln r_s is (1 - ln 2)/pi^2
    assert abs(F.PZ_A - (1 - math.log(2)) / math.pi ** 2) < 2e-4
    # both branches meet at r_s = 1 (within the parametrization's rounding)
    n1 = 3.0 / (4.0 * math.pi)
    lo = F.xc_pz(np.array([n1 * (1 + 1e-12)]))
    hi = F.xc_pz(np.array([n1 * (1 - 1e-12)]))
    assert abs(lo[0][0] - hi[0][0]) < 1e-4 and abs(lo[1][0] - hi[1][0]) < 1e-4
    assert np.all(ec < 0) and np.all(np.diff(ec[np.argsort(rs)]) > 0)
    # below the floor (and for negative densities) the value at the floor:
    # continuous in rho, small, constant
    v0, e0 = F.xc_pz(np.array([0.0, -1e-9, 1e-40, F.RHO_FLOOR, 2 * F.RHO_FLOOR]))
    assert np.all(v0[:4] == v0[3]) and np.all(e0[:4] == e0[3])
    assert -1e-3 < v0[3] < 0 and v0[4] < v0[3]


def test_occupations_count_and_limits():
    rng = np.random.default_rng(2)
    ev = np.sort(rng.random((3, 6)), axis=1)
    kw = np.array([0.5, 0.25, 0.25])
    f, mu = F.occupations(ev, kw, 3.4, 0.02)
    assert abs(f.sum() - 3.4) < 1e-12
    assert np.all(f >= 0) and np.all(f <= 2 * kw[:, None] + 1e-15)
    f0, _ = F.occupations(ev, kw, 2.0, 1e-6)
    order = np.argsort((ev).ravel())
    # tiny width: the lowest states fill first
    filled = np.cumsum((2 * np.broadcast_to(kw[:, None], ev.shape)).ravel()[order])
    assert f0.ravel()[order[0]] > 0.99 * 2 * np.broadcast_to(kw[:, None], ev.shape).ravel()[order[0]]
    assert filled[0] <= 2.0


def test_pulay_coefficients_minimise_the_residual():
    """The bordered solve's combination has the least |sum a_i R_i| among
    coefficients summing to 1 (checked by a direct constrained minimization),
    and a single step is plain Kerker mixing."""
    m = Hm.model_from_workload(_cell(grid=(8, 8)))
    mx = F.Mixer(m, 0.4, 1.1)
    rng = np.random.default_rng(5)
    nq = len(m.zb.zq)
    rins = [rng.standard_normal((nq, 8, 8)) for _ in range(3)]
    routs = [r + 0.1 * rng.standard_normal((nq, 8, 8)) for r in rins]
    new1 = mx.step(rins[0], routs[0])
    kerker = F.to_r(F.to_g(rins[0]) + mx.kerker(F.to_g(routs[0]) - F.to_g(rins[0])))
    assert np.abs(new1 - kerker).max() < 1e-12
    mx.step(rins[1], routs[1])
    mx.step(rins[2], routs[2])
    R = [h[1] for h in mx.hist]
    A = np.array([[mx.dot(a, b) for b in R] for a in R])

    def obj(x):
        a = np.append(x, 1 - x.sum())
        return a @ A @ a

    best = optimize.minimize(obj, np.zeros(2), tol=1e-14).x
    a_best = np.append(best, 1 - best.sum())
    M = np.block([[A, np.ones((3, 1))], [np.ones((1, 3)), np.zeros((1, 1))]])
    a = np.linalg.solve(M, np.r_[0, 0, 0, 1.0])[:3]
    assert abs(obj(a[:2]) - obj(best)) < 1e-10 * obj(best)
    assert np.abs(a - a_best).max() < 1e-5


def test_kerker_factor_keeps_the_charge():
    """The paper's factor on g != 0; at g = 0 the factor of the first shell, a
    profile scaling, so a residual with no net charge moves none."""
    m = Hm.model_from_workload(_cell(grid=(8, 8)))
    mx = F.Mixer(m, 0.7, 0.8)
    _, gn = F.grid_freqs(m)
    g2 = gn * gn
    assert abs(mx.K[3, 1] - 0.7 * g2[3, 1] / (g2[3, 1] + 0.64)) < 1e-15
    g1 = np.min(g2[g2 > 0])
    assert abs(mx.K[0, 0] - 0.7 * g1 / (g1 + 0.64)) < 1e-15
    rng = np.random.default_rng(1)
    R = F.to_g(rng.standard_normal((len(m.zb.zq), 8, 8)))
    R[:, 0, 0] -= np.sum(m.zb.wq * R[:, 0, 0]) / np.sum(m.zb.wq)      # no net charge
    assert abs(np.sum(m.zb.wq * mx.kerker(R)[:, 0, 0])) < 1e-14


def test_scf_reaches_a_self_consistent_density():
    """At convergence the density built from the eigenvectors of H[V_scf]
    reproduces V_scf (the fixed point), and it holds nelec electrons."""
    w = _cell(nk=2)
    out = F.scf(w, nbands=4, nelec=2.0, sigma=0.02, W=0.6, gmax=1.2, tol=1e-8, max_iter=80)
    assert out["dv"] < 1e-8, out["iterations"]
    m0 = Hm.model_from_workload(w)
    ms = [Hm.model_from_workload(w, ik, table=out["vscf"]) for ik in range(w.nk)]
    evs, coefs = [], []
    for m in ms:
        ev, C = E.generalized_lowest(m.dense_H(), m.dense_S(), 4, vectors=True)
        evs.append(ev)
        coefs.append(C.T.reshape(4, m.nb, m.ng))
    f, _ = F.occupations(np.array(evs), np.full(w.nk, 1.0 / w.nk), 2.0, 0.02)
    rho = F.density(ms, coefs, f)
    assert abs(_integral(m0, rho) - 2.0) < 1e-10
    v = F.to_r(F.hartree_g(m0, F.to_g(rho))) + F.xc_pz(rho)[0]
    assert np.abs(v - out["vscf"]).max() < 1e-6
