"""GPU parity of the self-consistent loop's device steps (§II.B.1, §III.A)
against the oracle: the density from given eigenvectors, the Coulomb
potential and the LDA potential of given densities, and the whole loop.

Tolerances: density, Hartree and LDA are FP64 on both sides with different
summation orders (the device's radix-2 FFTs and exponential sweeps against
numpy's FFT and the oracle's direct sums): 1e-11 of the largest value.  The
loops converge to the same fixed point along different paths (the device
eigensolver's vectors and the mixer's singular-history handling differ from
the oracle's dense solves): eigenvalues within 1e-6 Ha and V_scf within 1e-6
of the oracle's at a potential tolerance of 1e-8 Ha."""
import math

import numpy as np
import pytest

from oracle import eigen as E
from oracle import hamiltonian as Hm
from oracle import scf as F
from paper_1406_4960_gb300 import workloads as W

from gpu_util import gmap, lib_block

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELD_TOL = 1e-11


@pytest.fixture(scope="module")
def mbmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1406_4960_gb300 import mb
    mb.load(build_if_missing=True)
    return mb


def _cell(nk=2, grid=(16, 16)):
    a = 4.2
    atoms = [W.Atom((0.7, 1.1, -0.6), -0.5, 0.8, Z=1.0, Rcore=0.5),
             W.Atom((2.9, 3.0, 0.7), -0.5, 0.8, Z=1.0, Rcore=0.5)]
    k = np.array([[0.0, 0.0], [0.31, -0.2], [-0.12, 0.4]][:nk])
    return W.Workload("scf", (a, 0.0), (0.35 * a, 0.93 * a), k, 4.0, W.uniform_breaks(-7.0, 7.0, 15),
                      6, 6, grid, atoms, 4)


def _field(h):
    zq, _ = h.zplanes()
    return torch.zeros((len(zq), h.grid[0], h.grid[1]), dtype=torch.float64, device="cuda")


def _rel(a, b):
    return float(np.abs(a - b).max() / max(1e-300, np.abs(b).max()))


def test_density_matches_oracle(mbmod):
    w = _cell(nk=3)
    h = mbmod.Handle.from_workload(w)
    nbands = 3
    models, coefs, blocks = [], [], []
    rng = np.random.default_rng(8)
    occ = rng.random((w.nk, nbands))
    for ik in range(w.nk):
        m = Hm.model_from_workload(w, ik)
        ev, C = E.generalized_lowest(m.dense_H(), m.dense_S(), nbands, vectors=True)
        Co = C.T.reshape(nbands, m.nb, m.ng)
        models.append(m)
        coefs.append(Co)
        ng, nb, ldg = h.sizes(ik)
        blocks.append(lib_block(Co, gmap(h, m, ik), ldg, np.complex128).ravel())
    evecs = torch.from_numpy(np.concatenate(blocks)).cuda()
    rho = _field(h)
    h.density(evecs, nbands, occ, rho)
    ref = F.density(models, coefs, occ)
    assert _rel(rho.cpu().numpy(), ref) < FIELD_TOL
    # normalization: the integral is the sum of the occupations
    m = models[0]
    tot = float(np.sum(m.zb.wq[:, None, None] * rho.cpu().numpy()) * m.Ac / (w.grid[0] * w.grid[1]))
    assert abs(tot - occ.sum()) < 1e-11
    h.close()


def test_density_of_the_eigensolver_vectors_is_normalized(mbmod):
    w = _cell(nk=2)
    h = mbmod.Handle.from_workload(w)
    nbands = 4
    need = sum(nbands * h.sizes(ik)[1] * h.sizes(ik)[2] for ik in range(w.nk))
    evecs = torch.zeros(need, dtype=torch.complex128, device="cuda")
    h.eigsolve(nbands, 1e-9, "fp64", evecs=evecs)
    occ = np.full((w.nk, nbands), 0.5)
    rho = _field(h)
    h.density(evecs, nbands, occ, rho)
    m = Hm.model_from_workload(w)
    tot = float(np.sum(m.zb.wq[:, None, None] * rho.cpu().numpy()) * m.Ac / (w.grid[0] * w.grid[1]))
    assert abs(tot - occ.sum()) < 1e-9
    assert float(rho.min()) >= 0.0
    h.close()


@pytest.mark.parametrize("grid", [(16, 16), (8, 32)])
def test_hartree_matches_oracle(mbmod, grid):
    w = _cell(grid=grid)
    h = mbmod.Handle.from_workload(w)
    m = Hm.model_from_workload(w)
    rng = np.random.default_rng(3)
    rho_h = F.core_density(m) + 0.01 * rng.random((len(m.zb.zq),) + grid)
    rho = torch.from_numpy(rho_h).cuda()
    vh = _field(h)
    h.hartree(rho, vh)
    ref = F.to_r(F.hartree_g(m, F.to_g(rho_h)))
    assert _rel(vh.cpu().numpy(), ref) < FIELD_TOL
    h.close()


def test_xc_matches_oracle(mbmod):
    w = _cell()
    h = mbmod.Handle.from_workload(w)
    zq, _ = h.zplanes()
    shape = (len(zq),) + w.grid
    rng = np.random.default_rng(6)
    rs = np.exp(rng.uniform(np.log(0.02), np.log(200.0), shape))
    rho_h = 3.0 / (4.0 * math.pi * rs ** 3)
    rho_h.reshape(-1)[:5] = [0.0, -1e-6, 1e-31, 1e-9, 3.0 / (4.0 * math.pi)]
    rho = torch.from_numpy(rho_h).cuda()
    v, e = _field(h), _field(h)
    h.xc_lda(rho, v, e)
    torch.cuda.synchronize()
    vr, er = F.xc_pz(rho_h)
    assert _rel(v.cpu().numpy(), vr) < 1e-13 and _rel(e.cpu().numpy(), er) < 1e-13
    vf = v.cpu().numpy().reshape(-1)
    assert vf[0] == vf[1] == vf[2] and vf[3] < vf[0] < 0
    h.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_scf_matches_oracle(mbmod, prec):
    w = _cell(nk=2)
    kw = dict(nbands=4, nelec=2.0, sigma=0.02, W=0.6, gmax=1.2)
    ref = F.scf(w, tol=1e-8, max_iter=80, **kw)
    h = mbmod.Handle.from_workload(w)
    vext = h.local_potential()
    rho = _field(h)
    ev, info = h.scf(kw["nbands"], 1e-8, kw["sigma"], nelec=kw["nelec"], mix_weight=kw["W"], g_max=kw["gmax"],
                     max_iter=80, eig_tol=1e-9, prec=prec, rho_out=rho)
    assert info.dv < 1e-8 and info.iterations > 3
    assert np.abs(ev - ref["evals"]).max() < 1e-6, (ev, ref["evals"])
    vscf = h.local_potential() - vext
    assert np.abs(vscf - ref["vscf"]).max() < 1e-6 * max(1.0, np.abs(ref["vscf"]).max())
    assert abs(info.nelec - 2.0) < 1e-8
    h.close()


def test_scf_with_kpoint_weights_matches_oracle(mbmod):
    """Non-uniform k-point weights (3/4 and 1/4) enter the occupations."""
    w = _cell(nk=2)
    kw = np.array([0.75, 0.25])
    ref = F.scf(w, nbands=4, nelec=2.0, sigma=0.02, W=0.5, gmax=1.0, tol=1e-8, max_iter=80, kweights=kw)
    h = mbmod.Handle.from_workload(w)
    ev, info = h.scf(4, 1e-8, 0.02, nelec=2.0, mix_weight=0.5, g_max=1.0, max_iter=80, eig_tol=1e-9, prec="fp64",
                     kweights=kw)
    assert info.dv < 1e-8
    assert np.abs(ev - ref["evals"]).max() < 1e-6
    h.close()


def test_scf_rejects_bad_options(mbmod):
    """Invalid requests return MB_EINVAL before any work: no width, no
    tolerance, more electrons than the bands hold, weights not summing to 1,
    an unknown precision."""
    w = _cell(nk=2)
    h = mbmod.Handle.from_workload(w)
    bad = [dict(sigma=0.0), dict(tol=0.0), dict(nelec=9.0), dict(kweights=[0.5, 0.4]), dict(prec="bf16")]
    for b in bad:
        kw = dict(nbands=4, tol=1e-6, sigma=0.02, nelec=2.0)
        kw.update(b)
        with pytest.raises(mbmod.MBError) as e:
            h.scf(kw.pop("nbands"), kw.pop("tol"), kw.pop("sigma"), max_iter=3, **kw)
        assert e.value.code == 1, b
    h.close()


def test_density_of_more_kpoints_than_one_launch_holds(mbmod):
    """40 k-points (the density launches take 32 at a time) with random
    coefficient blocks: the chunked launches and the fixed-order partial sum
    against the oracle."""
    rng = np.random.default_rng(12)
    w = _cell(nk=1)
    kpts = rng.uniform(-0.4, 0.4, (40, 2))
    import dataclasses
    w = dataclasses.replace(w, kpts=kpts)
    h = mbmod.Handle.from_workload(w)
    nbands = 2
    models, coefs, blocks = [], [], []
    occ = rng.random((w.nk, nbands))
    for ik in range(w.nk):
        m = Hm.model_from_workload(w, ik)
        C = W.random_block(nbands, m.nb, m.ng, seed=600 + ik)
        models.append(m)
        coefs.append(C)
        ng, nb, ldg = h.sizes(ik)
        blocks.append(lib_block(C, gmap(h, m, ik), ldg, np.complex128).ravel())
    evecs = torch.from_numpy(np.concatenate(blocks)).cuda()
    rho = _field(h)
    h.density(evecs, nbands, occ, rho)
    ref = F.density(models, coefs, occ)
    assert _rel(rho.cpu().numpy(), ref) < FIELD_TOL
    h.close()
