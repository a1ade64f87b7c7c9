"""GPU parity of the ultrasoft terms (§II.B.2) against the oracle: the
augmented overlap S = S_0 + sum q |beta><beta| in the S apply and in the
eigensolver (eigenvalues of H c = eps S c against the dense oracle), and the
self-consistent loop with strengths D = E + int V_eff Q and the augmented
density against the oracle's loop.  Tolerances as in the other parity
tests: applies 1e-10 (FP64) and 2e-5 (FP32) of max|Y|, eigenvalues 1e-6 Ha,
V_scf 1e-6 at a potential tolerance of 1e-8 Ha."""
import numpy as np
import pytest

from oracle import eigen as E
from oracle import hamiltonian as Hm
from oracle import scf as F
from paper_1406_4960_gb300 import workloads as W

from gpu_util import gmap, lib_block, oracle_block, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 2e-5}
EV_TOL = 1e-6


@pytest.fixture(scope="module")
def mbmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1406_4960_gb300 import mb
    mb.load(build_if_missing=True)
    return mb


def _cell(nproj=4, nk=2):
    a = 4.2
    kw = dict(e2s=-0.1, e12=0.05, Z=1.0, Rcore=0.5, q=(0.6, 0.3, 0.3, 0.3), q2s=0.25 if nproj == 5 else 0.0,
              q12=0.08 if nproj == 5 else 0.0, rQ=0.7)
    atoms = [W.Atom((0.7, 1.1, -0.6), -0.5, 0.8, nproj, (0.4, -0.2, -0.2, -0.2), 0.9, **kw),
             W.Atom((2.9, 3.0, 0.7), -0.5, 0.8, nproj, (0.4, -0.2, -0.2, -0.2), 0.9, **kw)]
    k = np.array([[0.0, 0.0], [0.31, -0.2]][:nk])
    return W.Workload("uspp", (a, 0.0), (0.35 * a, 0.93 * a), k, 4.0, W.uniform_breaks(-7.0, 7.0, 15),
                      6, 6, (16, 16), atoms, 4)


def _slab_uspp():
    w = W.with_core(W.scaled(W.slab(), ecut=6.0, n_int=23, nbands=5, name="slab-small"), 4.0, 0.6)
    return W.with_uspp(w, (0.5, 0.2, 0.2, 0.2), 0.8)


CASES = {"uspp4": lambda: _cell(4), "uspp5": lambda: _cell(5), "slab-small-uspp": _slab_uspp}


def _run(h, w, ik, X, prec, op):
    ng, nb, ldg = h.sizes(ik)
    m = Hm.model_from_workload(w, ik)
    perm = gmap(h, m, ik)
    cdt = np.complex128 if prec == "fp64" else np.complex64
    Xl = torch.from_numpy(lib_block(X, perm, ldg, cdt)).cuda()
    Yl = torch.full_like(Xl, complex(np.nan, np.nan))
    getattr(h, "apply_" + op)(ik, Xl, Yl, prec)
    torch.cuda.synchronize()
    Yh = Yl.cpu().numpy()
    assert np.all(Yh[:, :, ng:] == 0)
    return m, oracle_block(Yh, perm)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_augmented_S_and_H_match_oracle(mbmod, case, prec):
    w = CASES[case]()
    h = mbmod.Handle.from_workload(w)
    for ik in range(w.nk):
        ng, nb, ldg = h.sizes(ik)
        X = W.random_block(w.nbands, nb, ng, seed=500 + ik)
        m, Y = _run(h, w, ik, X, prec, "S")
        assert rel_err(Y, m.apply_S(X)) < TOL[prec], (case, ik, rel_err(Y, m.apply_S(X)))
        m, Y = _run(h, w, ik, X, prec, "H")
        assert rel_err(Y, m.apply_H(X)) < TOL[prec]
    h.close()


def test_augmented_S_inverse_is_refused(mbmod):
    w = _cell()
    h = mbmod.Handle.from_workload(w)
    ng, nb, ldg = h.sizes(0)
    X = torch.zeros((1, nb, ldg), dtype=torch.complex128, device="cuda")
    Y = torch.zeros_like(X)
    with pytest.raises(mbmod.MBError) as e:
        h.apply_Sinv(0, X, Y, "fp64")
    assert e.value.code == 6
    h.close()


@pytest.mark.parametrize("nproj", [4, 5])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_eigsolve_with_augmented_S_matches_dense(mbmod, nproj, prec):
    w = _cell(nproj)
    h = mbmod.Handle.from_workload(w)
    ev, info = h.eigsolve(w.nbands, 1e-8, prec)
    for ik in range(w.nk):
        m = Hm.model_from_workload(w, ik)
        ref = E.generalized_lowest(m.dense_H(), m.dense_S(), w.nbands)
        assert np.abs(ev[ik] - ref).max() < EV_TOL, (ik, ev[ik], ref)
    h.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_uspp_scf_matches_oracle(mbmod, prec):
    w = _cell()
    ref = F.scf(w, nbands=4, nelec=2.0, sigma=0.02, W=0.5, gmax=1.0, tol=1e-8, max_iter=80)
    h = mbmod.Handle.from_workload(w)
    vext = h.local_potential()
    ev, info = h.scf(4, 1e-8, 0.02, nelec=2.0, mix_weight=0.5, g_max=1.0, max_iter=80, eig_tol=1e-9, prec=prec)
    assert info.dv < 1e-8 and info.iterations > 3
    assert np.abs(ev - ref["evals"]).max() < 1e-6, (ev, ref["evals"])
    vscf = h.local_potential() - vext
    assert np.abs(vscf - ref["vscf"]).max() < 1e-6 * max(1.0, np.abs(ref["vscf"]).max())
    assert abs(info.nelec - 2.0) < 1e-8
    h.close()
