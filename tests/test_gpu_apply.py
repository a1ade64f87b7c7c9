"""GPU parity of mb_apply_H / mb_apply_S / mb_apply_Sinv against the oracle.

Tolerances (max abs error / max |Y|):
* FP64: 1e-10.  The FFT path and the oracle's direct G-space contraction round
  differently; each is O(eps64 * log2(N1 N2) * kappa * nquad) relative, far
  below this bound.
* FP32: 2e-5.  float rounding of the FFT (~log2(N) * 6e-8), of the banded
  kinetic rows (|D| >> |Y| for smooth vectors, cancellation ~1e2 * 6e-8) and
  of the projector sums.
"""
import dataclasses

import numpy as np
import pytest

from oracle import hamiltonian as Hm
from paper_1406_4960_gb300 import workloads as W

from gpu_util import gmap, lib_block, oracle_block, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 2e-5}


@pytest.fixture(scope="module")
def mbmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1406_4960_gb300 import mb
    mb.load(build_if_missing=True)
    return mb


def _small_slab():
    w = W.slab()
    return W.scaled(w, ecut=6.0, n_int=23, nbands=5, name="slab-small")


def _small_graphene():
    w = W.graphene()
    return W.scaled(w, ecut=4.0, n_int=17, nbands=3, name="graphene-small")


def _small_kbatch():
    # 32x32 grid and 160-wide G rows: the FP64 register-FFT plane kernel then
    # runs 11 planes per group (an odd count, which once misaligned its
    # double-precision B-value table in shared memory)
    w = W.kbatch(4)
    return W.scaled(w, ecut=12.0, n_int=15, nbands=7, name="kbatch-small")


def _small_slab_2s():
    # second s channel (nproj = 5) with a 1s-2s coupling on every atom
    w = _small_slab()
    atoms = [dataclasses.replace(a, nproj=5, e2s=-0.35, e12=0.23) for a in w.atoms]
    return dataclasses.replace(w, atoms=atoms, name="slab2s-small")


def _order(w, k):
    # B-splines of order k with k Gauss points per interval: every order other
    # than 6 takes the radix-2 plane kernel, the order-k epilogue and S kernel
    # and the per-k-point S^-1 kernel
    return dataclasses.replace(w, order=k, nquad=k, name="%s-k%d" % (w.name, k))


CASES = {
    "tiny": lambda: W.tiny(),
    "tiny-k8": lambda: _order(W.tiny(), 8),
    "slab-small-k4": lambda: _order(_small_slab(), 4),
    "slab-small": _small_slab,
    "graphene-small": _small_graphene,
    "kbatch-small": _small_kbatch,
    "slab2s-small": _small_slab_2s,
}


def _run_apply(mbmod, h, w, ik, X, prec, op="H"):
    ng, nb, ldg = h.sizes(ik)
    m = Hm.model_from_workload(w, ik)
    perm = gmap(h, m, ik)
    cdt = np.complex128 if prec == "fp64" else np.complex64
    tdt = torch.complex128 if prec == "fp64" else torch.complex64
    Xl = torch.from_numpy(lib_block(X, perm, ldg, cdt)).cuda()
    Yl = torch.full_like(Xl, complex(np.nan, np.nan))
    getattr(h, "apply_" + op)(ik, Xl, Yl, prec)
    torch.cuda.synchronize()
    Yh = Yl.cpu().numpy()
    assert np.all(Yh[:, :, ng:] == 0), "padding columns must be written as zero"
    return m, oracle_block(Yh, perm)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_apply_H_matches_oracle(mbmod, case, prec):
    w = CASES[case]()
    h = mbmod.Handle.from_workload(w)
    for ik in range(w.nk):
        ng, nb, ldg = h.sizes(ik)
        X = W.random_block(w.nbands, nb, ng, seed=100 + ik)
        m, Y = _run_apply(mbmod, h, w, ik, X, prec)
        ref = m.apply_H(X)
        assert rel_err(Y, ref) < TOL[prec], (case, ik, rel_err(Y, ref))
    h.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_apply_S_and_Sinv(mbmod, prec):
    w = _small_slab()
    h = mbmod.Handle.from_workload(w)
    ng, nb, ldg = h.sizes(1)
    X = W.random_block(4, nb, ng, seed=7)
    m, Y = _run_apply(mbmod, h, w, 1, X, prec, "S")
    assert rel_err(Y, m.apply_S(X)) < TOL[prec]
    m, Z = _run_apply(mbmod, h, w, 1, X, prec, "Sinv")
    ref = np.einsum("ij,bjg->big", np.linalg.inv(m.S), X)
    assert rel_err(Z, ref) < (1e-11 if prec == "fp64" else 1e-4)
    h.close()


def test_apply_single_band_and_degenerate_inputs(mbmod):
    w = W.tiny()
    h = mbmod.Handle.from_workload(w)
    ng, nb, ldg = h.sizes(0)
    X = W.random_block(1, nb, ng, seed=3)
    m, Y = _run_apply(mbmod, h, w, 0, X, "fp64")
    assert rel_err(Y, m.apply_H(X)) < TOL["fp64"]
    Z = np.zeros((2, nb, ng), dtype=np.complex128)
    m, Y0 = _run_apply(mbmod, h, w, 0, Z, "fp64")
    assert np.all(Y0 == 0)
    h.close()


def test_apply_is_deterministic_and_batch_matches(mbmod):
    w = _small_slab()
    h = mbmod.Handle.from_workload(w)
    Xs, Ys = [], []
    for ik in range(w.nk):
        ng, nb, ldg = h.sizes(ik)
        X = W.random_block(w.nbands, nb, ng, seed=200 + ik, ld=ldg)
        Xs.append(torch.from_numpy(X).cuda())
        Ys.append(torch.zeros_like(Xs[-1]))
    h.apply_H_batch(list(range(w.nk)), Xs, Ys, "fp64")
    Y1 = [y.clone() for y in Ys]
    h.apply_H_batch(list(range(w.nk)), Xs, Ys, "fp64")
    for a, b in zip(Y1, Ys):
        assert torch.equal(a, b)
    for ik in range(w.nk):
        Yk = torch.zeros_like(Xs[ik])
        h.apply_H(ik, Xs[ik], Yk, "fp64")
        assert (Yk - Y1[ik]).abs().max().item() <= 1e-12 * Y1[ik].abs().max().item()
    h.close()


def test_local_potential_override_constant_shift(mbmod):
    """A caller table V = V0 everywhere turns the local term into V0 * S."""
    w = W.tiny()
    h = mbmod.Handle.from_workload(w)
    zq, wq = h.zplanes()
    V0 = 0.25
    h.set_local_potential(np.full((len(zq), w.grid[0], w.grid[1]), V0))
    ng, nb, ldg = h.sizes(0)
    X = W.random_block(2, nb, ng, seed=5)
    m0 = Hm.model_from_workload(w, with_atoms=False, local_components=[(0, 0, lambda z: V0)])
    perm = gmap(h, m0)
    Xl = torch.from_numpy(lib_block(X, perm, ldg, np.complex128)).cuda()
    Yl = torch.zeros_like(Xl)
    h.apply_H(0, Xl, Yl, "fp64")
    Y = oracle_block(Yl.cpu().numpy(), perm)
    assert rel_err(Y, m0.apply_H(X)) < TOL["fp64"]
    h.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_slab_batch_matches_oracle(mbmod, prec):
    """All 4 k-points x 32 bands of the C(001)-like slab in one batched apply
    (the launch the benchmark times), every output element against the
    oracle's matrix-free apply."""
    w = W.slab()
    h = mbmod.Handle.from_workload(w)
    cdt = np.complex128 if prec == "fp64" else np.complex64
    Xs, Ys, Xo, perms, models = [], [], [], [], []
    for ik in range(w.nk):
        ng, nb, ldg = h.sizes(ik)
        m = Hm.model_from_workload(w, ik)
        perm = gmap(h, m, ik)
        X = W.random_block(w.nbands, nb, ng, seed=300 + ik)
        Xo.append(X)
        perms.append(perm)
        models.append(m)
        Xs.append(torch.from_numpy(lib_block(X, perm, ldg, cdt)).cuda())
        Ys.append(torch.full_like(Xs[-1], complex(np.nan, np.nan)))
    h.apply_H_batch(list(range(w.nk)), Xs, Ys, prec)
    torch.cuda.synchronize()
    for ik in range(w.nk):
        Yh = Ys[ik].cpu().numpy()
        assert np.all(Yh[:, :, len(perms[ik]):] == 0)
        Y = oracle_block(Yh, perms[ik])
        ref = models[ik].apply_H(Xo[ik])
        assert rel_err(Y, ref) < TOL[prec], (ik, rel_err(Y, ref))
    h.close()


@pytest.fixture(scope="module")
def graphene_ref():
    """The full 4x4 graphene cell (1417 G, 80 splines, 128 projectors, 64x64
    grid) with an 80-band block, and the oracle's H X of it."""
    w = W.graphene()
    m = Hm.model_from_workload(w)
    X = W.random_block(w.nbands, m.nb, m.ng, seed=9)
    return w, m, X, m.apply_H(X)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_graphene_matches_oracle(mbmod, graphene_ref, prec):
    w, m, X, ref = graphene_ref
    h = mbmod.Handle.from_workload(w)
    ng, nb, ldg = h.sizes(0)
    perm = gmap(h, m)
    cdt = np.complex128 if prec == "fp64" else np.complex64
    Xl = torch.from_numpy(lib_block(X, perm, ldg, cdt)).cuda()
    Yl = torch.full_like(Xl, complex(np.nan, np.nan))
    h.apply_H(0, Xl, Yl, prec)
    torch.cuda.synchronize()
    Yh = Yl.cpu().numpy()
    assert np.all(Yh[:, :, ng:] == 0)
    Y = oracle_block(Yh, perm)
    assert rel_err(Y, ref) < TOL[prec], rel_err(Y, ref)
    h.close()


def test_invalid_arguments_are_rejected(mbmod):
    w = W.tiny()
    with pytest.raises(mbmod.MBError):
        mbmod.Handle(w.a1, w.a2, w.kpts, w.ecut, w.breaks, w.order, w.atoms, (4, 4))  # grid too small for the disc
    with pytest.raises(mbmod.MBError):
        mbmod.Handle(w.a1, w.a2, w.kpts, w.ecut, w.breaks[::-1], w.order, w.atoms, w.grid)
    with pytest.raises(mbmod.MBError):
        mbmod.Handle(w.a1, w.a2, w.kpts, w.ecut, w.breaks, w.order, w.atoms, (12, 16))  # not 2^n
    h = mbmod.Handle.from_workload(w)
    ng, nb, ldg = h.sizes(0)
    X = torch.zeros((2, nb, ldg), dtype=torch.complex128, device="cuda")
    Y = torch.zeros_like(X)
    assert h._lib.mb_apply_H(h._h, 5, X.data_ptr(), Y.data_ptr(), 2, 0, None) == 1   # bad k index
    assert h._lib.mb_apply_H(h._h, 0, X.data_ptr(), Y.data_ptr(), 0, 0, None) == 1   # no bands
    assert h._lib.mb_apply_H(h._h, 0, X.data_ptr(), Y.data_ptr(), 2, 7, None) == 1   # bad precision
    with pytest.raises(mbmod.MBError):
        h.apply_H(0, X, torch.zeros((2, nb, ldg), dtype=torch.complex64, device="cuda"))  # dtype
    with pytest.raises(mbmod.MBError):
        h.apply_H(0, X, X)                            # in place is not allowed
    zq, _ = h.zplanes()
    with pytest.raises(mbmod.MBError):
        h.set_local_potential(np.full((3,), 1.0))     # wrong size
    with pytest.raises(mbmod.MBError):
        h.set_local_potential(np.full((len(zq), 16, 16), np.nan))
    h.close()


# BF16 keeps 8 significant bits: unit roundoff u = 2^-8.  Each product of the
# two tensor-core contractions (W = X^T conj(q) and the back-projection C q)
# has both operands rounded, a relative error of about 2u; with independent
# rounding errors a sum of such products is off by about 2u of its value, so
# the projector term carries about 2 * 2u = 1.6e-2 of its own size.  2e-2 of
# the largest projector element is asserted.
BF16_NL_TOL = 2e-2


def _zero_kb(w):
    return dataclasses.replace(w, atoms=[dataclasses.replace(a, E=(0.0, 0.0, 0.0, 0.0), e2s=0.0, e12=0.0)
                                         for a in w.atoms])


@pytest.mark.parametrize("case", ["slab-small", "graphene-small", "slab2s-small"])
def test_apply_bf16_projector_contraction_on_tensor_cores(mbmod, case):
    """MB_BF16 runs both projector contractions on the tensor cores (tcgen05,
    BF16 operands, FP32 accumulation).  Its projector part, isolated as
    H X - H_{E=0} X, matches the FP32 path within the BF16 bound above."""
    w = CASES[case]()
    h = mbmod.Handle.from_workload(w)
    h0 = mbmod.Handle.from_workload(_zero_kb(w))
    for ik in range(w.nk):
        ng, nb, ldg = h.sizes(ik)
        X = torch.from_numpy(W.random_block(w.nbands, nb, ng, seed=60 + ik, ld=ldg)).to(torch.complex64).cuda()
        Y32, Y16, Yloc = (torch.zeros_like(X) for _ in range(3))
        h.apply_H(ik, X, Y32, "fp32")
        h.apply_H(ik, X, Y16, "bf16")
        h0.apply_H(ik, X, Yloc, "fp32")
        torch.cuda.synchronize()
        nl32, nl16 = Y32 - Yloc, Y16 - Yloc
        scale = nl32.abs().max().item()
        assert scale > 0
        assert (nl16 - nl32).abs().max().item() <= BF16_NL_TOL * scale, (ik, (nl16 - nl32).abs().max().item() / scale)
    h.close()
    h0.close()


@pytest.mark.parametrize("case", ["slab-small", "graphene-small", "slab2s-small"])
def test_apply_bf16_matches_oracle(mbmod, case):
    """The whole MB_BF16 apply against the FP64 oracle: within the FP32
    tolerance of the local and kinetic part plus the BF16 bound of the
    projector part (the oracle's H X - H_{E=0} X sets its size)."""
    w = CASES[case]()
    h = mbmod.Handle.from_workload(w)
    for ik in range(w.nk):
        ng, nb, ldg = h.sizes(ik)
        X = W.random_block(w.nbands, nb, ng, seed=80 + ik)
        m, Y = _run_apply(mbmod, h, w, ik, X, "bf16")
        ref = m.apply_H(X)
        nl = ref - Hm.model_from_workload(_zero_kb(w), ik).apply_H(X)
        bound = TOL["fp32"] * np.abs(ref).max() + BF16_NL_TOL * np.abs(nl).max()
        err = np.abs(Y - ref).max()
        assert err <= bound, (ik, err, bound)
    h.close()


@pytest.mark.parametrize("case", ["tiny", "slab-small", "graphene-small", "kbatch-small"])
def test_every_plane_kernel_instance_matches_oracle(mbmod, case):
    """Every compiled compact-plane instance that can run the batch (the
    autotuner may pick any of them), as a static grid and as a persistent
    work-queue launch, and the register-FFT kernel beside them, with two run
    counts each, against the oracle in FP32.  The persistent launches run
    back to back, so each starts from the counters the previous one reset."""
    w = CASES[case]()
    h = mbmod.Handle.from_workload(w)
    ids = h.plane_kernel_candidates(w.nk, w.nbands, "fp32")
    assert ids, "no compact-plane instance for %s" % case
    Xs, perms, models, Xo = [], [], [], []
    for ik in range(w.nk):
        ng, nb, ldg = h.sizes(ik)
        m = Hm.model_from_workload(w, ik)
        perm = gmap(h, m, ik)
        X = W.random_block(w.nbands, nb, ng, seed=900 + ik)
        Xo.append(X)
        perms.append(perm)
        models.append(m)
        Xs.append(torch.from_numpy(lib_block(X, perm, ldg, np.complex64)).cuda())
    refs = [models[ik].apply_H(Xo[ik]) for ik in range(w.nk)]
    for kid in ids + [-2]:
        for waves, persistent in ((0, False), (8, False), (0, True), (8, True)):
            if kid == -2 and persistent:
                continue
            h.plane_kernel_select(w.nk, w.nbands, "fp32", kid, waves, persistent)
            Ys = [torch.full_like(x, complex(np.nan, np.nan)) for x in Xs]
            h.apply_H_batch(list(range(w.nk)), Xs, Ys, "fp32")
            torch.cuda.synchronize()
            for ik in range(w.nk):
                Yh = Ys[ik].cpu().numpy()
                assert np.all(Yh[:, :, len(perms[ik]):] == 0)
                err = rel_err(oracle_block(Yh, perms[ik]), refs[ik])
                assert err < TOL["fp32"], (case, h.plane_kernel_name(w.nk, w.nbands, "fp32"), waves, ik, err)
    h.close()


@pytest.mark.parametrize("case", ["slab", "slab-small", "slab-small-k4", "graphene-small", "tiny-k8"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_apply_S_and_Sinv_batched_match_oracle(mbmod, case, prec):
    """S X and S^-1 X for every k-point in one batched call (S: the TMA-staged
    tile kernel at every order; S^-1: the tile kernel at order 6, the
    per-k-point kernel at orders 4 and 8) against the oracle's S and a dense
    inverse of it, every element."""
    w = W.slab() if case == "slab" else CASES[case]()
    h = mbmod.Handle.from_workload(w)
    cdt = np.complex128 if prec == "fp64" else np.complex64
    Xs, Xo, perms, models = [], [], [], []
    for ik in range(w.nk):
        ng, nb, ldg = h.sizes(ik)
        m = Hm.model_from_workload(w, ik)
        perm = gmap(h, m, ik)
        X = W.random_block(w.nbands, nb, ng, seed=1300 + ik)
        Xo.append(X)
        perms.append(perm)
        models.append(m)
        Xs.append(torch.from_numpy(lib_block(X, perm, ldg, cdt)).cuda())
    iks = list(range(w.nk))
    for op in ("S", "Sinv"):
        Ys = [torch.full_like(x, complex(np.nan, np.nan)) for x in Xs]
        getattr(h, "apply_%s_batch" % op)(iks, Xs, Ys, prec)
        h.status()
        for ik in iks:
            Yh = Ys[ik].cpu().numpy()
            assert np.all(Yh[:, :, len(perms[ik]):] == 0)
            Y = oracle_block(Yh, perms[ik])
            m = models[ik]
            ref = m.apply_S(Xo[ik]) if op == "S" else np.einsum("ij,bjg->big", np.linalg.inv(m.S), Xo[ik])
            tol = TOL[prec] if op == "S" else (1e-11 if prec == "fp64" else 1e-4)
            assert rel_err(Y, ref) < tol, (op, ik, rel_err(Y, ref))
    h.close()


def test_largest_grid_radix2_fallback_and_fp64_refusal(mbmod):
    """A 128 x 128 grid: beyond the register-FFT and compact-plane kernels,
    the FP32 apply takes the radix-2 plane kernel (one 128 KB plane in shared
    memory) and matches the oracle; an FP64 plane (256 KB) does not fit in
    shared memory, and the FP64 apply is refused with MB_EUNSUPPORTED instead
    of launching."""
    w = dataclasses.replace(W.tiny(), grid=(128, 128), nbands=3, name="tiny-128")
    h = mbmod.Handle.from_workload(w)
    ng, nb, ldg = h.sizes(0)
    X = W.random_block(w.nbands, nb, ng, seed=21)
    m, Y = _run_apply(mbmod, h, w, 0, X, "fp32")
    assert rel_err(Y, m.apply_H(X)) < TOL["fp32"]
    Xd = torch.zeros((w.nbands, nb, ldg), dtype=torch.complex128, device="cuda")
    with pytest.raises(mbmod.MBError) as e:
        h.apply_H(0, Xd, torch.zeros_like(Xd), "fp64")
    assert e.value.code == 6
    h.close()
