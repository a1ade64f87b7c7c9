"""The C ABI driven straight through ctypes, without the package's binding:
mb_setup -> mb_sizes -> mb_gvectors -> mb_apply_H / mb_apply_S ->
mb_destroy on the tiny cell, the result against the oracle.  The structs are
declared here from include/mb.h alone, so a layout drift between the header,
the library and the binding shows up as a failure."""
import ctypes

import numpy as np
import pytest

from oracle import hamiltonian as Hm
from paper_1406_4960_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


class Cell(ctypes.Structure):
    _fields_ = [("a1", ctypes.c_double * 2), ("a2", ctypes.c_double * 2)]


class Atom(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_double * 3), ("A", ctypes.c_double), ("w", ctypes.c_double),
                ("nproj", ctypes.c_int), ("E", ctypes.c_double * 4), ("rc", ctypes.c_double),
                ("E2s", ctypes.c_double), ("E12", ctypes.c_double), ("Z", ctypes.c_double),
                ("Rcore", ctypes.c_double), ("q", ctypes.c_double * 4), ("q2s", ctypes.c_double),
                ("q12", ctypes.c_double), ("rQ", ctypes.c_double)]


class Opts(ctypes.Structure):
    _fields_ = [("n1", ctypes.c_int), ("n2", ctypes.c_int), ("nquad", ctypes.c_int),
                ("device", ctypes.c_int), ("max_bands", ctypes.c_int),
                ("precond_shift", ctypes.c_double)]


def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1406_4960_gb300 import build
    lib = ctypes.CDLL(build.build())
    D = ctypes.POINTER(ctypes.c_double)
    I = ctypes.POINTER(ctypes.c_int)
    V = ctypes.c_void_p
    lib.mb_setup.argtypes = [ctypes.POINTER(Cell), D, ctypes.c_int, ctypes.c_double, D, ctypes.c_int,
                             ctypes.c_int, ctypes.POINTER(Atom), ctypes.c_int, ctypes.POINTER(Opts),
                             ctypes.POINTER(V)]
    lib.mb_sizes.argtypes = [V, ctypes.c_int, I, I, I]
    lib.mb_gvectors.argtypes = [V, ctypes.c_int, I]
    lib.mb_apply_H.argtypes = [V, ctypes.c_int, V, V, ctypes.c_int, ctypes.c_int, V]
    lib.mb_apply_S.argtypes = [V, ctypes.c_int, V, V, ctypes.c_int, ctypes.c_int, V]
    lib.mb_destroy.argtypes = [V]
    lib.mb_destroy.restype = None
    return lib


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 2e-5)])
def test_raw_c_abi_apply_matches_oracle(prec, tol):
    lib = _lib()
    w = W.tiny()
    cell = Cell((ctypes.c_double * 2)(*w.a1), (ctypes.c_double * 2)(*w.a2))
    atoms = (Atom * len(w.atoms))()
    for i, a in enumerate(w.atoms):
        atoms[i].pos = (ctypes.c_double * 3)(*a.pos)
        atoms[i].A, atoms[i].w, atoms[i].nproj, atoms[i].rc = a.A, a.w, a.nproj, a.rc
        atoms[i].E = (ctypes.c_double * 4)(*a.E)
    kp = np.ascontiguousarray(w.kpts, dtype=np.float64)
    br = np.ascontiguousarray(w.breaks, dtype=np.float64)
    D = ctypes.POINTER(ctypes.c_double)
    opts = Opts(w.grid[0], w.grid[1], w.nquad, 0, 16, 0.0)
    h = ctypes.c_void_p()
    rc = lib.mb_setup(ctypes.byref(cell), kp.ctypes.data_as(D), kp.shape[0], w.ecut, br.ctypes.data_as(D),
                      len(br), w.order, atoms, len(w.atoms), ctypes.byref(opts), ctypes.byref(h))
    assert rc == 0 and h.value
    ng, nb, ldg = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    assert lib.mb_sizes(h, 0, ctypes.byref(ng), ctypes.byref(nb), ctypes.byref(ldg)) == 0
    ng, nb, ldg = ng.value, nb.value, ldg.value
    assert ldg % 32 == 0 and ldg >= ng
    idx = (ctypes.c_int * (2 * ng))()
    assert lib.mb_gvectors(h, 0, idx) == 0
    gl = np.array(idx[:], dtype=np.int64).reshape(ng, 2)
    m = Hm.model_from_workload(w)
    ora = {tuple(v): i for i, v in enumerate(m.gidx.tolist())}
    perm = np.array([ora[tuple(v)] for v in gl.tolist()])
    nbands = 3
    X = W.random_block(nbands, nb, ng, seed=17)
    Xl = np.zeros((nbands, nb, ldg), dtype=np.complex128 if prec == 0 else np.complex64)
    Xl[:, :, :ng] = X[:, :, perm]
    Xd = torch.from_numpy(Xl).cuda()
    for op, ref in ((lib.mb_apply_H, m.apply_H(X)), (lib.mb_apply_S, m.apply_S(X))):
        Yd = torch.zeros_like(Xd)
        assert op(h, 0, Xd.data_ptr(), Yd.data_ptr(), nbands, prec, None) == 0
        torch.cuda.synchronize()
        Y = np.zeros_like(X)
        Y[:, :, perm] = Yd.cpu().numpy()[:, :, :ng]
        assert np.abs(Y - ref).max() / np.abs(ref).max() < tol
    lib.mb_destroy(h)
