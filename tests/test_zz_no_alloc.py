"""mb_apply_H_noalloc -- the H apply for callers that must not allocate device
memory while they run (a fixed device-memory budget owned by their own pool,
or a pipeline that cannot take the synchronization cudaMalloc/cudaFree may
cause).  Its scratch is a fixed array compiled into the library, shared by
every call, so the check runs the call twice in a row: the second call starts
from whatever the first one left in that array.

This file is collected last on purpose, and it needs nothing from the other
tests: it passes alone in a fresh process as well as after the full suite."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 2e-5}   # the parity tolerances of the apply tests


def _lib_and_mb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1406_4960_gb300 import mb
    return mb.load(build_if_missing=True), mb


@pytest.mark.parametrize("case,prec,ik", [("tiny", "fp64", 0), ("slab", "fp32", 1)])
def test_noalloc_matches_apply_H_on_two_calls(case, prec, ik):
    lib, mb = _lib_and_mb()
    from paper_1406_4960_gb300 import workloads as W
    w = W.tiny() if case == "tiny" else W.slab()
    h = mb.Handle.from_workload(w)
    ng, nb, ldg = h.sizes(ik)
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    code = mb.PREC[prec]
    ref = None
    for call in range(2):
        X = torch.from_numpy(W.random_block(w.nbands, nb, ng, seed=40 + call, ld=ldg)).to(dt).cuda()
        Y_ref = torch.zeros_like(X)
        Y = torch.full_like(X, complex(np.nan, np.nan))
        h.apply_H(ik, X, Y_ref, prec)
        rc = lib.mb_apply_H_noalloc(h._h, ik, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()),
                                    w.nbands, code, None)
        assert rc == 0, mb.ERRORS.get(rc)
        torch.cuda.synchronize()
        err = ((Y - Y_ref).abs().max() / Y_ref.abs().max()).item()
        assert err <= TOL[prec], (call, err)
        assert torch.all(Y[:, :, ng:] == 0)
        ref = Y
    assert ref is not None
    h.close()


def test_noalloc_rejects_requests_beyond_its_array():
    lib, mb = _lib_and_mb()
    from paper_1406_4960_gb300 import workloads as W
    w = W.graphene()
    h = mb.Handle.from_workload(w)
    ng, nb, ldg = h.sizes(0)
    X = torch.zeros((w.nbands, nb, ldg), dtype=torch.complex128, device="cuda")
    Y = torch.zeros_like(X)
    rc = lib.mb_apply_H_noalloc(h._h, 0, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()),
                                w.nbands, mb.MB_FP64, None)
    assert rc == 1   # MB_EINVAL: 80 FP64 bands of the 1417-G graphene cell need more than 16 MiB
    h.close()
