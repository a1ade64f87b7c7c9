"""mb_apply_H_noalloc -- the H apply for callers that must not allocate device
memory while they run (a fixed device-memory budget owned by their own pool,
or a pipeline that cannot take the synchronization cudaMalloc/cudaFree may
cause).  Its scratch is a fixed array compiled into the library, shared by
every call, so the checks run it twice in a row, and each checked call comes
right after a call of another shape, so that it starts from the unrelated
leftovers of that call in the array.

This file is collected last on purpose, and it needs nothing from the other
tests: it passes alone in a fresh process as well as after the full suite."""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 2e-5, "bf16": 2e-5}   # the parity tolerances of the apply tests
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib_and_mb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1406_4960_gb300 import mb
    return mb.load(build_if_missing=True), mb


def _noalloc(lib, h, ik, X, Y, nbands, code):
    return lib.mb_apply_H_noalloc(h._h, ik, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()),
                                  nbands, code, None)


@pytest.mark.parametrize("case,prec,ik", [("tiny", "fp64", 0), ("slab", "fp32", 1), ("slab", "bf16", 2)])
def test_noalloc_matches_apply_H_on_two_calls(case, prec, ik):
    lib, mb = _lib_and_mb()
    from paper_1406_4960_gb300 import workloads as W
    w = W.tiny() if case == "tiny" else W.slab()
    h = mb.Handle.from_workload(w)
    ng, nb, ldg = h.sizes(ik)
    dt = torch.complex128 if prec == "fp64" else torch.complex64
    code = mb.PREC[prec]
    # a call of another shape, run before each checked call
    wo = W.slab() if case == "tiny" else W.tiny()
    ho = mb.Handle.from_workload(wo)
    po = "fp32" if case == "tiny" else "fp64"
    ngo, nbo, ldgo = ho.sizes(0)
    Xo = torch.from_numpy(W.random_block(wo.nbands, nbo, ngo, seed=7, ld=ldgo)).to(
        torch.complex64 if po == "fp32" else torch.complex128).cuda()
    Yo = torch.zeros_like(Xo)
    for call in range(2):
        assert _noalloc(lib, ho, 0, Xo, Yo, wo.nbands, mb.PREC[po]) == 0
        X = torch.from_numpy(W.random_block(w.nbands, nb, ng, seed=40 + call, ld=ldg)).to(dt).cuda()
        Y_ref = torch.zeros_like(X)
        Y = torch.full_like(X, complex(np.nan, np.nan))
        h.apply_H(ik, X, Y_ref, prec)
        rc = _noalloc(lib, h, ik, X, Y, w.nbands, code)
        assert rc == 0, mb.ERRORS.get(rc)
        torch.cuda.synchronize()
        err = ((Y - Y_ref).abs().max() / Y_ref.abs().max()).item()
        assert err <= TOL[prec], (call, err)
        assert torch.all(Y[:, :, ng:] == 0)
    ho.close()
    h.close()


def test_noalloc_rejects_requests_beyond_its_array():
    lib, mb = _lib_and_mb()
    from paper_1406_4960_gb300 import workloads as W
    w = W.graphene()
    h = mb.Handle.from_workload(w)
    ng, nb, ldg = h.sizes(0)
    X = torch.zeros((w.nbands, nb, ldg), dtype=torch.complex128, device="cuda")
    Y = torch.zeros_like(X)
    rc = _noalloc(lib, h, 0, X, Y, w.nbands, mb.MB_FP64)
    assert rc == 1   # MB_EINVAL: 80 FP64 bands of the 1417-G graphene cell need more than 16 MiB
    h.close()


def test_noalloc_first_call_inside_a_capture_is_refused():
    """In a fresh process, the first call on the device made while its
    stream is being captured gets MB_EINVAL (the array's address can only be
    looked up outside a capture); nothing is launched."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    code = r'''
import ctypes, sys, torch
sys.path.insert(0, sys.argv[1])
from paper_1406_4960_gb300 import mb, workloads as W
lib = mb.load()
w = W.tiny()
h = mb.Handle.from_workload(w)
ng, nb, ldg = h.sizes(0)
X = torch.zeros((2, nb, ldg), dtype=torch.complex128, device="cuda")
Y = torch.zeros_like(X)
s = torch.cuda.Stream()
g = torch.cuda.CUDAGraph()
with torch.cuda.graph(g, stream=s):
    rc = lib.mb_apply_H_noalloc(h._h, 0, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()), 2, 0,
                                ctypes.c_void_p(s.cuda_stream))
print("RC", rc)
h.close()
'''
    out = subprocess.run([sys.executable, "-c", code, ROOT], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    assert "RC 1" in out.stdout, out.stdout
