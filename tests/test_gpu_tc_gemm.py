"""tcgen05 building blocks (tensor memory accumulators).

* BF16 GEMM against a plain PyTorch FP32 matmul of the same BF16 operands.
  Products of BF16 values are exact in FP32; only the summation order
  differs, so the bound is a few FP32 ulps of sum |a||b|.
* The eigensolver's Gram A^H B of FP32 complex vectors (TF32 operands split
  as hi + lo, three products) against the FP64 product of the same FP32
  values: the split drops only lo*lo (2^-22 relative) and the accumulation is
  FP32 within a chunk, so the bound is 1e-5 of sum |a||b|."""
import ctypes

import numpy as np

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1406_4960_gb300 import mb
    l = mb.load(build_if_missing=True)
    l.mb_debug_gemm_bf16.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int] * 3 + [ctypes.c_void_p]
    l.mb_debug_gram_tc32.argtypes = [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    l.mb_debug_combine_ff.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_longlong, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    return l


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (300, 96, 368), (256, 224, 130), (130, 320, 96), (64, 16, 16)])
def test_tc_gemm_matches_fp32_matmul(lib, M, N, K):
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    Bt = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    D = torch.full((M, N), float("nan"), device="cuda", dtype=torch.float32)
    rc = lib.mb_debug_gemm_bf16(A.data_ptr(), Bt.data_ptr(), D.data_ptr(), M, N, K, None)
    assert rc == 0
    torch.cuda.synchronize()
    ref = A.float() @ Bt.float().T
    bound = 1e-5 * (A.float().abs() @ Bt.float().abs().T).max().item()
    assert (D - ref).abs().max().item() <= bound


# (ma, mb, n, nsplit): the solver's shapes (36 x 36 Gram-Schmidt products over
# a slab vector, the 5 x 41 Krylov rows), the largest tile, ragged chunk
# tails, chunks past the end of the vectors (empty CTAs), single vectors
@pytest.mark.parametrize("ma,mb,n,nsplit", [(36, 36, 23040, 76), (5, 41, 5000, 7), (64, 64, 1000, 3),
                                            (17, 9, 333, 5), (36, 36, 10, 16), (1, 1, 97, 2), (3, 64, 2049, 1)])
def test_tc_gram_matches_fp64(lib, ma, mb, n, nsplit):
    rng = np.random.default_rng(ma * 1000 + mb * 10 + nsplit)
    V = (rng.standard_normal((ma + mb, n)) + 1j * rng.standard_normal((ma + mb, n))).astype(np.complex64)
    V[:, ::7] *= 1e-3                                   # a spread of magnitudes
    Vd = torch.from_numpy(V).cuda()
    G = np.full(2 * ma * mb, np.nan)
    rc = lib.mb_debug_gram_tc32(Vd.data_ptr(), n, ma, mb, nsplit, G.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None)
    assert rc == 0
    G = G.reshape(ma, mb, 2)
    G = G[..., 0] + 1j * G[..., 1]
    A = V[:ma].astype(np.complex128)
    B = V[ma:].astype(np.complex128)
    ref = A.conj() @ B.T
    bound = 1e-5 * (np.abs(A) @ np.abs(B).T)
    assert np.all(np.abs(G - ref) <= bound)


def test_tc_gram_rejects_bad_sizes(lib):
    G = np.zeros(2)
    p = G.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    x = torch.zeros(8, dtype=torch.complex64, device="cuda")
    assert lib.mb_debug_gram_tc32(x.data_ptr(), 4, 1, 65, 1, p, None) == 1      # 2 mb > 128
    assert lib.mb_debug_gram_tc32(x.data_ptr(), 4, 65, 1, 1, p, None) == 1      # ma > 64
    assert lib.mb_debug_gram_tc32(x.data_ptr(), 0, 1, 1, 1, p, None) == 1       # empty vectors


# (ma, mc, n): the finish phase's root rotations (41 -> 36, 36 -> 36), a
# partial column group, a ragged element count
@pytest.mark.parametrize("ma,mc,n", [(41, 36, 23040), (36, 36, 5000), (7, 13, 999), (1, 9, 33)])
def test_float_float_rotation_matches_fp64(lib, ma, mc, n):
    """The mixed solver's FP64 root rotations run in float-float arithmetic;
    they must agree with an FP64 product to float-float accuracy: products
    keep 48 bits and each output sums 4 ma of them, so the error stays below
    ~4 ma 2^-48 of sum |a||y| (2e-12 here; the FP32 level would be 6e-8)."""
    rng = np.random.default_rng(ma * 100 + mc)
    A = rng.standard_normal((ma, n)) + 1j * rng.standard_normal((ma, n))
    A[:, ::5] *= 1e-6                                  # a spread of magnitudes
    Y = rng.standard_normal((ma, mc)) + 1j * rng.standard_normal((ma, mc))
    Y[0, :] *= 1e3
    Ad = torch.from_numpy(A).cuda()
    Cd = torch.full((mc, n), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
    Yh = np.ascontiguousarray(Y).view(np.float64)
    rc = lib.mb_debug_combine_ff(Ad.data_ptr(), Yh.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n, ma, mc,
                                 Cd.data_ptr(), None)
    assert rc == 0
    C = Cd.cpu().numpy()
    ref = Y.T @ A
    bound = 2e-12 * (np.abs(Y).T @ np.abs(A))
    assert np.all(np.abs(C - ref) <= bound)
