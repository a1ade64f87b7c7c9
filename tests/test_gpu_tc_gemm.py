"""tcgen05 BF16 GEMM building block (tensor memory accumulator) against a
plain PyTorch FP32 matmul of the same BF16 operands.  Products of BF16
values are exact in FP32; only the summation order differs, so the bound is
a few FP32 ulps of sum |a||b|."""
import ctypes

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
