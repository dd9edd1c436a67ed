"""The tcgen05/TMA bf16 GEMM of the shared-A solver against a plain PyTorch float32 product of
the same bf16 operands (and against the library's CUDA-core GEMM)."""
import ctypes

import pytest

from tests._lib import built_lib

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return built_lib()


def _run(L, A, B, splits, tensor_cores):
    rows, K = A.shape
    N = B.shape[0]
    C = torch.full((splits, N, rows), float("nan"), dtype=torch.float32, device="cuda")
    rc = L.mfipm_gemm_bf16(A.data_ptr(), B.data_ptr(), C.data_ptr(), rows, N, K, splits, tensor_cores,
                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, L.mfipm_last_error()
    return C.sum(0)


@pytest.mark.parametrize("rows,N,K,splits", [(128, 32, 64, 1), (256, 128, 1024, 1), (300, 16, 200, 1),
                                             (4096, 128, 16384, 4), (1000, 6, 520, 2), (512, 256, 4096, 3)])
def test_tensor_core_gemm_matches_fp32_reference(L, rows, N, K, splits):
    g = torch.Generator(device="cuda").manual_seed(rows + N + K)
    A = torch.randn(rows, K, generator=g, device="cuda").to(torch.bfloat16)
    B = torch.randn(N, K, generator=g, device="cuda").to(torch.bfloat16)
    ref = (A.float() @ B.float().T).T  # N x rows
    for mode in (1, 3):  # four- and three-stage rings
        C = _run(L, A, B, splits, mode)
        err = (C - ref).abs().max().item() / ref.abs().max().item()
        assert err <= 1e-5, (mode, err)
    if splits == 1:
        Cs = _run(L, A, B, 1, 0)
        assert (Cs - ref).abs().max().item() / ref.abs().max().item() <= 1e-5


def test_integer_digit_products_are_exact(L):
    """Integer bf16 digits |d| <= 128, as in the residual's slices: each split-K chunk of 1024
    products sums exactly in the float32 accumulator, up to the edge |sum| = 2^24."""
    rows, N, K, splits = 512, 64, 4096, 4  # chunks of 1024
    g = torch.Generator(device="cuda").manual_seed(5)
    A = torch.randint(-128, 129, (rows, K), generator=g, device="cuda")
    B = torch.randint(-128, 129, (N, K), generator=g, device="cuda")
    A[:8] = 128
    B[:4] = 128
    B[4:8] = -128  # chunk sums of exactly +-2^24
    Ab, Bb = A.to(torch.bfloat16), B.to(torch.bfloat16)
    assert torch.equal(Ab.long(), A) and torch.equal(Bb.long(), B)
    C = torch.full((splits, N, rows), float("nan"), dtype=torch.float32, device="cuda")
    rc = L.mfipm_gemm_bf16(Ab.data_ptr(), Bb.data_ptr(), C.data_ptr(), rows, N, K, splits, 1,
                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, L.mfipm_last_error()
    torch.cuda.synchronize()
    for sp in range(splits):
        k0, k1 = sp * 1024, (sp + 1) * 1024
        ref = (B[:, k0:k1].cpu() @ A[:, k0:k1].cpu().T)  # int64, N x rows
        assert torch.equal(C[sp].double().cpu(), ref.double()), sp
    assert C[0, 0, 0].item() == 2.0 ** 24
