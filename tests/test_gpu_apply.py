"""mfipm_apply_A / mfipm_apply_At / mfipm_kkt_residual against the oracle's float64
operator products and kkt_rel: partial DCT on both the direct (n < 1024) and the multi-pass
(n >= 1024, including the lockstep solver's sizes) arithmetic, dense float64 and bf16 A.
Every call gets exactly mfipm_workspace_size bytes of workspace."""
import numpy as np
import pytest

import workloads as W
from oracle import mfipm_oracle as O
from tests._lib import built_lib

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    built_lib()


def mf():
    import paper_1208_5435_gb300 as M
    return M


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _exact_ws(M, op):
    return torch.empty(M.workspace_bytes([op]), dtype=torch.uint8, device="cuda")


@pytest.mark.parametrize("n", [64, 512, 1024, 4096, 1 << 17])
def test_dct_products_match_oracle(n):
    M = mf()
    p = W.dct_problem(n, n // 4 + 3, max(1, n // 100), seed=95, j=n)
    op = M.PartialDCT(n, torch.from_numpy(p.rows))
    ref = O.Operator.from_dct_rows(n, p.rows, explicit=False)
    rng = np.random.default_rng(n)
    x, y = rng.standard_normal(n), rng.standard_normal(p.m)
    ws = _exact_ws(M, op)
    Ax = M.apply_A(op, torch.from_numpy(x), ws=ws).cpu().numpy()
    Aty = M.apply_At(op, torch.from_numpy(y), ws=ws).cpu().numpy()
    assert _rel(Ax, ref.mv(x)) <= 1e-12
    assert _rel(Aty, ref.rmv(y)) <= 1e-12
    assert abs(Ax @ y - x @ Aty) <= 1e-12 * np.linalg.norm(x) * np.linalg.norm(y)  # adjoint pair


@pytest.mark.parametrize("kind", ["f64", "bf16"])
def test_dense_products_match_numpy(kind):
    M = mf()
    if kind == "f64":
        p = W.dense_problem(96, 300, 6, seed=96)
        op, A = M.Dense(torch.from_numpy(p.A)), p.A
    else:
        p = W.bf16_dense_problems(64, 192, 4, 1, seed=97)[0]
        bits = torch.from_numpy(p.a_bf16.view(np.int16)).view(torch.bfloat16)
        op, A = M.DenseBF16(bits, p.a_scale), p.A
    rng = np.random.default_rng(7)
    x, y = rng.standard_normal(p.n), rng.standard_normal(p.m)
    ws = torch.empty(M.workspace_bytes([op], M.SolverParams(precision=2 if kind == "bf16" else None)),
                     dtype=torch.uint8, device="cuda")
    assert _rel(M.apply_A(op, torch.from_numpy(x), ws=ws).cpu().numpy(), A @ x) <= 1e-13
    assert _rel(M.apply_At(op, torch.from_numpy(y), ws=ws).cpu().numpy(), A.T @ y) <= 1e-13


@pytest.mark.parametrize("n", [256, 4096])
def test_kkt_residual_matches_oracle(n):
    M = mf()
    p = W.dct_problem(n, n // 4, max(1, n // 100), seed=98, j=n)
    op = M.PartialDCT(n, torch.from_numpy(p.rows))
    ref = O.Operator.from_dct_rows(n, p.rows, explicit=False)
    x_gpu, info = M.solve(op, torch.from_numpy(p.b), p.tau, M.SolverParams(tol=1e-12))
    x_rand = np.random.default_rng(8).standard_normal(n)
    for x in (x_gpu.cpu().numpy(), x_rand):
        k = M.kkt_residual(op, torch.from_numpy(p.b), p.tau, torch.from_numpy(x))
        ko = O.kkt_rel(ref, p.b, p.tau, x)
        assert abs(k - ko) <= 1e-9 * max(ko, 1e-12) + 1e-13, (k, ko)
    assert M.kkt_residual(op, torch.from_numpy(p.b), p.tau, x_gpu) <= 1e-6
    # x = 0 is optimal exactly when tau >= ||A^T b||_inf
    tau0 = 1.01 * float(np.abs(ref.rmv(p.b)).max())
    assert M.kkt_residual(op, torch.from_numpy(p.b), tau0, torch.zeros(n, dtype=torch.float64)) == 0.0


def test_bad_rows_rejected():
    M = mf()
    op = M.PartialDCT(4096, torch.tensor([5, 3, 9], dtype=torch.int64))
    from paper_1208_5435_gb300 import _capi as C
    with pytest.raises(C.MfipmError):
        M.apply_A(op, torch.zeros(4096, dtype=torch.float64))
