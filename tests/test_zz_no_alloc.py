"""mfipm_solve_noalloc: the solve for callers that cannot allocate device memory (it uses
the library's fixed device scratch instead of a caller workspace).  Its results must equal
those of mfipm_solve, call after call, although every call reuses the same scratch.
Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import workloads as W
from tests._lib import built_lib

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RELX_TOL = 1e-6


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return built_lib()


def _params(C, L, **kw):
    p = C.Params()
    L.mfipm_params_default(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _solve_both(L, C, op, b, tau, p, n):
    """One mfipm_solve (caller workspace) and two mfipm_solve_noalloc calls in a row."""
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    nb = ctypes.c_size_t()
    assert L.mfipm_workspace_size(ctypes.byref(op), 1, ctypes.byref(p), ctypes.byref(nb)) == 0
    ws = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
    x_ref = torch.empty(n, dtype=torch.float64, device="cuda")
    info = C.Info()
    rc = L.mfipm_solve(ctypes.byref(op), b.data_ptr(), tau, ctypes.byref(p), x_ref.data_ptr(), None,
                       ws.data_ptr(), nb.value, ctypes.byref(info), stream)
    assert rc == 0, L.mfipm_last_error()
    outs = []
    for _ in range(2):
        x = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        inf = C.Info()
        rc = L.mfipm_solve_noalloc(ctypes.byref(op), b.data_ptr(), tau, ctypes.byref(p), x.data_ptr(), None,
                                   ctypes.byref(inf), stream)
        assert rc == 0, L.mfipm_last_error()
        assert inf.status == 0
        outs.append(x.cpu().numpy())
    return x_ref.cpu().numpy(), outs


def test_noalloc_matches_workspace_solve_dct(L):
    from paper_1208_5435_gb300 import _capi as C
    pr = W.dct_problem(4096, 1024, 41, seed=90)
    rows = torch.from_numpy(pr.rows).cuda()
    b = torch.from_numpy(pr.b).cuda()
    op = C.Operator()
    op.kind, op.a_dtype, op.m, op.n, op.A, op.a_scale, op.lda, op.rows = (
        C.OP_PARTIAL_DCT, 0, pr.m, pr.n, None, 1.0, 0, rows.data_ptr())
    xr, outs = _solve_both(L, C, op, b, pr.tau, _params(C, L), pr.n)
    for x in outs:
        assert np.linalg.norm(x - xr) <= RELX_TOL * np.linalg.norm(xr)


def test_noalloc_matches_workspace_solve_dense(L):
    from paper_1208_5435_gb300 import _capi as C
    pr = W.dense_problem(128, 512, 8, seed=91)
    A = torch.from_numpy(pr.A).cuda()
    b = torch.from_numpy(pr.b).cuda()
    op = C.Operator()
    op.kind, op.a_dtype, op.m, op.n, op.A, op.a_scale, op.lda, op.rows = (
        C.OP_DENSE, C.A_F64, pr.m, pr.n, A.data_ptr(), 1.0, pr.n, None)
    xr, outs = _solve_both(L, C, op, b, pr.tau, _params(C, L, precision=C.PREC_FP64), pr.n)
    for x in outs:
        assert np.linalg.norm(x - xr) <= RELX_TOL * np.linalg.norm(xr)


def test_noalloc_rejects_problems_beyond_the_fixed_scratch(L):
    from paper_1208_5435_gb300 import _capi as C
    n = 65536
    rows = torch.arange(0, n, 4, dtype=torch.int64, device="cuda")
    b = torch.zeros(rows.numel(), dtype=torch.float64, device="cuda")
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    op = C.Operator()
    op.kind, op.a_dtype, op.m, op.n, op.A, op.a_scale, op.lda, op.rows = (
        C.OP_PARTIAL_DCT, 0, rows.numel(), n, None, 1.0, 0, rows.data_ptr())
    info = C.Info()
    rc = L.mfipm_solve_noalloc(ctypes.byref(op), b.data_ptr(), 0.1, ctypes.byref(_params(C, L)), x.data_ptr(), None,
                               ctypes.byref(info), None)
    assert rc == C.MFIPM_INVALID_ARG
    assert "scratch" in L.mfipm_last_error().decode()
