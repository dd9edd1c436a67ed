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


def _solve_both(L, C, op, b, tau, p, n, with_zs=False):
    """One mfipm_solve (caller workspace) and two mfipm_solve_noalloc calls in a row; with
    with_zs the final iterates (zs_out) are returned beside x."""
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    nb = ctypes.c_size_t()
    assert L.mfipm_workspace_size(ctypes.byref(op), 1, ctypes.byref(p), ctypes.byref(nb)) == 0
    ws = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
    x_ref = torch.empty(n, dtype=torch.float64, device="cuda")
    zs_ref = torch.empty(4 * n, dtype=torch.float64, device="cuda") if with_zs else None
    info = C.Info()
    rc = L.mfipm_solve(ctypes.byref(op), b.data_ptr(), tau, ctypes.byref(p), x_ref.data_ptr(),
                       zs_ref.data_ptr() if with_zs else None, ws.data_ptr(), nb.value, ctypes.byref(info), stream)
    assert rc == 0, L.mfipm_last_error()
    outs, zouts = [], []
    for _ in range(2):
        x = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        zs = torch.full((4 * n,), float("nan"), dtype=torch.float64, device="cuda") if with_zs else None
        inf = C.Info()
        rc = L.mfipm_solve_noalloc(ctypes.byref(op), b.data_ptr(), tau, ctypes.byref(p), x.data_ptr(),
                                   zs.data_ptr() if with_zs else None, ctypes.byref(inf), stream)
        assert rc == 0, L.mfipm_last_error()
        assert inf.status == 0
        outs.append(x.cpu().numpy())
        if with_zs:
            zouts.append(zs.cpu().numpy())
    if with_zs:
        return x_ref.cpu().numpy(), outs, zs_ref.cpu().numpy(), zouts
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


def _dense_op(C, pr, A):
    op = C.Operator()
    op.kind, op.a_dtype, op.m, op.n, op.A, op.a_scale, op.lda, op.rows = (
        C.OP_DENSE, C.A_F64, pr.m, pr.n, A.data_ptr(), 1.0, pr.n, None)
    return op


def test_noalloc_matches_workspace_solve_dense_fp32_pcg(L):
    """The dense operator with the float32 PCG layout (half the PCG bytes of the float64 one)."""
    from paper_1208_5435_gb300 import _capi as C
    pr = W.dense_problem(96, 384, 6, seed=92)
    A = torch.from_numpy(pr.A).cuda()
    b = torch.from_numpy(pr.b).cuda()
    xr, outs = _solve_both(L, C, _dense_op(C, pr, A), b, pr.tau, _params(C, L, precision=C.PREC_FP32_PCG), pr.n)
    for x in outs:
        assert np.linalg.norm(x - xr) <= RELX_TOL * np.linalg.norm(xr)


def test_noalloc_writes_the_final_iterate(L):
    """zs_out (the input of mfipm_backward) through the fixed scratch equals the workspace solve's."""
    from paper_1208_5435_gb300 import _capi as C
    pr = W.dct_problem(2048, 512, 20, seed=93)
    rows = torch.from_numpy(pr.rows).cuda()
    b = torch.from_numpy(pr.b).cuda()
    op = C.Operator()
    op.kind, op.a_dtype, op.m, op.n, op.A, op.a_scale, op.lda, op.rows = (
        C.OP_PARTIAL_DCT, 0, pr.m, pr.n, None, 1.0, 0, rows.data_ptr())
    xr, outs, zr, zouts = _solve_both(L, C, op, b, pr.tau, _params(C, L), pr.n, with_zs=True)
    for x, z in zip(outs, zouts):
        assert np.linalg.norm(x - xr) <= RELX_TOL * np.linalg.norm(xr)
        assert np.all(np.isfinite(z)) and np.all(z > 0)
        assert np.linalg.norm(z - zr) <= RELX_TOL * np.linalg.norm(zr)


def test_noalloc_serves_a_small_bf16_problem(L):
    """A dense bf16 A with MFIPM_PREC_BF16_A takes the shared-A solver, as in mfipm_solve."""
    from paper_1208_5435_gb300 import _capi as C
    pr = W.bf16_dense_problems(128, 512, 6, 1, seed=94)[0]
    bits = torch.from_numpy(pr.a_bf16.view(np.int16)).cuda()
    b = torch.from_numpy(pr.b).cuda()
    op = C.Operator()
    op.kind, op.a_dtype, op.m, op.n, op.A, op.a_scale, op.lda, op.rows = (
        C.OP_DENSE, C.A_BF16, pr.m, pr.n, bits.data_ptr(), pr.a_scale, pr.n, None)
    xr, outs = _solve_both(L, C, op, b, pr.tau, _params(C, L, precision=C.PREC_BF16_A), pr.n)
    for x in outs:
        assert np.linalg.norm(x - xr) <= RELX_TOL * np.linalg.norm(xr)
