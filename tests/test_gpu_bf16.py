"""Shared-A multi-right-hand-side solver (bf16 A with a per-tensor scale): parity with the
float64 oracle, which uses the exact matrix a_scale * bf16(A)."""
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


def _solve(probs, **kw):
    import paper_1208_5435_gb300 as M
    bits = torch.from_numpy(probs[0].a_bf16.view(np.int16)).view(torch.bfloat16).cuda()
    op = M.DenseBF16(bits, probs[0].a_scale)
    xs, infos = M.solve_batched([op] * len(probs), [torch.from_numpy(p.b) for p in probs], [p.tau for p in probs],
                                M.SolverParams(**kw))
    return [x.cpu().numpy() for x in xs], infos


def test_shared_bf16_matches_oracle_small():
    probs = W.bf16_dense_problems(512, 2048, 20, 8, seed=2001)
    xs, infos = _solve(probs, tol=1e-12)
    op = O.Operator.from_dense(probs[0].A)
    for p, x, info in zip(probs, xs, infos):
        assert info["status"] == 0, info
        xo = O.ipm(op, p.b, p.tau).x
        assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo), (np.linalg.norm(x - xo) / np.linalg.norm(xo), info)


def test_shared_bf16_uneven_columns_and_odd_sizes():
    probs = W.bf16_dense_problems(200, 700, 9, 3, seed=2002)
    xs, infos = _solve(probs, tol=1e-12)
    op = O.Operator.from_dense(probs[0].A)
    for p, x, info in zip(probs, xs, infos):
        assert info["status"] == 0
        xo = O.ipm(op, p.b, p.tau).x
        assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)


def test_shared_bf16_cuda_core_gemm_agrees():
    """The solver with the CUDA-core GEMM reaches the same minimisers as with tcgen05."""
    import paper_1208_5435_gb300 as M
    probs = W.bf16_dense_problems(256, 1024, 10, 4, seed=2003)
    xt, _ = _solve(probs, tol=1e-12)
    M.lib().mfipm_set_gemm_mode(0)
    try:
        xs, infos = _solve(probs, tol=1e-12)
    finally:
        M.lib().mfipm_set_gemm_mode(1)
    for a, b in zip(xt, xs):
        assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(b)


def test_shared_bf16_full_size_certificates():
    """4096 x 16384, 64 right-hand sides: every column reaches kkt_rel <= 1e-6 (float64,
    computed on the GPU) and four columns are re-certified on the CPU."""
    probs = W.make_workload("bf16_4096x16384_64rhs")
    xs, infos = _solve(probs)
    assert all(i["status"] == 0 and i["kkt_rel"] <= 1e-6 for i in infos), [i["kkt_rel"] for i in infos][:8]
    op = O.Operator.from_dense(probs[0].A)
    for j in (0, 17, 42, 63):
        k = O.kkt_rel(op, probs[j].b, probs[j].tau, xs[j])
        assert k <= 1e-6
        P, D = O.dual_gap_certificate(op, probs[j].b, probs[j].tau, xs[j])
        assert 0 <= P - D <= 1e-5 * (1 + abs(P))  # certificate slack at the default gap tolerance


def test_residual_modes_agree():
    """The residual by exact digit slices on the tensor cores (default) and by the biased
    float32 accumulator on the CUDA cores reach the same minimisers, both at the oracle's."""
    import paper_1208_5435_gb300 as M
    probs = W.bf16_dense_problems(256, 1024, 10, 6, seed=2004)
    op = O.Operator.from_dense(probs[0].A)
    xt, it = _solve(probs, tol=1e-12)
    M.lib().mfipm_set_residual_mode(0)
    try:
        xc, ic = _solve(probs, tol=1e-12)
    finally:
        M.lib().mfipm_set_residual_mode(1)
    for p, a, b, i1, i2 in zip(probs, xt, xc, it, ic):
        assert i1["status"] == 0 and i2["status"] == 0
        xo = O.ipm(op, p.b, p.tau).x
        assert np.linalg.norm(a - xo) <= 1e-6 * np.linalg.norm(xo)
        assert np.linalg.norm(a - b) <= 1e-7 * np.linalg.norm(b)
