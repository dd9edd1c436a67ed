"""The corrector of the Algorithm (Sec. 5.1, reading R6) on every solver path, against the
float64 oracle run with the same alpha_tilde.

With the paper's alpha_tilde = 0.1 the corrector test (alpha_P or alpha_D <= alpha_tilde)
rarely fires on these well-conditioned problems, so a mistake in the trial point, its
right-hand side or the combined step could hide behind the predictor.  alpha_tilde = 1
makes the test true at every iteration (step lengths never exceed 1): every direction is
then predictor + corrector on both sides, and x must still match the oracle's minimiser."""
import ctypes

import numpy as np
import pytest

import workloads as W
from oracle import mfipm_oracle as O
from tests._lib import built_lib

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RELX_TOL = 1e-6
EVERY = dict(alpha_tilde=1.0, tol=1e-12)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    built_lib()


def mf():
    import paper_1208_5435_gb300 as M
    return M


def relx(x, xo):
    return np.linalg.norm(x - xo) / max(np.linalg.norm(xo), 1e-300)


def oracle_every(op, p):
    res = O.ipm(op, p.b, p.tau, O.OracleParams(alpha_tilde=1.0))
    assert res.converged and res.correctors == res.iters - 1 > 0
    return res


def check(info, x, res):
    assert info["status"] == 0, info
    # every iteration that computed a direction took a corrector
    assert info["correctors"] == info["ipm_iters"] > 0, info
    assert relx(x, res.x) <= RELX_TOL, (relx(x, res.x), info)
    # the combined steps stay in the same iteration band as the exact-direction oracle
    assert abs(info["ipm_iters"] - (res.iters - 1)) <= 8, (info, res.iters)


@pytest.mark.parametrize("n,G,outer", [(1024, 1, 0), (1024, 4, 0), (4096, 1, 0), (4096, 8, 0),
                                       (1024, 2, 1), (4096, 1, 1)])
def test_persistent_dct_corrector_every_iteration(n, G, outer):
    M = mf()
    p = W.dct_problem(n, n // 4, max(1, n // 100), seed=311, j=n)
    res = oracle_every(O.Operator.from_dct_rows(p.n, p.rows), p)
    x, info = M.solve(M.PartialDCT(p.n, torch.from_numpy(p.rows)), torch.from_numpy(p.b), p.tau,
                      M.SolverParams(cluster_size=G, outer=outer, **EVERY))
    check(info, x.cpu().numpy(), res)


@pytest.mark.parametrize("precision", [0, 1])
def test_dense_corrector_every_iteration(precision):
    M = mf()
    p = W.dense_problem(128, 512, 10, seed=312)
    res = oracle_every(O.Operator.from_dense(p.A), p)
    x, info = M.solve(M.Dense(torch.from_numpy(p.A)), torch.from_numpy(p.b), p.tau,
                      M.SolverParams(precision=precision, **EVERY))
    check(info, x.cpu().numpy(), res)


def test_persistent_batch_corrector_every_iteration():
    """Both phases of the persistent kernel (cluster problems and single-CTA problems)."""
    M = mf()
    ns = [4096, 256, 1024, 2048, 512, 4096]
    probs = [W.dct_problem(n, n // 4, max(1, n // 60), seed=313, j=j) for j, n in enumerate(ns)]
    ops = [M.PartialDCT(p.n, torch.from_numpy(p.rows)) for p in probs]
    xs, infos = M.solve_batched(ops, [torch.from_numpy(p.b) for p in probs], [p.tau for p in probs],
                                M.SolverParams(cluster_size=4, **EVERY))
    for p, x, info in zip(probs, xs, infos):
        check(info, x.cpu().numpy(), oracle_every(O.Operator.from_dct_rows(p.n, p.rows), p))


def test_lockstep_dct_corrector_every_iteration():
    """The lockstep multi-pass solver (reached at n = 2048 by lowering its threshold), two
    problems of one n in lockstep."""
    M = mf()
    L = M.lib()
    assert L.mfipm_set_large_dct_threshold(ctypes.c_int64(2048)) == 0
    try:
        probs = [W.dct_problem(2048, 512, 20, seed=314, j=j) for j in range(2)]
        ops = [M.PartialDCT(p.n, torch.from_numpy(p.rows)) for p in probs]
        xs, infos = M.solve_batched(ops, [torch.from_numpy(p.b) for p in probs], [p.tau for p in probs],
                                    M.SolverParams(**EVERY))
    finally:
        assert L.mfipm_set_large_dct_threshold(ctypes.c_int64(1 << 17)) == 0
    for p, x, info in zip(probs, xs, infos):
        check(info, x.cpu().numpy(), oracle_every(O.Operator.from_dct_rows(p.n, p.rows), p))


def test_shared_bf16_corrector_every_iteration():
    """The shared-A bf16 solver (tcgen05 GEMMs in the PCG, tensor-core residual)."""
    M = mf()
    probs = W.bf16_dense_problems(256, 1024, 10, 3, seed=315)
    bits = torch.from_numpy(probs[0].a_bf16.view(np.int16)).view(torch.bfloat16).cuda()
    op = M.DenseBF16(bits, probs[0].a_scale)
    xs, infos = M.solve_batched([op] * len(probs), [torch.from_numpy(p.b) for p in probs], [p.tau for p in probs],
                                M.SolverParams(**EVERY))
    ref = O.Operator.from_dense(probs[0].A)
    for p, x, info in zip(probs, xs, infos):
        check(info, x.cpu().numpy(), oracle_every(ref, p))


def test_default_alpha_tilde_matches_oracle_counts():
    """With the paper's alpha_tilde = 0.1 the GPU takes a corrector exactly when its own step
    lengths fall to 0.1; on this problem the exact-direction oracle and the GPU both take none
    or few, and reach the same minimiser."""
    M = mf()
    p = W.dct_problem(4096, 1024, 40, seed=316)
    res = O.ipm(O.Operator.from_dct_rows(p.n, p.rows), p.b, p.tau)
    x, info = M.solve(M.PartialDCT(p.n, torch.from_numpy(p.rows)), torch.from_numpy(p.b), p.tau,
                      M.SolverParams(tol=1e-12))
    assert info["status"] == 0 and relx(x.cpu().numpy(), res.x) <= RELX_TOL
    assert 0 <= info["correctors"] <= info["ipm_iters"]
