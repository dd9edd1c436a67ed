"""Multiple centrality correctors (reading R19: the variant Sec. 5.1 names as the origin of
its single-corrector method) on the persistent kernel, against the float64 oracle running
the same variant with exact Newton directions: the same minimiser, correctors taken, and an
iteration count in the oracle's band.  The lockstep solvers reject the variant."""
import ctypes

import numpy as np
import pytest

import workloads as W
from oracle import mfipm_oracle as O
from tests._lib import built_lib

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RELX_TOL = 1e-6
K = 3


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


def oracle_mcc(op, p):
    res = O.ipm(op, p.b, p.tau, O.OracleParams(mcc=K))
    assert res.converged
    return res


@pytest.mark.parametrize("n,G", [(1024, 1), (1024, 4), (4096, 1), (4096, 8)])
def test_dct_mcc_matches_oracle(n, G):
    M = mf()
    p = W.dct_problem(n, n // 4, max(1, n // 100), seed=321, j=n)
    res = oracle_mcc(O.Operator.from_dct_rows(p.n, p.rows), p)
    x, info = M.solve(M.PartialDCT(p.n, torch.from_numpy(p.rows)), torch.from_numpy(p.b), p.tau,
                      M.SolverParams(tol=1e-12, cluster_size=G, centrality_correctors=K))
    assert info["status"] == 0, info
    assert relx(x.cpu().numpy(), res.x) <= RELX_TOL, (relx(x.cpu().numpy(), res.x), info)
    assert info["correctors"] > 0
    assert abs(info["ipm_iters"] - (res.iters - 1)) <= 8, (info, res.iters)


@pytest.mark.parametrize("precision", [0, 1])
def test_dense_mcc_matches_oracle(precision):
    M = mf()
    p = W.dense_problem(128, 512, 10, seed=322)
    res = oracle_mcc(O.Operator.from_dense(p.A), p)
    x, info = M.solve(M.Dense(torch.from_numpy(p.A)), torch.from_numpy(p.b), p.tau,
                      M.SolverParams(tol=1e-12, precision=precision, centrality_correctors=K))
    assert info["status"] == 0, info
    assert relx(x.cpu().numpy(), res.x) <= RELX_TOL, (relx(x.cpu().numpy(), res.x), info)
    assert info["correctors"] > 0


def test_batch_mcc_both_phases():
    M = mf()
    ns = [4096, 512, 1024, 2048, 4096, 256]
    probs = [W.dct_problem(n, n // 4, max(1, n // 60), seed=323, j=j) for j, n in enumerate(ns)]
    ops = [M.PartialDCT(p.n, torch.from_numpy(p.rows)) for p in probs]
    xs, infos = M.solve_batched(ops, [torch.from_numpy(p.b) for p in probs], [p.tau for p in probs],
                                M.SolverParams(tol=1e-12, cluster_size=4, centrality_correctors=K))
    for p, x, info in zip(probs, xs, infos):
        res = oracle_mcc(O.Operator.from_dct_rows(p.n, p.rows), p)
        assert info["status"] == 0 and relx(x.cpu().numpy(), res.x) <= RELX_TOL, info
    assert sum(i["correctors"] for i in infos) > 0


def test_lockstep_paths_reject_mcc():
    M = mf()
    L = M.lib()
    assert L.mfipm_set_large_dct_threshold(ctypes.c_int64(2048)) == 0
    try:
        p = W.dct_problem(2048, 512, 20, seed=324)
        with pytest.raises(M.MfipmError) as e:
            M.solve(M.PartialDCT(p.n, torch.from_numpy(p.rows)), torch.from_numpy(p.b), p.tau,
                    M.SolverParams(centrality_correctors=2))
        assert e.value.code == 6
    finally:
        assert L.mfipm_set_large_dct_threshold(ctypes.c_int64(1 << 17)) == 0
    pb = W.bf16_dense_problems(128, 512, 6, 1, seed=325)[0]
    op = M.DenseBF16(torch.from_numpy(pb.a_bf16.view(np.int16)).view(torch.bfloat16), pb.a_scale)
    with pytest.raises(M.MfipmError) as e:
        M.solve(op, torch.from_numpy(pb.b), pb.tau, M.SolverParams(centrality_correctors=2))
    assert e.value.code == 6
