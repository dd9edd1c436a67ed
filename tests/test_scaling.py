"""The PCG-against-direct workload (Sec. 5.7) on the CPU: its generator, and the paper's
observation on it at small sizes, checked with the oracle's two Newton solvers: PCG
directions need about as many IPM iterations as exact (direct) ones."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import mfipm_oracle as O


def test_sizes_and_problems():
    probs = W.make_workload("pcg_vs_direct")
    assert [p.n for p in probs] == [1 << e for e in range(5, 13)]
    for p in probs:
        assert p.m == p.n // 4 and p.A.shape == (p.m, p.n)
        assert np.count_nonzero(p.x_hat) == math.ceil(p.m / 20)
        assert p.tau == 1e-3
        assert np.array_equal(p.A @ p.x_hat, p.b)  # noiseless
        assert abs(p.A.var() * p.m - 1.0) < 0.2   # N(0, 1/m) entries


def test_pcg_iterations_match_direct_at_small_sizes():
    for p in W.make_workload("pcg_vs_direct", count=4):
        op = O.Operator.from_dense(p.A)
        direct = O.ipm(op, p.b, p.tau, O.OracleParams(tol=1e-10, solver="cholesky"))
        pcg = O.ipm(op, p.b, p.tau, O.OracleParams(tol=1e-10, solver="pcg"))
        assert direct.converged and pcg.converged
        assert abs(direct.iters - pcg.iters) <= 2, (p.n, direct.iters, pcg.iters)
        assert np.linalg.norm(direct.x - pcg.x) <= 1e-5 * np.linalg.norm(direct.x)


def test_bp_limit_pcg_with_noiseless_settings():
    """Tiny tau (Table regparams) with the paper's noiseless settings: the PCG variant of the
    oracle agrees with its direct variant, and the solution approaches the sparse signal."""
    p = W.dct_problem(1024, 256, 10, 1008, 0, sigma=0.0, values="pm1")
    op = O.Operator.from_dct_rows(p.n, p.rows)
    direct = O.ipm(op, p.b, 1e-10, O.OracleParams(tol=1e-14))
    pcg = O.ipm(op, p.b, 1e-10, O.OracleParams(tol=1e-14, solver="pcg", tol_pcg=1e-6))
    assert direct.converged and pcg.converged
    assert np.linalg.norm(pcg.x - direct.x) <= 1e-6 * np.linalg.norm(direct.x)
    assert np.linalg.norm(direct.x - p.x_hat) <= 1e-5 * np.linalg.norm(p.x_hat)


def test_direct_comparison_arm_matches_the_oracle():
    """bench.py's same-GPU direct arm of the PCG-against-direct leg (Sec. 5.7), run here on CPU
    tensors: the same minimiser and the same number of Newton directions as the oracle's
    direct IPM, which it restates independently (Woodbury Cholesky, readings R1-R8)."""
    import bench
    torch = pytest.importorskip("torch")
    p = W.scaling_problems(1007, (6, 8))[1]
    A, b = torch.from_numpy(p.A), torch.from_numpy(p.b)
    x, its = bench.direct_ipm_gpu(A, b, p.tau, 1e-10)
    r = O.ipm(O.Operator.from_dense(p.A), p.b, p.tau, O.OracleParams(tol=1e-10, solver="woodbury"))
    assert np.linalg.norm(x.numpy() - r.x) <= 1e-8 * np.linalg.norm(r.x)
    assert its == r.iters - 1
