"""Parity of the CUDA solver (through the C ABI) with the float64 CPU oracle.

Bar: relative l2 error of x against the oracle's minimiser <= 1e-6 for the FP64 and the
FP32-PCG paths; at full benchmark sizes (beyond the oracle's direct solve) the l1
certificates computed independently on the CPU."""
import numpy as np
import pytest

import workloads as W
from oracle import mfipm_oracle as O
from tests._lib import built_lib

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RELX_TOL = 1e-6
_cache = {}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    built_lib()


def mf():
    import paper_1208_5435_gb300 as M
    return M


def oracle_solution(p):
    key = (p.kind, p.n, p.m, p.seed)
    if key not in _cache:
        op = O.Operator.from_dense(p.A) if p.kind == "dense" else O.Operator.from_dct_rows(p.n, p.rows)
        res = O.ipm(op, p.b, p.tau)
        assert res.converged
        _cache[key] = res.x
    return _cache[key]


def gpu_solve(p, **kw):
    """Solve through the C ABI; parity runs use the oracle's gap tolerance 1e-12."""
    M = mf()
    kw.setdefault("tol", 1e-12)
    op = M.Dense(torch.from_numpy(p.A)) if p.kind == "dense" else M.PartialDCT(p.n, torch.from_numpy(p.rows))
    x, info = M.solve(op, torch.from_numpy(p.b), p.tau, M.SolverParams(**kw))
    return x.cpu().numpy(), info


def relx(x, xo):
    return np.linalg.norm(x - xo) / max(np.linalg.norm(xo), 1e-300)


@pytest.mark.parametrize("n,G", [(64, 1), (64, 4), (256, 1), (256, 2), (256, 8), (1024, 1), (1024, 4),
                                 (1024, 16), (4096, 1), (4096, 2), (4096, 8), (4096, 16)])
def test_dct_matches_oracle(n, G):
    p = W.dct_problem(n, n // 4, max(1, n // 100), seed=77, j=n)
    xo = oracle_solution(p)
    x, info = gpu_solve(p, cluster_size=G)
    assert info["status"] == 0, info
    assert relx(x, xo) <= RELX_TOL, (relx(x, xo), info)
    assert info["kkt_rel"] < 1e-7
    assert 5 <= info["ipm_iters"] <= 40


def test_dct_ragged_rows_and_m_not_power_of_two():
    p = W.dct_problem(2048, 300, 12, seed=78)
    xo = oracle_solution(p)
    x, info = gpu_solve(p)
    assert info["status"] == 0 and relx(x, xo) <= RELX_TOL


@pytest.mark.parametrize("pcg", ["fp64", "fp32"])
def test_dense_cfg1_matches_oracle(pcg):
    p = W.make_workload("dense_fp64_256x1024")[0]
    xo = oracle_solution(p)
    x, info = gpu_solve(p, precision=0 if pcg == "fp64" else 1)
    assert info["status"] == 0, info
    assert relx(x, xo) <= RELX_TOL, (relx(x, xo), info)


@pytest.mark.parametrize("G", [1, 4, 16])
def test_dense_ragged_columns(G):
    p = W.dense_problem(250, 1000, 10, seed=79)
    xo = oracle_solution(p)
    x, info = gpu_solve(p, cluster_size=G)
    assert info["status"] == 0 and relx(x, xo) <= RELX_TOL, (relx(x, xo), info)


def test_batched_uneven_matches_oracle_and_plain():
    M = mf()
    ns = [256, 4096, 512, 2048, 1024, 4096, 256, 1024, 2048, 512, 8192, 256]
    probs = [W.dct_problem(n, n // 4, max(1, n // 50), seed=80, j=j) for j, n in enumerate(ns)]
    ops = [M.PartialDCT(p.n, torch.from_numpy(p.rows)) for p in probs]
    xs, infos = M.solve_batched(ops, [torch.from_numpy(p.b) for p in probs], [p.tau for p in probs],
                                M.SolverParams(tol=1e-12))
    for p, x, info in zip(probs, xs, infos):
        assert info["status"] == 0, info
        assert relx(x.cpu().numpy(), oracle_solution(p)) <= RELX_TOL
    # the batched launch with one cluster size reproduces the single-problem solve bit for bit
    G = 1
    xs1, _ = M.solve_batched(ops[:3], [torch.from_numpy(p.b) for p in probs[:3]], [p.tau for p in probs[:3]],
                             M.SolverParams(cluster_size=G))
    for p, op, xb in zip(probs[:3], ops[:3], xs1):
        x1, _ = M.solve(op, torch.from_numpy(p.b), p.tau, M.SolverParams(cluster_size=G))
        assert torch.equal(x1, xb)


def test_closed_form_full_dct():
    """m = n: A orthonormal, x* = S_tau(A^T b)."""
    n = 1024
    rng = np.random.default_rng(5)
    rows = np.arange(n, dtype=np.int64)
    b = rng.standard_normal(n)
    atb = O.dct_rows_apply_t(b, rows, n)
    tau = 0.3 * np.abs(atb).max()
    p = W.Problem("dct", n, n, b, tau, np.zeros(n), rows=rows)
    x, info = gpu_solve(p)
    assert info["status"] == 0
    assert np.abs(x - O.soft_threshold(atb, tau)).max() < 1e-7


def test_zero_solution_for_large_tau():
    p = W.dct_problem(1024, 256, 10, seed=81)
    atb = O.dct_rows_apply_t(p.b, p.rows, p.n)
    p.tau = 1.01 * np.abs(atb).max()
    x, info = gpu_solve(p)
    assert info["status"] == 0 and np.abs(x).max() < 1e-8


def test_invalid_rows_rejected():
    M = mf()
    rows = torch.tensor([3, 3, 7, 9], dtype=torch.int64)
    op = M.PartialDCT(64, rows)
    with pytest.raises(M.MfipmError) as e:
        M.solve(op, torch.ones(4, dtype=torch.float64), 0.1)
    assert e.value.code == 1
    op = M.PartialDCT(64, torch.tensor([1, 5, 64, 70], dtype=torch.int64))
    with pytest.raises(M.MfipmError):
        M.solve(op, torch.ones(4, dtype=torch.float64), 0.1)


def test_full_size_dct_65536_certificates():
    """Benchmark size: the oracle's direct solve is out of reach, so check the l1
    optimality certificates on the CPU with the library DCT."""
    p = W.make_workload("dct_65536")[0]
    x, info = gpu_solve(p, tol=1e-10)
    assert info["status"] == 0, info
    op = O.Operator.from_dct_rows(p.n, p.rows, explicit=False)
    k = O.kkt_rel(op, p.b, p.tau, x)
    assert k <= 1e-6 and abs(k - info["kkt_rel"]) <= 1e-7 + 0.1 * k
    P, D = O.dual_gap_certificate(op, p.b, p.tau, x)
    assert 0 <= P - D <= 1e-6 * (1 + abs(P))
    v_on, v_off = O.optimality_violation(op, p.b, p.tau, x, support_tol=1e-5)
    assert v_on < 1e-5 * p.tau * 10 and v_off < 1e-5 * p.tau * 10


@pytest.mark.parametrize("n,G", [(1024, 4), (4096, 8), (4096, 1)])
def test_dct_float64_outer_mode_matches_oracle_and_df_mode(n, G):
    """The native float64 outer loop and the double-float one reach the same minimiser."""
    p = W.dct_problem(n, n // 4, max(1, n // 100), seed=77, j=n)
    xo = oracle_solution(p)
    x64, info64 = gpu_solve(p, cluster_size=G, outer=1)
    xdf, infodf = gpu_solve(p, cluster_size=G, outer=0)
    assert info64["status"] == 0 and infodf["status"] == 0
    assert relx(x64, xo) <= RELX_TOL and relx(xdf, xo) <= RELX_TOL
    assert relx(xdf, x64) <= 1e-7


def test_no_measurements_gives_zero():
    """m = 0 (no sampled rows): the objective is tau ||x||_1, minimised by x = 0."""
    M = mf()
    op = M.PartialDCT(1024, torch.zeros(0, dtype=torch.int64))
    x, info = M.solve(op, torch.zeros(0, dtype=torch.float64), 0.1, M.SolverParams(tol=1e-12))
    assert info["status"] == 0 and float(x.abs().max()) <= 1e-8 and info["kkt_rel"] <= 1e-8


@pytest.mark.parametrize("n,G", [(1024, 1), (1024, 4), (4096, 2), (4096, 16)])
def test_dct_float64_pcg_matches_oracle(n, G):
    """The partial-DCT operator with the float64 PCG (precision MFIPM_PREC_FP64)."""
    p = W.dct_problem(n, n // 4, max(1, n // 100), seed=77, j=n)
    xo = oracle_solution(p)
    x, info = gpu_solve(p, cluster_size=G, precision=0)
    assert info["status"] == 0, info
    assert relx(x, xo) <= RELX_TOL, (relx(x, xo), info)
    # the float64 PCG matches the float32 one's IPM iteration count to within a few iterations
    x32, info32 = gpu_solve(p, cluster_size=G)
    assert abs(info["ipm_iters"] - info32["ipm_iters"]) <= 4
