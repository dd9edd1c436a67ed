"""mfipm_autotune: the tuned configuration is one of the candidates, the solves it leaves
behind match the oracle, and later solves of the same batch shape use it (bitwise equal to
the tuner's final solve); after mfipm_clear_tuning the default configuration returns."""
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


def _oracle_x(p):
    op = O.Operator.from_dense(p.A) if p.kind == "dense" else O.Operator.from_dct_rows(p.n, p.rows)
    return O.ipm(op, p.b, p.tau).x


def test_autotune_dct_batch():
    M = mf()
    M.clear_tuning()
    sizes = [512, 8192, 1024, 2048, 4096, 8192, 512, 2048]
    probs = [W.dct_problem(n, n // 4, max(1, n // 60), seed=99, j=j) for j, n in enumerate(sizes)]
    ops = [M.PartialDCT(p.n, torch.from_numpy(p.rows)) for p in probs]
    bs = [torch.from_numpy(p.b) for p in probs]
    taus = [p.tau for p in probs]
    prm = M.SolverParams(tol=1e-12)
    xs, infos, tun = M.autotune(ops, bs, taus, prm)
    assert tun["path"] == 1 and tun["candidates"] >= 2
    assert tun["cluster_size"] in (1, 2, 4, 8) and tun["cta_max_n"] in (2048, 4096, 8192)
    assert 0 < tun["best_ms"] <= tun["default_ms"]
    for p, x, i in zip(probs, xs, infos):
        xo = _oracle_x(p)
        assert i["status"] == 0
        assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-6 * np.linalg.norm(xo)
    # the table entry now drives the solve: same configuration, same arithmetic
    xs2, _ = M.solve_batched(ops, bs, taus, prm)
    assert all(torch.equal(a, b) for a, b in zip(xs, xs2))
    M.clear_tuning()
    xs3, infos3 = M.solve_batched(ops, bs, taus, prm)
    for p, x in zip(probs, xs3):
        xo = _oracle_x(p)
        assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-6 * np.linalg.norm(xo)


def test_autotune_bf16_gemm_splits():
    M = mf()
    M.clear_tuning()
    probs = W.bf16_dense_problems(256, 1024, 8, 4, seed=100)
    bits = torch.from_numpy(probs[0].a_bf16.view(np.int16)).view(torch.bfloat16)
    op = M.DenseBF16(bits, probs[0].a_scale)
    ops = [op] * len(probs)
    xs, infos, tun = M.autotune(ops, [torch.from_numpy(p.b) for p in probs], [p.tau for p in probs],
                                M.SolverParams())
    assert tun["path"] == 2 and 1 <= tun["splits1"] <= 8 and 1 <= tun["splits2"] <= 8
    assert tun["candidates"] == 32 and tun["best_ms"] <= tun["default_ms"] + 1e-9
    assert tun["stages1"] in (3, 4) and tun["stages2"] in (3, 4)
    ref = O.Operator.from_dense(probs[0].A)
    for p, x, i in zip(probs, xs, infos):
        assert i["status"] == 0
        assert O.kkt_rel(ref, p.b, p.tau, x.cpu().numpy()) <= 1e-6
    M.clear_tuning()
