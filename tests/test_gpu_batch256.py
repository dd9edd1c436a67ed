"""Parity on the headline workload: the 256-problem uneven partial-DCT batch (n drawn from
2^12..2^16, m = n/4, k in [n/100, n/20]) solved in ONE mfipm_solve_batched call with the
benchmark's parameters, i.e. the launch the benchmark times (both phases of the persistent
kernel: clusters for n > 16384, single CTAs below).

* relative l2 error of x <= 1e-6 against the float64 oracle's direct solve (Woodbury form)
  on two problems of every class the oracle reaches (n = 4096 and n = 8192);
* for all 256 problems, the prox (KKT) residual <= 1e-6 and the l1 dual-gap certificate,
  both computed on the CPU by the oracle's functions with the library DCT, and the
  solver's own info.kkt_rel agreeing with the CPU value.
The oracle cannot reach n = 16384..65536 in a test's time (reading R13): there parity is
the certificates."""
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


def test_dct_batch_256_against_oracle_and_certificates():
    import paper_1208_5435_gb300 as M
    probs = W.make_workload("dct_batch_256")
    assert len(probs) == 256
    ops = [M.PartialDCT(p.n, torch.from_numpy(p.rows)) for p in probs]
    params = M.SolverParams()          # the benchmark's parameters (tol 1e-10, tol_pcg 1e-2)
    xs, infos = M.solve_batched(ops, [torch.from_numpy(p.b) for p in probs], [p.tau for p in probs], params)
    xs = [x.cpu().numpy() for x in xs]
    assert sum(i["status"] == 0 for i in infos) == 256, [i for i in infos if i["status"] != 0][:3]
    # both phases ran: some problems need a cluster (n > 16384), some a single CTA
    ns = {p.n for p in probs}
    assert {4096, 8192}.issubset(ns) and {32768, 65536}.issubset(ns)

    # (1) the oracle's direct solve on two problems of each class it reaches
    picked = {4096: [], 8192: []}
    for j, p in enumerate(probs):
        if p.n in picked and len(picked[p.n]) < 2:
            picked[p.n].append(j)
    for n, idx in picked.items():
        assert len(idx) == 2
        for j in idx:
            p = probs[j]
            res = O.ipm(O.Operator.from_dct_rows(p.n, p.rows), p.b, p.tau, O.OracleParams(solver="woodbury"))
            assert res.converged
            rel = np.linalg.norm(xs[j] - res.x) / np.linalg.norm(res.x)
            assert rel <= 1e-6, (j, n, rel, infos[j])

    # (2) certificates for every problem, on the CPU
    worst_kkt, worst_gap = 0.0, 0.0
    for j, (p, x, info) in enumerate(zip(probs, xs, infos)):
        op = O.Operator.from_dct_rows(p.n, p.rows, explicit=False)
        k = O.kkt_rel(op, p.b, p.tau, x)
        assert k <= 1e-6, (j, p.n, k)
        assert abs(k - info["kkt_rel"]) <= 1e-8 + 0.05 * k, (j, k, info["kkt_rel"])
        P, D = O.dual_gap_certificate(op, p.b, p.tau, x)
        gap = (P - D) / max(1.0, abs(P))
        assert -1e-12 <= gap <= 1e-5, (j, p.n, gap)
        worst_kkt, worst_gap = max(worst_kkt, k), max(worst_gap, gap)
    print(f"dct_batch_256: max kkt_rel {worst_kkt:.2e}, max dual-gap bound {worst_gap:.2e}, "
          f"correctors {sum(i['correctors'] for i in infos)}")
