"""The PCG-against-direct workload (Sec. 5.7) on the GPU: every size n = 2^5..2^12 through the
dense float64 persistent kernel against the float64 oracle with direct Newton solves: x to
relative l2 1e-6 at tol 1e-12, and at the default tol 1e-10 about as many IPM iterations as
the exact-direction oracle (the paper's observation for PCG directions)."""
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


def test_every_size_matches_the_direct_oracle():
    import paper_1208_5435_gb300 as M
    for p in W.make_workload("pcg_vs_direct"):
        op = M.Dense(torch.from_numpy(p.A))
        ref_op = O.Operator.from_dense(p.A)
        x, info = M.solve(op, torch.from_numpy(p.b), p.tau, M.SolverParams(tol=1e-12))
        ref = O.ipm(ref_op, p.b, p.tau, O.OracleParams(tol=1e-12))
        xg = x.cpu().numpy()
        assert info["status"] == 0, (p.n, info)
        assert np.linalg.norm(xg - ref.x) <= 1e-6 * np.linalg.norm(ref.x), p.n
        _, info10 = M.solve(op, torch.from_numpy(p.b), p.tau, M.SolverParams())
        direct10 = O.ipm(ref_op, p.b, p.tau, O.OracleParams(tol=1e-10))
        # Newton directions taken: ipm_iters on the GPU; the oracle counts its gap checks
        assert abs(info10["ipm_iters"] - (direct10.iters - 1)) <= 2, (p.n, info10["ipm_iters"], direct10.iters)
