"""Basis pursuit through a tiny tau (Sec. 5.4 and Table regparams): noiseless partial-DCT
measurements solved with every tau of the table, 1e-10 .. 1e-2, and the paper's noiseless
settings (tol between 1e-10 and 1e-14, tolpcg between 1e-2 and 1e-6).  A tolpcg of 1e-6 is
beyond a float32 PCG, so these run the float64 PCG of the dense path on the explicit rows of
the DCT.  Against the float64 direct-solve oracle at tol 1e-14: x to 1e-6 relative, and for
tau <= 1e-7 the sparse signal itself to r.e. 1e-5 (the basis-pursuit limit)."""
import numpy as np
import pytest

import workloads as W
from oracle import mfipm_oracle as O
from tests._lib import built_lib

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (tau, tol, tolpcg)
SETTINGS = [(1e-10, 1e-14, 1e-6), (1e-8, 1e-14, 1e-4), (1e-7, 1e-12, 1e-2), (1e-5, 1e-12, 1e-2),
            (1e-4, 1e-10, 1e-2), (1e-3, 1e-10, 1e-2), (1e-2, 1e-10, 1e-2)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    built_lib()


@pytest.mark.parametrize("tau,tol,tol_pcg", SETTINGS)
def test_tiny_tau_matches_direct_oracle(tau, tol, tol_pcg):
    import paper_1208_5435_gb300 as M
    p = W.dct_problem(1024, 256, 10, 1008, 0, sigma=0.0, values="pm1")
    A = O.dct_matrix_rows(p.n, p.rows)
    ref = O.ipm(O.Operator.from_dense(A), p.b, tau, O.OracleParams(tol=1e-14))
    x, info = M.solve(M.Dense(torch.from_numpy(A)), torch.from_numpy(p.b), tau,
                      M.SolverParams(tol=tol, tol_pcg=tol_pcg))
    xg = x.cpu().numpy()
    assert info["status"] == 0, info
    assert np.linalg.norm(xg - ref.x) <= 1e-6 * np.linalg.norm(ref.x)
    if tau <= 1e-7:
        assert np.linalg.norm(xg - p.x_hat) <= 1e-5 * np.linalg.norm(p.x_hat)


@pytest.mark.parametrize("tau,tol,tol_pcg", SETTINGS)
def test_tiny_tau_matrix_free_float64_pcg(tau, tol, tol_pcg):
    """The same basis-pursuit settings on the matrix-free partial-DCT operator with the float64
    PCG (precision MFIPM_PREC_FP64: FFT chain, PCG vectors and preconditioner in float64), which
    reaches the tolpcg 1e-6 of the noiseless settings without explicit rows."""
    import paper_1208_5435_gb300 as M
    p = W.dct_problem(1024, 256, 10, 1008, 0, sigma=0.0, values="pm1")
    A = O.dct_matrix_rows(p.n, p.rows)
    ref = O.ipm(O.Operator.from_dense(A), p.b, tau, O.OracleParams(tol=1e-14))
    x, info = M.solve(M.PartialDCT(p.n, torch.from_numpy(p.rows)), torch.from_numpy(p.b), tau,
                      M.SolverParams(tol=tol, tol_pcg=tol_pcg, precision=0))
    xg = x.cpu().numpy()
    assert info["status"] == 0, info
    assert np.linalg.norm(xg - ref.x) <= 1e-6 * np.linalg.norm(ref.x)
    if tau <= 1e-7:
        assert np.linalg.norm(xg - p.x_hat) <= 1e-5 * np.linalg.norm(p.x_hat)
