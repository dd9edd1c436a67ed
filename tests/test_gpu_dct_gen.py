"""Partial DCT of lengths that are not powers of two (the mixed-radix chain, one CTA per
problem): n = 1000 of the phase-transition experiment (Sec. 5.8; n/2 = 2^2 5^3), an odd half
length (n = 250, n/2 = 5^3), radix 3 (n = 96, 6000), and the largest length the chain takes
(n = 16200, n/2 = 2^2 3^4 5^2), against the float64 oracle, whose partial DCT is the
definition of the orthonormal DCT-II rows at any n."""
import numpy as np
import pytest

import workloads as W
from oracle import mfipm_oracle as O
from tests._lib import built_lib

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RELX_TOL = 1e-6


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


def oracle_x(p, **kw):
    res = O.ipm(O.Operator.from_dct_rows(p.n, p.rows), p.b, p.tau, O.OracleParams(tol=1e-12, **kw))
    assert res.converged
    return res


@pytest.mark.parametrize("n", [1000, 250, 96, 6000, 2000])
def test_matches_oracle(n):
    M = mf()
    p = W.dct_problem(n, n // 4, max(1, n // 100), seed=331, j=n)
    x, info = M.solve(M.PartialDCT(p.n, torch.from_numpy(p.rows)), torch.from_numpy(p.b), p.tau,
                      M.SolverParams(tol=1e-12))
    assert info["status"] == 0, info
    assert relx(x.cpu().numpy(), oracle_x(p).x) <= RELX_TOL, (n, info)


def test_largest_length_certificates():
    """n = 16200 (24 bytes of shared memory per complex point: 194 KB): the prox residual and
    the dual-gap certificate of x on the CPU (the oracle's implicit DCT at any length)."""
    M = mf()
    p = W.dct_problem(16200, 4050, 160, seed=332)
    x, info = M.solve(M.PartialDCT(p.n, torch.from_numpy(p.rows)), torch.from_numpy(p.b), p.tau, M.SolverParams())
    assert info["status"] == 0, info
    op = O.Operator.from_dct_rows(p.n, p.rows, explicit=False)
    xg = x.cpu().numpy()
    k = O.kkt_rel(op, p.b, p.tau, xg)
    assert k <= 1e-6 and abs(k - info["kkt_rel"]) <= 1e-8 + 0.05 * k, (k, info)
    P, D = O.dual_gap_certificate(op, p.b, p.tau, xg)
    assert -1e-12 <= (P - D) / max(1.0, abs(P)) <= 1e-5


def test_batch_mixes_lengths():
    """One batched call with general and power-of-two lengths: every problem runs on the
    mixed-radix chain (a power of two is radices 4 and 2)."""
    M = mf()
    ns = [1000, 1024, 250, 4096, 6000, 96, 512, 3000]
    probs = [W.dct_problem(n, n // 4, max(1, n // 60), seed=333, j=j) for j, n in enumerate(ns)]
    ops = [M.PartialDCT(p.n, torch.from_numpy(p.rows)) for p in probs]
    xs, infos = M.solve_batched(ops, [torch.from_numpy(p.b) for p in probs], [p.tau for p in probs],
                                M.SolverParams(tol=1e-12))
    for p, x, info in zip(probs, xs, infos):
        assert info["status"] == 0, (p.n, info)
        assert relx(x.cpu().numpy(), oracle_x(p).x) <= RELX_TOL, (p.n, info)


@pytest.mark.parametrize("outer,precision", [(1, 0), (1, 1)])
def test_float64_variants(outer, precision):
    """The float64 outer loop with the float32 PCG, and the float64 PCG (basis pursuit through
    a tiny tau at tolpcg 1e-6, Sec. 5.4)."""
    M = mf()
    if precision == 1:
        p = W.dct_problem(1000, 300, 12, seed=334, sigma=0.0, tau_frac=1e-8)
        prm = M.SolverParams(tol=1e-12, tol_pcg=1e-6, precision=1, outer=1)
    else:
        p = W.dct_problem(1000, 250, 10, seed=335)
        prm = M.SolverParams(tol=1e-12, outer=1)
    x, info = M.solve(M.PartialDCT(p.n, torch.from_numpy(p.rows)), torch.from_numpy(p.b), p.tau, prm)
    assert info["status"] == 0, info
    assert relx(x.cpu().numpy(), oracle_x(p).x) <= RELX_TOL, info


def test_corrector_every_iteration():
    """alpha_tilde = 1: the corrector of the Algorithm (Sec. 5.1) at every iteration on the
    mixed-radix chain, against the oracle with the same alpha_tilde."""
    M = mf()
    p = W.dct_problem(1000, 250, 10, seed=336)
    res = O.ipm(O.Operator.from_dct_rows(p.n, p.rows), p.b, p.tau, O.OracleParams(alpha_tilde=1.0))
    assert res.converged and res.correctors > 0
    x, info = M.solve(M.PartialDCT(p.n, torch.from_numpy(p.rows)), torch.from_numpy(p.b), p.tau,
                      M.SolverParams(alpha_tilde=1.0, tol=1e-12))
    assert info["status"] == 0 and info["correctors"] == info["ipm_iters"] > 0, info
    assert relx(x.cpu().numpy(), res.x) <= RELX_TOL


def test_zs_out_is_in_natural_order():
    """The final iterate [u; v; s_u; s_v] comes back in natural index order: x = u - v, and the
    dual residual f_z = s - (c + F F^T z) of Eq. fzfs rebuilt from it on the CPU is the one the
    solver reports (info.dual_res = ||f_z|| / (1 + ||c||))."""
    M = mf()
    p = W.dct_problem(1000, 250, 10, seed=337)
    x, info, zs = M.solve(M.PartialDCT(p.n, torch.from_numpy(p.rows)), torch.from_numpy(p.b), p.tau,
                          M.SolverParams(), return_zs=True)
    zs = zs.cpu().numpy()
    n = p.n
    u, v, su, sv = zs[:n], zs[n:2 * n], zs[2 * n:3 * n], zs[3 * n:]
    # x = u - v in the iterate's own arithmetic, then rounded: equal to u - v in float64 up to
    # the rounding of the two terms
    assert np.all(np.abs(u - v - x.cpu().numpy()) <= 1e-13 * (np.abs(u) + np.abs(v)))
    assert min(u.min(), v.min(), su.min(), sv.min()) > 0
    op = O.Operator.from_dct_rows(n, p.rows)
    g = op.rmv(op.mv(u - v) - p.b)  # A^T (A x - b)
    fz = np.concatenate([su - (p.tau + g), sv - (p.tau - g)])
    atb = op.rmv(p.b)
    cn = np.sqrt(2 * n * p.tau ** 2 + 2 * atb @ atb)
    assert abs(np.linalg.norm(fz) / (1 + cn) - info["dual_res"]) <= 1e-2 * info["dual_res"] + 1e-12, info


@pytest.mark.parametrize("n", [8, 12, 20, 30, 90])
def test_smallest_lengths(n):
    """The shortest transforms (n/2 = 4, 6, 10, 15, 45: a lone radix-4 stage, radix 2 after 3,
    odd halves) against the oracle, every row sampled but one."""
    M = mf()
    p = W.dct_problem(n, n - 1, 2, seed=338, j=n)
    x, info = M.solve(M.PartialDCT(p.n, torch.from_numpy(p.rows)), torch.from_numpy(p.b), p.tau,
                      M.SolverParams(tol=1e-12))
    assert info["status"] == 0, (n, info)
    assert relx(x.cpu().numpy(), oracle_x(p).x) <= RELX_TOL, (n, info)


def test_full_basis_is_the_soft_threshold():
    """m = n = 1000 (A orthonormal and square): the minimiser is S_tau(A^T b) in closed form."""
    M = mf()
    p = W.dct_problem(1000, 1000, 20, seed=339)
    x, info = M.solve(M.PartialDCT(p.n, torch.from_numpy(p.rows)), torch.from_numpy(p.b), p.tau,
                      M.SolverParams(tol=1e-12))
    atb = O.Operator.from_dct_rows(p.n, p.rows).rmv(p.b)
    assert info["status"] == 0 and relx(x.cpu().numpy(), O.soft_threshold(atb, p.tau)) <= RELX_TOL, info


def test_no_measurements_gives_zero():
    """m = 0: the objective is tau ||x||_1, minimised by x = 0."""
    M = mf()
    op = M.PartialDCT(1000, torch.zeros(0, dtype=torch.int64))
    x, info = M.solve(op, torch.zeros(0, dtype=torch.float64), 0.1, M.SolverParams(tol=1e-12))
    assert info["status"] == 0 and float(x.abs().max()) <= 1e-8 and info["kkt_rel"] <= 1e-8
