"""The lockstep multi-pass partial-DCT solver (problems above the cluster solver's n = 65536):
parity with the float64 oracle at oracle sizes, reached by lowering the multi-pass
threshold; the full-size n = 2^20 problems of the adjoint workload through the l1
certificates and a finite-difference check of the derivative."""
import ctypes

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


@pytest.fixture
def threshold():
    from paper_1208_5435_gb300 import _capi as C
    L = C.lib()

    def set_(n):
        assert L.mfipm_set_large_dct_threshold(ctypes.c_int64(n)) == 0

    yield set_
    set_(1 << 17)


def _op(M, p):
    return M.PartialDCT(p.n, torch.from_numpy(p.rows))


def _oracle(p):
    res = O.ipm(O.Operator.from_dct_rows(p.n, p.rows), p.b, p.tau)
    assert res.converged
    return res


def relx(x, xo):
    return np.linalg.norm(x - xo) / max(np.linalg.norm(xo), 1e-300)


@pytest.mark.parametrize("n", [1024, 2048, 4096, 8192])
def test_multipass_matches_oracle(threshold, n):
    threshold(1024)
    M = mf()
    p = W.dct_problem(n, n // 4, max(1, n // 100), seed=91, j=n)
    x, info = M.solve(_op(M, p), torch.from_numpy(p.b), p.tau, M.SolverParams(tol=1e-12))
    assert info["status"] == 0
    xo = _oracle(p).x
    assert relx(x.cpu().numpy(), xo) <= RELX_TOL, relx(x.cpu().numpy(), xo)
    assert 5 <= info["ipm_iters"] <= 60


def test_mixed_batch_splits_between_solvers(threshold):
    """n = 2048 stays on the persistent kernel; n = 4096 (two problems, one group) and
    n = 8192 run as lockstep groups: every x matches the oracle and the single solves."""
    threshold(4096)
    M = mf()
    probs = [W.dct_problem(n, n // 4, max(1, n // 80), seed=92, j=j)
             for j, n in enumerate([4096, 2048, 8192, 4096])]
    ops = [_op(M, p) for p in probs]
    xs, infos = M.solve_batched(ops, [torch.from_numpy(p.b) for p in probs], [p.tau for p in probs],
                                M.SolverParams(tol=1e-12))
    for p, x, info in zip(probs, xs, infos):
        assert info["status"] == 0
        assert relx(x.cpu().numpy(), _oracle(p).x) <= RELX_TOL
    # a lockstep group gives each problem the result of its single solve
    x0, _ = M.solve(ops[0], torch.from_numpy(probs[0].b), probs[0].tau, M.SolverParams(tol=1e-12))
    assert torch.equal(x0, xs[0])


def test_ragged_rows_in_a_group(threshold):
    """Problems of one length with different m (so different rho = m/n) in one group."""
    threshold(2048)
    M = mf()
    probs = [W.dct_problem(2048, m, 20, seed=93, j=m) for m in (300, 777, 1500)]
    xs, infos = M.solve_batched([_op(M, p) for p in probs], [torch.from_numpy(p.b) for p in probs],
                                [p.tau for p in probs], M.SolverParams(tol=1e-12))
    for p, x, info in zip(probs, xs, infos):
        assert info["status"] == 0
        assert relx(x.cpu().numpy(), _oracle(p).x) <= RELX_TOL


def test_zero_solution_for_large_tau(threshold):
    """tau >= ||A^T b||_inf <=> x* = 0 (l1 optimality)."""
    threshold(1024)
    M = mf()
    p = W.dct_problem(4096, 1024, 40, seed=94)
    tau = 1.01 * float(np.abs(W.dct_apply_t(p.b, p.rows, p.n)).max())
    x, info = M.solve(_op(M, p), torch.from_numpy(p.b), tau, M.SolverParams(tol=1e-12))
    assert info["status"] == 0 and float(x.abs().max()) <= 1e-8


def test_multipass_backward_matches_oracle_adjoint(threshold):
    threshold(1024)
    M = mf()
    p = W.dct_problem(4096, 1024, 40, seed=104, j=4096)
    op = _op(M, p)
    prm = M.SolverParams(tol=1e-12)
    b = torch.from_numpy(p.b).cuda()
    x, info, zs = M.solve(op, b, p.tau, prm, return_zs=True)
    gx = np.random.default_rng(2).standard_normal(p.n)
    gbs, gts, _, infos = M.backward([op], [b], [p.tau], [x], [zs], [torch.from_numpy(gx).cuda()], prm)
    res = _oracle(p)
    rb, rt, _ = O.adjoint_kkt(O.Operator.from_dct_rows(p.n, p.rows), p.b, p.tau, res.z, res.s, gx)
    gb = gbs[0].cpu().numpy()
    # float32 adjoint PCG to min(tol_pcg, 1e-6): measured 3.2e-7 (grad_b), 1.4e-7 (grad_tau)
    assert np.abs(gb - rb).max() <= 5e-6 * np.abs(rb).max()
    assert abs(gts[0] - rt) <= 5e-6 * max(1.0, abs(rt))
    assert infos[0]["status"] == 0 and infos[0]["pcg_iters"] > 0


def _certificates(p, x):
    op = O.Operator.from_dct_rows(p.n, p.rows, explicit=False)
    kkt = O.kkt_rel(op, p.b, p.tau, x)
    P, D = O.dual_gap_certificate(op, p.b, p.tau, x)
    return kkt, (P - D) / max(1.0, abs(P))


def test_full_size_n_1m_certificates_and_derivative():
    """Two n = 2^20, m = 2^18 problems of the adjoint workload: kkt_rel <= 1e-6 and a small
    l1 duality-gap certificate (oracle quantities on the CPU); the derivative in tau of
    L = 1/2||x* - x_hat||^2 against a central difference of two more GPU solves."""
    M = mf()
    probs = W.make_workload("dct_adjoint_32x1M", count=2)
    ops = [_op(M, p) for p in probs]
    bs = [torch.from_numpy(p.b).cuda() for p in probs]
    prm = M.SolverParams(tol=1e-10)
    xs, infos, zss = M.solve_batched(ops, bs, [p.tau for p in probs], prm, return_zs=True)
    for p, x, info in zip(probs, xs, infos):
        assert info["status"] == 0
        kkt, gap = _certificates(p, x.cpu().numpy())
        assert kkt <= 1e-6 and gap <= 1e-5, (kkt, gap)
    p, x = probs[0], xs[0].cpu().numpy()
    gx = torch.from_numpy(x - p.x_hat).cuda()
    gbs, gts, _, binfo = M.backward(ops[:1], bs[:1], [p.tau], xs[:1], zss[:1], [gx], prm)
    assert binfo[0]["status"] == 0 and np.isfinite(gbs[0].cpu().numpy()).all()
    prm_fd = M.SolverParams(tol=1e-12)
    L = lambda t: 0.5 * float(np.sum((M.solve(ops[0], bs[0], t, prm_fd)[0].cpu().numpy() - p.x_hat) ** 2))
    ht = 1e-4 * p.tau
    fd_t = (L(p.tau + ht) - L(p.tau - ht)) / (2 * ht)
    assert abs(fd_t - gts[0]) <= 1e-3 * abs(fd_t) + 1e-9, (fd_t, gts[0])


def test_no_measurements_gives_zero_multipass(threshold):
    threshold(1024)
    M = mf()
    op = M.PartialDCT(2048, torch.zeros(0, dtype=torch.int64))
    x, info = M.solve(op, torch.zeros(0, dtype=torch.float64), 0.1, M.SolverParams(tol=1e-12))
    assert info["status"] == 0 and float(x.abs().max()) <= 1e-8 and info["kkt_rel"] <= 1e-8
