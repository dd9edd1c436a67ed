"""mfipm_backward (reverse-mode derivative of x*(b, tau, A)) against the oracle's exact KKT
adjoint and against central finite differences of the GPU forward solve."""
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


def _op(M, p):
    return M.Dense(torch.from_numpy(p.A)) if p.kind == "dense" else M.PartialDCT(p.n, torch.from_numpy(p.rows))


def _fwd_bwd(p, gx, want_A=False, **kw):
    M = mf()
    kw.setdefault("tol", 1e-12)
    prm = M.SolverParams(**kw)
    op = _op(M, p)
    b = torch.from_numpy(p.b).cuda()
    x, info, zs = M.solve(op, b, p.tau, prm, return_zs=True)
    assert info["status"] == 0
    gbs, gts, gAs, infos = M.backward([op], [b], [p.tau], [x], [zs], [torch.from_numpy(gx).cuda()], prm, want_A=want_A)
    return (x.cpu().numpy(), gbs[0].cpu().numpy(), gts[0], gAs[0].cpu().numpy() if want_A else None, infos[0])


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("pcg", ["fp64", "fp32"])
def test_dense_backward_matches_oracle_adjoint(pcg):
    p = W.dense_problem(24, 64, 4, seed=103, sigma=1e-2)
    gx = np.random.default_rng(1).standard_normal(p.n)
    x, gb, gt, gA, info = _fwd_bwd(p, gx, want_A=True, precision=0 if pcg == "fp64" else 1)
    op = O.Operator.from_dense(p.A)
    res = O.ipm(op, p.b, p.tau)
    rb, rt, rA = O.adjoint_kkt(op, p.b, p.tau, res.z, res.s, gx)
    # measured: 3e-10 on grad_b and grad_tau and 2e-8 on grad_A, whose entries are ~1e-13
    # (float64 PCG); 3e-7 (float32 PCG, tolerance min(tol_pcg, 1e-6))
    tol = 1e-7 if pcg == "fp64" else 5e-6
    assert _rel(gb, rb) <= tol and abs(gt - rt) <= tol * max(1.0, abs(rt)) and _rel(gA, rA) <= tol


@pytest.mark.parametrize("n,G", [(1024, 1), (1024, 4), (4096, 8)])
def test_dct_backward_matches_oracle_adjoint(n, G):
    p = W.dct_problem(n, n // 4, n // 100, seed=104, j=n)
    gx = np.random.default_rng(2).standard_normal(p.n)
    x, gb, gt, _, info = _fwd_bwd(p, gx, cluster_size=G)
    op = O.Operator.from_dct_rows(p.n, p.rows)
    res = O.ipm(op, p.b, p.tau)
    rb, rt, _ = O.adjoint_kkt(op, p.b, p.tau, res.z, res.s, gx)
    # float32 adjoint PCG to min(tol_pcg, 1e-6): measured <= 3.5e-7 (grad_b), 1e-6 (grad_tau)
    assert _rel(gb, rb) <= 5e-6, _rel(gb, rb)
    assert abs(gt - rt) <= 5e-6 * max(1.0, abs(rt))


def test_dct_backward_finite_differences_n4096():
    """L = 1/2||x* - x_hat||^2 at n = 2^12: directional derivatives in b and tau against
    central differences of the GPU forward solve (support unchanged inside the step)."""
    M = mf()
    p = W.make_workload("dct_adjoint_32x1M", count=1, scale_n=4096)[0]
    x, gb, gt, _, info = _fwd_bwd(p, np.zeros(p.n))  # warm
    gx = x - p.x_hat
    x, gb, gt, _, info = _fwd_bwd(p, gx)
    op = M.PartialDCT(p.n, torch.from_numpy(p.rows))
    prm = M.SolverParams(tol=1e-13)
    L = lambda b, t: 0.5 * float(np.sum((M.solve(op, torch.from_numpy(b).cuda(), t, prm)[0].cpu().numpy() - p.x_hat) ** 2))
    rng = np.random.default_rng(3)
    db = rng.standard_normal(p.m)
    h = 1e-4 * np.linalg.norm(p.b) / np.linalg.norm(db)
    fd_b = (L(p.b + h * db, p.tau) - L(p.b - h * db, p.tau)) / (2 * h)
    assert abs(fd_b - gb @ db) <= 1e-3 * abs(fd_b) + 1e-9, (fd_b, gb @ db)
    ht = 1e-4 * p.tau
    fd_t = (L(p.b, p.tau + ht) - L(p.b, p.tau - ht)) / (2 * ht)
    assert abs(fd_t - gt) <= 1e-3 * abs(fd_t) + 1e-9, (fd_t, gt)


def test_batched_backward_equals_single():
    M = mf()
    probs = [W.dct_problem(n, n // 4, n // 50, seed=105, j=j) for j, n in enumerate([512, 2048, 1024])]
    ops = [_op(M, p) for p in probs]
    bs = [torch.from_numpy(p.b).cuda() for p in probs]
    prm = M.SolverParams(tol=1e-12, cluster_size=1)
    xs, infos, zss = M.solve_batched(ops, bs, [p.tau for p in probs], prm, return_zs=True)
    gxs = [torch.ones(p.n, dtype=torch.float64, device="cuda") for p in probs]
    gbs, gts, _, _ = M.backward(ops, bs, [p.tau for p in probs], xs, zss, gxs, prm)
    for j in range(3):
        gb1, gt1, _, _ = M.backward([ops[j]], [bs[j]], [probs[j].tau], [xs[j]], [zss[j]], [gxs[j]], prm)
        assert torch.equal(gb1[0], gbs[j]) and gt1[0] == gts[j]


def test_autograd_function_matches_backward():
    M = mf()
    p = W.dense_problem(32, 96, 5, seed=106, sigma=1e-2)
    A = torch.from_numpy(p.A).cuda().requires_grad_(True)
    b = torch.from_numpy(p.b).cuda().requires_grad_(True)
    tau = torch.tensor(p.tau, dtype=torch.float64, device="cuda", requires_grad=True)
    xh = torch.from_numpy(p.x_hat).cuda()
    x = M.solve_differentiable(M.Dense(A.detach()), b, tau, M.SolverParams(tol=1e-12))
    loss = 0.5 * ((x - xh) ** 2).sum()
    loss.backward()
    op = O.Operator.from_dense(p.A)
    res = O.ipm(op, p.b, p.tau)
    gx = res.x - p.x_hat
    rb, rt, rA = O.adjoint_kkt(op, p.b, p.tau, res.z, res.s, gx)
    assert _rel(b.grad.cpu().numpy(), rb) <= 1e-5
    assert abs(tau.grad.item() - rt) <= 1e-5 * max(1.0, abs(rt))
