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


def test_general_length_beside_the_multi_pass_path():
    """A batch with n = 1000 and a power of two at or above the multi-pass threshold (lowered
    to 2048): the general length runs on the mixed-radix persistent kernel, the other in the
    lockstep multi-pass solver, in one call."""
    import ctypes
    M = mf()
    L = M.lib()
    assert L.mfipm_set_large_dct_threshold(ctypes.c_int64(2048)) == 0
    try:
        probs = [W.dct_problem(1000, 250, 10, seed=340), W.dct_problem(2048, 512, 20, seed=341)]
        ops = [M.PartialDCT(p.n, torch.from_numpy(p.rows)) for p in probs]
        xs, infos = M.solve_batched(ops, [torch.from_numpy(p.b) for p in probs], [p.tau for p in probs],
                                    M.SolverParams(tol=1e-12))
    finally:
        assert L.mfipm_set_large_dct_threshold(ctypes.c_int64(1 << 17)) == 0
    for p, x, info in zip(probs, xs, infos):
        assert info["status"] == 0, (p.n, info)
        assert relx(x.cpu().numpy(), oracle_x(p).x) <= RELX_TOL, (p.n, info)


def test_fixed_scratch_entry_point_takes_a_general_length():
    """mfipm_solve_noalloc on n = 1000 (the roots table sits in the fixed scratch too): the
    same x as mfipm_solve with a workspace, twice in a row."""
    import ctypes
    from paper_1208_5435_gb300 import _capi as C
    M = mf()
    L = M.lib()
    p = W.dct_problem(1000, 250, 10, seed=342)
    rows = torch.from_numpy(p.rows).cuda()
    b = torch.from_numpy(p.b).cuda()
    op = C.Operator()
    op.kind, op.a_dtype, op.m, op.n, op.A, op.a_scale, op.lda, op.rows = C.OP_PARTIAL_DCT, 0, p.m, p.n, None, 1.0, 0, rows.data_ptr()
    prm = C.Params()
    L.mfipm_params_default(ctypes.byref(prm))
    prm.tol = 1e-12
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    nb = ctypes.c_size_t()
    assert L.mfipm_workspace_size(ctypes.byref(op), 1, ctypes.byref(prm), ctypes.byref(nb)) == 0
    ws = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
    x_ref = torch.empty(p.n, dtype=torch.float64, device="cuda")
    info = C.Info()
    assert L.mfipm_solve(ctypes.byref(op), b.data_ptr(), p.tau, ctypes.byref(prm), x_ref.data_ptr(), None,
                         ws.data_ptr(), nb.value, ctypes.byref(info), stream) == 0, L.mfipm_last_error()
    for _ in range(2):
        x = torch.full((p.n,), float("nan"), dtype=torch.float64, device="cuda")
        inf = C.Info()
        assert L.mfipm_solve_noalloc(ctypes.byref(op), b.data_ptr(), p.tau, ctypes.byref(prm), x.data_ptr(), None,
                                     ctypes.byref(inf), stream) == 0, L.mfipm_last_error()
        assert inf.status == 0
        assert relx(x.cpu().numpy(), x_ref.cpu().numpy()) <= RELX_TOL
    assert relx(x_ref.cpu().numpy(), oracle_x(p).x) <= RELX_TOL


def test_backward_matches_oracle_adjoint():
    """mfipm_backward at n = 1000 against the oracle's exact KKT adjoint (grad_b = A w with
    the forward chain of the mixed-radix transform, grad_tau); the float32 adjoint PCG to
    min(tol_pcg, 1e-6), the bar of the power-of-two chain."""
    M = mf()
    p = W.dct_problem(1000, 250, 10, seed=343)
    gx = np.random.default_rng(3).standard_normal(p.n)
    prm = M.SolverParams(tol=1e-12)
    op = M.PartialDCT(p.n, torch.from_numpy(p.rows))
    b = torch.from_numpy(p.b).cuda()
    x, info, zs = M.solve(op, b, p.tau, prm, return_zs=True)
    assert info["status"] == 0
    gbs, gts, _, infos = M.backward([op], [b], [p.tau], [x], [zs], [torch.from_numpy(gx).cuda()], prm)
    ref = O.Operator.from_dct_rows(p.n, p.rows)
    res = O.ipm(ref, p.b, p.tau)
    rb, rt, _ = O.adjoint_kkt(ref, p.b, p.tau, res.z, res.s, gx)
    gb = gbs[0].cpu().numpy()
    assert np.abs(gb - rb).max() <= 5e-6 * np.abs(rb).max(), np.abs(gb - rb).max() / np.abs(rb).max()
    assert abs(gts[0] - rt) <= 5e-6 * max(1.0, abs(rt))


def test_operator_products_and_kkt():
    """mfipm_apply_A, mfipm_apply_At and mfipm_kkt_residual at n = 1000 against the oracle's
    DCT rows (direct sums from the definition)."""
    M = mf()
    p = W.dct_problem(1000, 250, 10, seed=344)
    op = M.PartialDCT(p.n, torch.from_numpy(p.rows))
    ref = O.Operator.from_dct_rows(p.n, p.rows)
    rng = np.random.default_rng(4)
    xr, yr = rng.standard_normal(p.n), rng.standard_normal(p.m)
    ax = M.apply_A(op, torch.from_numpy(xr)).cpu().numpy()
    aty = M.apply_At(op, torch.from_numpy(yr)).cpu().numpy()
    assert relx(ax, ref.mv(xr)) <= 1e-12 and relx(aty, ref.rmv(yr)) <= 1e-12
    k = M.kkt_residual(op, torch.from_numpy(p.b), p.tau, torch.from_numpy(xr))
    assert abs(k - O.kkt_rel(ref, p.b, p.tau, xr)) <= 1e-12 * max(1.0, k)
