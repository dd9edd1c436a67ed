"""Pins for the oracle's derivatives of the solution map: central finite differences of the
oracle's own solve (x* is piecewise linear in (b, tau, A) with fixed support, so central
differences with a small step are exact up to the solve's accuracy), and the two derivative
forms (exact KKT adjoint at the final iterate, closed form on the support) against each
other."""
import numpy as np
import pytest

import workloads as W
from oracle import mfipm_oracle as O

P_TIGHT = O.OracleParams(tol=1e-14, max_iter=150)


def _solve(A, b, tau):
    return O.ipm(O.Operator.from_dense(A), b, tau, P_TIGHT)


def _margin(A, b, tau, x):
    g = A.T @ (A @ x - b)
    off = np.abs(x) <= 1e-7
    return float(np.min(tau - np.abs(g[off]))) / tau if off.any() else 1.0


@pytest.mark.parametrize("seed", [3, 4])
def test_adjoint_matches_finite_differences(seed):
    p = W.dense_problem(24, 64, 4, seed=100 + seed, sigma=1e-2)
    A, b, tau = p.A, p.b, p.tau
    res = _solve(A, b, tau)
    x = res.x
    assert _margin(A, b, tau, x) > 1e-3
    rng = np.random.default_rng(seed)
    gx = rng.standard_normal(A.shape[1])
    gb, gt, gA = O.adjoint_kkt(O.Operator.from_dense(A), b, tau, res.z, res.s, gx)
    gb2, gt2, gA2 = O.adjoint_support(A, b, tau, x, gx)
    assert np.abs(gb - gb2).max() <= 1e-8 * np.abs(gb2).max()
    assert abs(gt - gt2) <= 1e-8 * abs(gt2) + 1e-12
    assert np.abs(gA - gA2).max() <= 1e-8 * np.abs(gA2).max()
    # central differences of L = grad_x . x*(.) along random directions
    h = 1e-5
    db = rng.standard_normal(b.size)
    fd_b = (gx @ _solve(A, b + h * db, tau).x - gx @ _solve(A, b - h * db, tau).x) / (2 * h)
    assert abs(fd_b - gb @ db) <= 1e-6 * (abs(fd_b) + 1e-3)
    ht = 1e-5 * tau
    fd_t = (gx @ _solve(A, b, tau + ht).x - gx @ _solve(A, b, tau - ht).x) / (2 * ht)
    assert abs(fd_t - gt) <= 1e-6 * (abs(fd_t) + 1e-3)
    dA = rng.standard_normal(A.shape)
    fd_A = (gx @ _solve(A + h * dA, b, tau).x - gx @ _solve(A - h * dA, b, tau).x) / (2 * h)
    assert abs(fd_A - np.sum(gA * dA)) <= 1e-6 * (abs(fd_A) + 1e-3)


def test_adjoint_of_orthonormal_closed_form():
    """Orthonormal square A: x* = S_tau(A^T b), so dL/db = A (grad_x * 1[x != 0]) and
    dL/dtau = -sum_{x_i != 0} sign(x_i) grad_x_i."""
    n = 32
    rng = np.random.default_rng(7)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    b = rng.standard_normal(n)
    tau = 0.3 * np.abs(Q.T @ b).max()
    res = _solve(Q, b, tau)
    gx = rng.standard_normal(n)
    on = np.abs(O.soft_threshold(Q.T @ b, tau)) > 0
    gb, gt, _ = O.adjoint_kkt(O.Operator.from_dense(Q), b, tau, res.z, res.s, gx)
    assert np.abs(gb - Q @ (gx * on)).max() < 1e-8
    assert abs(gt + np.sum(np.sign(Q.T @ b)[on] * gx[on])) < 1e-8
