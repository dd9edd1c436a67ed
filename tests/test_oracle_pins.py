"""Pins for the CPU oracle: each check ties the oracle to something other than itself
(a closed form, brute force, a textbook linear solve, a theorem of the paper, a library
routine, or a value the paper prints).  The last group plants mistakes in the oracle and
checks that some pin catches each one."""
import dataclasses
import itertools
import json
import math
import os

import numpy as np
import pytest
import scipy.fft
import scipy.stats

import workloads as W
from oracle import mfipm_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(s):
    return np.random.default_rng(s)


def _gauss_problem(m, n, k, seed, sigma=1e-3, tau_frac=0.05):
    rng = _rng(seed)
    A = rng.standard_normal((m, n)) / np.sqrt(m)
    x = np.zeros(n)
    x[rng.choice(n, k, replace=False)] = rng.choice([-1.0, 1.0], k)
    b = A @ x + sigma * rng.standard_normal(m)
    tau = tau_frac * np.abs(A.T @ b).max()
    return A, b, tau


# ---------------------------------------------------------------- pin functions
def pin_closed_form_error(seed=3, n=48):
    """Orthonormal square A: x* = S_tau(A^T b) (separable problem)."""
    rng = _rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    b = rng.standard_normal(n)
    tau = 0.4 * np.abs(Q.T @ b).max()
    res = O.ipm(O.Operator.from_dense(Q), b, tau)
    return float(np.abs(res.x - O.soft_threshold(Q.T @ b, tau)).max())


def brute_force_l1ls(A, b, tau):
    """Enumerate sign patterns s in {-1,0,1}^n; on the support solve the stationarity
    equations A_S^T A_S x_S = A_S^T b - tau s_S and keep the consistent candidate."""
    m, n = A.shape
    best = None
    for signs in itertools.product((-1, 0, 1), repeat=n):
        s = np.array(signs, dtype=float)
        S = np.nonzero(s)[0]
        x = np.zeros(n)
        if S.size:
            if S.size > m:
                continue
            AS = A[:, S]
            G = AS.T @ AS
            if np.linalg.cond(G) > 1e12:
                continue
            x[S] = np.linalg.solve(G, AS.T @ b - tau * s[S])
            if np.any(np.sign(x[S]) != s[S]):
                continue
        g = A.T @ (A @ x - b)
        off = np.setdiff1d(np.arange(n), S)
        if off.size and np.any(np.abs(g[off]) > tau * (1 + 1e-9)):
            continue
        f = tau * np.abs(x).sum() + 0.5 * np.sum((A @ x - b) ** 2)
        if best is None or f < best[0]:
            best = (f, x)
    return best[1]


def pin_brute_force_error(seed=5, m=5, n=8):
    A, b, tau = _gauss_problem(m, n, 2, seed, sigma=0.05, tau_frac=0.15)
    xb = brute_force_l1ls(A, b, tau)
    res = O.ipm(O.Operator.from_dense(A), b, tau)
    return float(np.abs(res.x - xb).max())


def pin_full_kkt_error(seed=7, m=3, n=6):
    """Eliminated system (Eqs. redNewtonA/B) vs the 4n x 4n block system (Eq. sepregaugeq)
    solved with a textbook dense solver."""
    rng = _rng(seed)
    A = rng.standard_normal((m, n))
    op = O.Operator.from_dense(A)
    b = rng.standard_normal(m)
    tau = 0.3
    z = rng.uniform(0.1, 2.0, 2 * n)
    s = rng.uniform(0.1, 2.0, 2 * n)
    c = O.c_vector(op, b, tau)
    fz, mu = O.residuals(op, b, tau, z, s, c)
    fs = 0.3 * mu - z * s
    Ft = np.hstack([A, -A])
    FFt = Ft.T @ Ft
    K = np.block([[FFt, -np.eye(2 * n)], [np.diag(s), np.diag(z)]])
    sol = np.linalg.solve(K, np.concatenate([fz, fs]))
    d = s / z
    rhs = O.newton_rhs(fz, fs, z)
    errs = []
    for solver in (O.solve_full_cholesky, O.solve_woodbury):
        dz = solver(op, d, rhs)
        ds = O.recover_ds(fs, z, d, dz)
        errs.append(float(np.abs(np.concatenate([dz, ds]) - sol).max() / np.abs(sol).max()))
    # and f_z against its definition s - c - F F^T z with c written out
    atb = A.T @ b
    c_def = np.concatenate([tau * np.ones(n) - atb, tau * np.ones(n) + atb])
    errs.append(float(np.abs(fz - (s - c_def - FFt @ z)).max()))
    return max(errs)


def pin_central_path_error(seed=17, n=10):
    """On the central path z o s = mu e, mu from Eq. fzfs equals that mu and the perturbed
    complementarity residual is zero for sigma = 1 (Sec. 4)."""
    rng = _rng(seed)
    A = rng.standard_normal((4, n))
    op = O.Operator.from_dense(A)
    b = rng.standard_normal(4)
    z = rng.uniform(0.1, 3.0, 2 * n)
    mu0 = 0.37
    s = mu0 / z
    _, mu = O.residuals(op, b, 0.2, z, s, O.c_vector(op, b, 0.2))
    fs = O.complementarity_rhs(z, s, 1.0, mu)
    return max(abs(mu - mu0), float(np.abs(fs).max()))


def pin_theorem_error(seed=11, n=16, m=4, kind="dct"):
    """Theorem thm:ne2_prec: P^-1 H has eigenvalue 1 with multiplicity n, and its other n
    eigenvalues are those of (Theta^-1 + rho I)^-1 (Theta^-1 + A^T A) with
    Theta = Theta_u + Theta_v (Lemma lem:ne2_prec)."""
    rng = _rng(seed)
    if kind == "dct":
        rows = np.sort(rng.choice(n, m, replace=False))
        op = O.Operator.from_dct_rows(n, rows)
    else:
        op = O.Operator.from_dense(rng.standard_normal((m, n)) / np.sqrt(m))
    A = op.dense
    rho = O.rho_of(op)
    d = np.exp(rng.uniform(-6, 6, 2 * n))
    H = O.newton_matrix(op, d)
    Pinv = np.stack([O.precond_apply(d, rho, e) for e in np.eye(2 * n)], axis=1)
    ev = np.sort(np.linalg.eigvals(Pinv @ H).real)
    ones = np.abs(ev - 1.0) < 1e-7
    theta = 1.0 / d[:n] + 1.0 / d[n:]
    Hn = np.diag(1.0 / theta) + A.T @ A
    Pn = np.diag(1.0 / theta + rho)
    evn = np.sort(np.linalg.eigvals(np.linalg.solve(Pn, Hn)).real)
    # remove n copies of 1 from the 2n spectrum and compare the rest with the Lemma's
    rest = list(ev)
    for _ in range(n):
        i = int(np.argmin(np.abs(np.array(rest) - 1.0)))
        rest.pop(i)
    err_rest = float(np.max(np.abs(np.sort(rest) - evn) / np.maximum(1.0, np.abs(evn))))
    count_err = 0.0 if ones.sum() >= n else 1.0
    return max(err_rest, count_err)


def pin_pcg_one_iteration(seed=13, n=32):
    """A A^T = I with m = n (full DCT) gives A^T A = I, rho = 1 and P = H exactly
    (Eq. eq:ne2_P), so PCG converges in one iteration to the exact solution."""
    rng = _rng(seed)
    op = O.Operator.from_dct_rows(n, np.arange(n))
    rho = O.rho_of(op)
    d = np.exp(rng.uniform(-4, 4, 2 * n))
    r = rng.standard_normal(2 * n)
    x, it = O.pcg(op, d, r, rho, 1e-12)
    xd = np.linalg.solve(O.newton_matrix(op, d), r)
    return it, float(np.abs(x - xd).max() / np.abs(xd).max()), abs(rho - 1.0)


def pin_corrector_error(seed=19, m=3, n=6, aP=0.07, aD=0.04):
    """One corrector step of the Algorithm (Sec. 5.1) at a fixed interior (z, s), against the
    4n x 4n block system of Eq. sepregaugeq solved by a textbook dense solver.  The predictor
    solves K [dz; ds] = [f_z; f_s] with K = [[F F^T, -I], [S, Z]] at (z, s); under reading R6
    the corrector solves the same K for the residuals of Eq. fzfs at the trial point
    (z + aP dz, s + aD ds) with sigma3 and the trial point's mu; the combined direction is
    the sum.  Every quantity here is written out from Eqs. sepregaugeq and fzfs, not taken
    from the oracle."""
    rng = _rng(seed)
    A = rng.standard_normal((m, n))
    b = rng.standard_normal(m)
    tau, sigma = 0.3, 0.1
    z = rng.uniform(0.1, 2.0, 2 * n)
    s = rng.uniform(0.1, 2.0, 2 * n)
    Ft = np.hstack([A, -A])
    FFt = Ft.T @ Ft
    atb = A.T @ b
    c_def = np.concatenate([tau * np.ones(n) - atb, tau * np.ones(n) + atb])
    K = np.block([[FFt, -np.eye(2 * n)], [np.diag(s), np.diag(z)]])
    mu = float(z @ s) / (2 * n)
    pred = np.linalg.solve(K, np.concatenate([s - c_def - FFt @ z, sigma * mu - z * s]))
    zt, st = z + aP * pred[:2 * n], s + aD * pred[2 * n:]
    mut = float(zt @ st) / (2 * n)
    corr = np.linalg.solve(K, np.concatenate([st - c_def - FFt @ zt, 0.8 * mut - zt * st]))
    want = pred + corr
    # the oracle's predictor and corrector (Eqs. redNewtonA/B, exact solves)
    op = O.Operator.from_dense(A)
    c = O.c_vector(op, b, tau)
    fz, mu_o = O.residuals(op, b, tau, z, s, c)
    fs = O.complementarity_rhs(z, s, sigma, mu_o)
    d = s / z
    dz = O.solve_full_cholesky(op, d, O.newton_rhs(fz, fs, z))
    ds = O.recover_ds(fs, z, d, dz)
    dz2, ds2 = O.corrector_direction(op, b, tau, c, z, s, d, z + aP * dz, s + aD * ds, O.SIGMA3,
                                     lambda dd, r: O.solve_full_cholesky(op, dd, r))
    got = np.concatenate([dz + dz2, ds + ds2])
    return float(np.abs(got - want).max() / np.abs(want).max())


def pin_mcc_step_error(seed=31, m=3, n=6, aP=0.3, aD=0.5, mu_t=0.05):
    """One multiple-centrality corrector (reading R19) at a fixed interior (z, s) and a fixed
    direction, against the 4n x 4n block system of Eq. sepregaugeq with right-hand side
    (0, t): t written out here from the box [0.1 mu_t, 10 mu_t] around mu_t at the trial point
    of the aspiration steps alpha + 0.1."""
    rng = _rng(seed)
    A = rng.standard_normal((m, n))
    z = rng.uniform(0.05, 2.0, 2 * n)
    s = rng.uniform(0.05, 2.0, 2 * n)
    dz, ds = rng.standard_normal(2 * n), rng.standard_normal(2 * n)
    Ft = np.hstack([A, -A])
    K = np.block([[Ft.T @ Ft, -np.eye(2 * n)], [np.diag(s), np.diag(z)]])
    v = (z + min(1.0, aP + 0.1) * dz) * (s + min(1.0, aD + 0.1) * ds)
    t = np.where(v < 0.1 * mu_t, 0.1 * mu_t - v, np.where(v > 10 * mu_t, np.maximum(10 * mu_t - v, -10 * mu_t), 0.0))
    assert np.count_nonzero(t) > 0
    want = np.linalg.solve(K, np.concatenate([np.zeros(2 * n), t]))
    op = O.Operator.from_dense(A)
    d = s / z
    prm = O.OracleParams(mcc=1, mcc_gamma=-1e9)   # accept whatever the step does
    dz2, ds2, _, _, acc = O.centrality_correctors(z, s, d, dz, ds, aP, aD, mu_t, prm,
                                                  lambda dd, r: O.solve_full_cholesky(op, dd, r),
                                                  lambda a, b: (0.9, 0.9))
    got = np.concatenate([dz2 - dz, ds2 - ds])
    return float(np.abs(got - want).max() / np.abs(want).max()) if acc == 1 else 1.0


def _orthonormal_problem(seed, n=40):
    rng = _rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    b = rng.standard_normal(n)
    tau = 0.3 * np.abs(Q.T @ b).max()
    return Q, b, tau, rng


def pin_kkt_off_optimum_error(seed=23, n=40):
    """For orthonormal square Q, x - g(x) = x - Q^T (Q x - b) = Q^T b for EVERY x, so the prox
    residual has the closed form kkt_rel(x) = ||x - S_tau(Q^T b)|| / (1 + ||x||) at any x,
    not only at the minimiser."""
    Q, b, tau, rng = _orthonormal_problem(seed, n)
    op = O.Operator.from_dense(Q)
    xs = np.sign(Q.T @ b) * np.maximum(np.abs(Q.T @ b) - tau, 0.0)
    errs = []
    for scale in (1e-8, 1e-4, 1e-1, 1.0, 10.0):
        x = xs + scale * rng.standard_normal(n)
        want = np.linalg.norm(x - xs) / (1.0 + np.linalg.norm(x))
        # rounding of x - Q^T (Q x - b) is ~1e-16 |Q^T b|, so compare against a floor of 1e-7
        errs.append(abs(O.kkt_rel(op, b, tau, x) - want) / max(want, 1e-7))
    return max(errs)


def pin_certificate_chain_violation(seed=29, n=40):
    """For orthonormal square Q the minimum is known in closed form, P* = P(S_tau(Q^T b)).
    At perturbed x (several magnitudes) the certificate must satisfy weak duality,
    P(x) - D(nu) >= P(x) - P* >= 0, with nu dual-feasible (||Q^T nu||_inf <= tau).
    Returns the largest violation (0 when every inequality holds)."""
    Q, b, tau, rng = _orthonormal_problem(seed, n)
    op = O.Operator.from_dense(Q)
    xs = np.sign(Q.T @ b) * np.maximum(np.abs(Q.T @ b) - tau, 0.0)
    Pstar = tau * np.abs(xs).sum() + 0.5 * np.sum((Q @ xs - b) ** 2)
    viol = 0.0
    for scale in (0.0, 1e-6, 1e-3, 1e-1, 1.0, 10.0):
        x = xs + scale * rng.standard_normal(n)
        Px = tau * np.abs(x).sum() + 0.5 * np.sum((Q @ x - b) ** 2)
        P, D = O.dual_gap_certificate(op, b, tau, x)
        nu = O.dual_point(op, b, tau, x)
        tol = 1e-12 * (1.0 + abs(Pstar))
        viol = max(viol, abs(P - Px) - tol, D - Pstar - tol, Pstar - Px - tol,
                   float(np.abs(Q.T @ nu).max()) - tau * (1 + 1e-12))
    # x = 0 with tau < ||Q^T b||_inf: the unscaled residual -b is infeasible; the scaled
    # point must still bound P* from below
    P0, D0 = O.dual_gap_certificate(op, b, tau, np.zeros(n))
    viol = max(viol, D0 - Pstar - 1e-12 * (1.0 + abs(Pstar)))
    return max(viol, 0.0)


# ---------------------------------------------------------------- tests
@pytest.mark.parametrize("n", [256, 1000, 250])
def test_dct_rows_orthonormal_and_match_library(n):
    """The DCT rows from their definition at a power of two and at the general lengths of the
    mixed-radix chain (n = 1000 of Sec. 5.8; n/2 = 125 odd)."""
    rows = np.sort(_rng(1).choice(n, 64, replace=False))
    A = O.dct_matrix_rows(n, rows)
    assert np.abs(A @ A.T - np.eye(64)).max() < 1e-12          # Eq. eq:orthonormality
    x = _rng(2).standard_normal(n)
    lib = scipy.fft.dct(x, type=2, norm="ortho")[rows]          # library DCT-II
    assert np.abs(A @ x - lib).max() < 1e-12
    y = _rng(3).standard_normal(64)
    assert abs((A @ x) @ y - x @ (A.T @ y)) < 1e-12
    full = O.dct_matrix_rows(n, np.arange(n))
    assert np.abs(full.T @ full - np.eye(n)).max() < 1e-12


@pytest.mark.parametrize("n", [64, 60])
def test_closed_form_orthonormal_square(n):
    assert pin_closed_form_error() < 1e-9
    # full DCT (m = n) as well, at a power of two and at n = 60 (n/2 = 2^2 3 5)
    op = O.Operator.from_dct_rows(n, np.arange(n))
    b = _rng(4).standard_normal(n)
    tau = 0.3 * np.abs(op.rmv(b)).max()
    res = O.ipm(op, b, tau)
    assert np.abs(res.x - O.soft_threshold(op.rmv(b), tau)).max() < 1e-9


def test_zero_solution_iff_tau_large():
    A, b, _ = _gauss_problem(20, 60, 4, 21)
    op = O.Operator.from_dense(A)
    lam = np.abs(A.T @ b).max()
    res = O.ipm(op, b, 1.01 * lam)
    assert np.abs(res.x).max() < 1e-9
    res2 = O.ipm(op, b, 0.9 * lam)
    assert np.abs(res2.x).max() > 1e-4


def test_brute_force_support_enumeration():
    assert pin_brute_force_error() < 1e-8
    assert pin_brute_force_error(seed=6, m=4, n=7) < 1e-8


@pytest.mark.parametrize("kind", ["dense", "dct"])
def test_l1_optimality_and_dual_gap_certificate(kind):
    if kind == "dense":
        p = W.make_workload("dense_fp64_256x1024")[0]
        op = O.Operator.from_dense(p.A)
    else:
        p = W.make_workload("dct_65536", scale_n=2048)[0]
        op = O.Operator.from_dct_rows(p.n, p.rows)
    res = O.ipm(op, p.b, p.tau)
    assert res.converged and 10 <= res.iters <= 40          # Sec. 5.1: 10-20 iterations typical
    v_on, v_off = O.optimality_violation(op, p.b, p.tau, res.x, support_tol=1e-7)
    assert v_on < 1e-8 * max(1.0, p.tau) + 1e-10 and v_off < 1e-10
    P, D = O.dual_gap_certificate(op, p.b, p.tau, res.x)
    assert P - D >= -1e-12 and (P - D) / (1 + abs(P)) < 1e-10
    assert O.kkt_rel(op, p.b, p.tau, res.x) < 1e-10


def test_corrector_step_matches_block_system():
    assert pin_corrector_error() < 1e-10
    assert pin_corrector_error(seed=20, m=4, n=9, aP=0.01, aD=0.09) < 1e-10


@pytest.mark.parametrize("pin,bar", [(pin_closed_form_error, 1e-9), (pin_brute_force_error, 1e-8)])
def test_ipm_with_a_corrector_every_iteration(pin, bar, monkeypatch):
    """alpha_tilde = 1 makes the corrector test of the Algorithm true at every iteration
    (alpha <= 1 always): the closed-form and brute-force pins still hold, and every
    iteration that computed a direction also took a corrector."""
    seen = []
    orig = O.ipm

    def ipm_every(op, b, tau, params=None):
        q = dataclasses.replace(params or O.OracleParams(), alpha_tilde=1.0)
        r = orig(op, b, tau, q)
        seen.append(r)
        return r

    monkeypatch.setattr(O, "ipm", ipm_every)
    assert pin() < bar
    r = seen[-1]
    assert r.converged and r.correctors == r.iters - 1 > 0


def test_ipm_corrector_optimality_dense():
    A, b, tau = _gauss_problem(30, 90, 5, 61)
    op = O.Operator.from_dense(A)
    r = O.ipm(op, b, tau, O.OracleParams(alpha_tilde=1.0))
    r0 = O.ipm(op, b, tau)
    assert r.converged and r.correctors == r.iters - 1 > 0
    v_on, v_off = O.optimality_violation(op, b, tau, r.x, support_tol=1e-7)
    assert v_on < 1e-8 and v_off < 1e-10
    assert np.linalg.norm(r.x - r0.x) / np.linalg.norm(r0.x) < 1e-8


def test_mcc_step_matches_block_system():
    assert pin_mcc_step_error() < 1e-10
    assert pin_mcc_step_error(seed=32, m=4, n=9, aP=0.95, aD=0.2, mu_t=0.3) < 1e-10


@pytest.mark.parametrize("pin,bar", [(pin_closed_form_error, 1e-9), (pin_brute_force_error, 1e-8)])
def test_ipm_with_multiple_centrality_correctors(pin, bar, monkeypatch):
    """mcc = 3: the closed-form and brute-force pins still hold, and correctors were taken."""
    seen = []
    orig = O.ipm

    def ipm_mcc(op, b, tau, params=None):
        r = orig(op, b, tau, dataclasses.replace(params or O.OracleParams(), mcc=3))
        seen.append(r)
        return r

    monkeypatch.setattr(O, "ipm", ipm_mcc)
    assert pin() < bar
    assert seen[-1].converged


def test_mcc_takes_correctors_and_saves_iterations():
    A, b, tau = _gauss_problem(40, 160, 6, 81)
    op = O.Operator.from_dense(A)
    r0 = O.ipm(op, b, tau)
    r = O.ipm(op, b, tau, O.OracleParams(mcc=3))
    assert r.converged and r.correctors > 0 and r.iters <= r0.iters
    assert np.linalg.norm(r.x - r0.x) <= 1e-8 * np.linalg.norm(r0.x)


def test_kkt_rel_closed_form_away_from_optimum():
    assert pin_kkt_off_optimum_error() < 1e-9


def test_certificate_weak_duality_chain_away_from_optimum():
    assert pin_certificate_chain_violation() == 0.0
    # and the bound is tight at the optimum (gap ~ 0)
    Q, b, tau, _ = _orthonormal_problem(29)
    xs = O.soft_threshold(Q.T @ b, tau)
    P, D = O.dual_gap_certificate(O.Operator.from_dense(Q), b, tau, xs)
    assert abs(P - D) <= 1e-12 * (1 + abs(P))


def test_central_path_fixed_point():
    assert pin_central_path_error() < 1e-14


def test_newton_elimination_matches_full_system():
    assert pin_full_kkt_error() < 1e-10


def test_woodbury_matches_cholesky_direction():
    A, b, tau = _gauss_problem(10, 30, 3, 31)
    op = O.Operator.from_dense(A)
    d = np.exp(_rng(32).uniform(-10, 10, 60))
    r = _rng(33).standard_normal(60)
    x1 = O.solve_full_cholesky(op, d, r)
    x2 = O.solve_woodbury(op, d, r)
    assert np.abs(x1 - x2).max() / np.abs(x1).max() < 1e-9


@pytest.mark.parametrize("kind", ["dct", "dense"])
def test_theorem_eigenvalue_one_multiplicity_n(kind):
    assert pin_theorem_error(kind=kind) < 1e-6


def test_pcg_one_iteration_when_preconditioner_is_exact():
    it, err, drho = pin_pcg_one_iteration()
    assert it == 1 and err < 1e-10 and drho < 1e-12


def test_pcg_agrees_with_direct_and_ipm_variants_agree():
    A, b, tau = _gauss_problem(40, 120, 6, 41)
    op = O.Operator.from_dense(A)
    d = np.exp(_rng(42).uniform(-3, 3, 240))
    r = _rng(43).standard_normal(240)
    x, _ = O.pcg(op, d, r, O.rho_of(op), 1e-13, maxiter=2000)
    assert np.abs(x - O.solve_full_cholesky(op, d, r)).max() / np.abs(x).max() < 1e-8
    rd = O.ipm(op, b, tau)
    rp = O.ipm(op, b, tau, O.OracleParams(solver="pcg", tol=1e-11, tol_pcg=1e-2))
    assert np.linalg.norm(rp.x - rd.x) / np.linalg.norm(rd.x) < 1e-6
    # Sec. 5.7: the PCG variant needs about as few IPM iterations as the direct one
    assert abs(rp.iters - rd.iters) <= 4


def test_paper_parameters_golden():
    g = json.load(open(os.path.join(GOLDEN, "paper_parameters.json")))
    assert (O.SIGMA1, O.SIGMA2, O.SIGMA3) == (g["sigma1"], g["sigma2"], g["sigma3"])
    assert (O.ALPHA_BAR, O.ALPHA_TILDE) == (g["alpha_bar"], g["alpha_tilde"])
    assert (O.MAXITERS, O.MXITERPCG) == (g["maxiters"], g["mxiterpcg"])
    p = O.OracleParams()
    assert (p.sigma1, p.sigma2, p.sigma3, p.alpha_bar, p.alpha_tilde, p.max_iter) == (
        g["sigma1"], g["sigma2"], g["sigma3"], g["alpha_bar"], g["alpha_tilde"], g["maxiters"])
    # the Lemma's separator constants the paper prints
    C = lambda delta: 20 * (0.75 + delta + 2 * math.sqrt(1 + delta)) ** 2 / 3
    assert abs(C(0.0) - g["C_orthonormal_delta0"]) < 0.01
    assert abs(C(1.0) - g["C_near_orthonormal_delta1"]) < 0.01


def test_step_to_boundary_rules():
    z = np.array([1.0, 2.0, 0.5])
    assert O.step_to_boundary(z, np.array([1.0, 0.0, 3.0]), 0.995) == 1.0
    a = O.step_to_boundary(z, np.array([-4.0, 1.0, -0.25]), 0.995)
    assert abs(a - 0.995 * 0.25) < 1e-15
    assert O.step_to_boundary(z, np.array([-0.1, -0.1, -0.1]), 0.995) == 1.0


def test_workload_generators_deterministic():
    a = W.dct_problem(4096, 1024, 40, seed=9, j=3)
    b = W.dct_problem(4096, 1024, 40, seed=9, j=3)
    assert np.array_equal(a.rows, b.rows) and np.array_equal(a.b, b.b) and a.tau == b.tau
    assert np.all(np.diff(a.rows) > 0) and a.rows.min() >= 0 and a.rows.max() < 4096
    sizes = W.batch_sizes(256, 1003)
    assert all(n in (4096, 8192, 16384, 32768, 65536) and m == n // 4 and n // 100 <= k <= n // 20
               for n, m, k in sizes)
    bits = W.bf16_round(np.array([1.0, 1.00390625, 1.005859375, -3.0]))
    assert list(bits) == [0x3F80, 0x3F80, 0x3F81, 0xC040]   # ties to even, then round up


# ---------------------------------------------------------------- planted mistakes
@pytest.mark.parametrize("mutation", ["c_sign", "drop_sigma_mu", "ds_sign", "precond_offdiag",
                                      "rho_sign", "rhs_no_zinv", "step_eta", "corr_sigma1", "corr_zinv_trial",
                                      "corr_rhs_at_current", "corr_dropped"])
def test_planted_mistake_is_caught(monkeypatch, mutation):
    orig = {k: getattr(O, k) for k in ("c_vector", "residuals", "recover_ds", "precond_apply",
                                       "newton_rhs", "step_to_boundary", "ipm", "corrector_direction")}
    if mutation == "c_sign":
        monkeypatch.setattr(O, "c_vector", lambda op, b, tau: -orig["c_vector"](op, b, tau) + 2 * tau)
    elif mutation == "drop_sigma_mu":
        monkeypatch.setattr(O, "complementarity_rhs", lambda z, s, sigma, mu: -z * s)
    elif mutation == "ds_sign":
        monkeypatch.setattr(O, "recover_ds", lambda fs, z, d, dz: fs / z + d * dz)
    elif mutation == "precond_offdiag":
        def pa(d, rho, r):
            n = d.size // 2
            du, dv, ru, rv = d[:n], d[n:], r[:n], r[n:]
            det = (du + rho) * (dv + rho) - rho * rho
            return np.concatenate([((dv + rho) * ru - rho * rv) / det, (-rho * ru + (du + rho) * rv) / det])
        monkeypatch.setattr(O, "precond_apply", pa)
    elif mutation == "rho_sign":
        monkeypatch.setattr(O, "precond_apply", lambda d, rho, r: orig["precond_apply"](d, -rho, r))
    elif mutation == "rhs_no_zinv":
        monkeypatch.setattr(O, "newton_rhs", lambda fz, fs, z: fz + fs)
    elif mutation == "step_eta":
        monkeypatch.setattr(O, "step_to_boundary", lambda v, dv, eta: orig["step_to_boundary"](v, dv, 1.2))
    elif mutation == "corr_sigma1":          # predictor's centring in the corrector
        monkeypatch.setattr(O, "corrector_direction", lambda op, b, tau, c, z, s, d, zt, st, sigma3, solve:
                            orig["corrector_direction"](op, b, tau, c, z, s, d, zt, st, O.SIGMA1, solve))
    elif mutation == "corr_zinv_trial":      # Z^-1 of the trial point instead of the current one
        def cd(op, b, tau, c, z, s, d, zt, st, sigma3, solve):
            fzt, mut = O.residuals(op, b, tau, zt, st, c)
            fst = O.complementarity_rhs(zt, st, sigma3, mut)
            dz2 = solve(d, O.newton_rhs(fzt, fst, zt))
            return dz2, O.recover_ds(fst, zt, d, dz2)
        monkeypatch.setattr(O, "corrector_direction", cd)
    elif mutation == "corr_rhs_at_current":  # residuals of the current point, not the trial point
        monkeypatch.setattr(O, "corrector_direction", lambda op, b, tau, c, z, s, d, zt, st, sigma3, solve:
                            orig["corrector_direction"](op, b, tau, c, z, s, d, z, s, sigma3, solve))
    elif mutation == "corr_dropped":         # the predictor alone
        monkeypatch.setattr(O, "corrector_direction", lambda op, b, tau, c, z, s, d, zt, st, sigma3, solve:
                            (np.zeros_like(z), np.zeros_like(s)))

    caught = []
    for pin, ok in ((pin_closed_form_error, lambda e: e < 1e-9),
                    (pin_brute_force_error, lambda e: e < 1e-8),
                    (pin_full_kkt_error, lambda e: e < 1e-10),
                    (pin_theorem_error, lambda e: e < 1e-6),
                    (pin_central_path_error, lambda e: e < 1e-14),
                    (pin_corrector_error, lambda e: e < 1e-10)):
        try:
            with np.errstate(all="ignore"):
                e = pin()
            caught.append(not ok(e))
        except Exception:
            caught.append(True)
    try:
        it, err, _ = pin_pcg_one_iteration()
        caught.append(not (it == 1 and err < 1e-10))
    except Exception:
        caught.append(True)
    assert any(caught), f"mutation {mutation} slipped through every pin"


@pytest.mark.parametrize("mutation", ["kkt_zero", "kkt_no_prox", "nu_unscaled", "nu_zero_gap"])
def test_planted_certificate_mistake_is_caught(monkeypatch, mutation):
    """The certificates (the prox residual and the l1 dual-gap bound) are the only parity
    evidence at sizes beyond the oracle's direct solve; a mistake in either must fail a pin
    that holds away from the optimum."""
    orig_kkt, orig_dual = O.kkt_rel, O.dual_point
    if mutation == "kkt_zero":
        monkeypatch.setattr(O, "kkt_rel", lambda op, b, tau, x: 0.0)
    elif mutation == "kkt_no_prox":          # ||g|| instead of the prox residual
        monkeypatch.setattr(O, "kkt_rel", lambda op, b, tau, x: float(np.linalg.norm(O.gradient(op, b, x)))
                            / (1.0 + float(np.linalg.norm(x))))
    elif mutation == "nu_unscaled":          # residual not scaled into the dual feasible set
        monkeypatch.setattr(O, "dual_point", lambda op, b, tau, x: op.mv(x) - b)
    elif mutation == "nu_zero_gap":          # scaled by tau / ||g||_2 instead of the inf-norm
        def dp(op, b, tau, x):
            r = op.mv(x) - b
            g = float(np.linalg.norm(op.rmv(r)))
            return r * min(1.0, tau / g) * 4.0
        monkeypatch.setattr(O, "dual_point", dp)
    caught = []
    with np.errstate(all="ignore"):
        caught.append(not (pin_kkt_off_optimum_error() < 1e-9))
        caught.append(pin_certificate_chain_violation() != 0.0)
    assert any(caught), f"mutation {mutation} slipped through every certificate pin"


def test_pcg_breakdown_guard_returns_the_last_finite_iterate():
    """A matrix that is not positive definite (negative Theta^-1 here) makes p^T H p <= 0 on
    the first direction: the guarded PCG stops there with x = 0 instead of dividing by it."""
    A, b, tau = _gauss_problem(8, 24, 2, 71)
    op = O.Operator.from_dense(A)
    d = -1e3 * np.ones(48)
    x, it = O.pcg(op, d, _rng(72).standard_normal(48), O.rho_of(op), 1e-8)
    assert it == 0 and np.all(x == 0.0)
    # positive definite systems are untouched: the guarded PCG still solves them
    d = np.exp(_rng(73).uniform(-3, 3, 48))
    r = _rng(74).standard_normal(48)
    x, it = O.pcg(op, d, r, O.rho_of(op), 1e-12, maxiter=500)
    assert np.abs(x - O.solve_full_cholesky(op, d, r)).max() <= 1e-8 * np.abs(x).max()


@pytest.mark.parametrize("mutation", ["box_sign", "rhs_with_fz", "ds_without_t", "trial_current"])
def test_planted_mcc_mistake_is_caught(monkeypatch, mutation):
    orig_t, orig_cc = O.centrality_target, O.centrality_correctors
    if mutation == "box_sign":          # pushes away from the box
        monkeypatch.setattr(O, "centrality_target", lambda v, mu, lo, hi: -orig_t(v, mu, lo, hi))
    elif mutation == "rhs_with_fz":     # right-hand side (t, t) instead of (0, t)
        def cc(z, s, d, dz, ds, aP, aD, mu_t, p, solve, steps):
            t = O.centrality_target((z + min(1, aP + p.mcc_delta) * dz) * (s + min(1, aD + p.mcc_delta) * ds),
                                    mu_t, p.mcc_beta_min, p.mcc_beta_max)
            dzc = solve(d, O.newton_rhs(t, t, z))
            return dz + dzc, ds + O.recover_ds(t, z, d, dzc), 0.9, 0.9, 1
        monkeypatch.setattr(O, "centrality_correctors", cc)
    elif mutation == "ds_without_t":    # ds~ = -Theta^-1 dz~ (the Z^-1 t term dropped)
        def cc(z, s, d, dz, ds, aP, aD, mu_t, p, solve, steps):
            t = O.centrality_target((z + min(1, aP + p.mcc_delta) * dz) * (s + min(1, aD + p.mcc_delta) * ds),
                                    mu_t, p.mcc_beta_min, p.mcc_beta_max)
            dzc = solve(d, O.newton_rhs(np.zeros_like(t), t, z))
            return dz + dzc, ds - d * dzc, 0.9, 0.9, 1
        monkeypatch.setattr(O, "centrality_correctors", cc)
    elif mutation == "trial_current":   # products of the current point instead of the trial point
        def cc(z, s, d, dz, ds, aP, aD, mu_t, p, solve, steps):
            t = O.centrality_target(z * s, mu_t, p.mcc_beta_min, p.mcc_beta_max)
            dzc = solve(d, O.newton_rhs(np.zeros_like(t), t, z))
            return dz + dzc, ds + O.recover_ds(t, z, d, dzc), 0.9, 0.9, 1
        monkeypatch.setattr(O, "centrality_correctors", cc)
    with np.errstate(all="ignore"):
        try:
            e = pin_mcc_step_error()
        except Exception:
            e = 1.0
    assert not (e < 1e-10), f"mutation {mutation} slipped through"
