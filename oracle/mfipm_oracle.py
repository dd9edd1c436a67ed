"""CPU oracle for the matrix-free primal-dual IPM of l1-regularised least squares.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or run
this module: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  It shares no code with the CUDA path.

What it computes (all float64, plain numpy; scipy only for Cholesky and the
library DCT):

* the problem  min tau*||x||_1 + 1/2||Ax-b||^2  via the split x = u - v,
  z = [u; v] >= 0 and the QP  min tau*1^T z + 1/2||F^T z - b||^2,
  F^T = [A, -A]                                      (Sec. 1, Eqs. uvDef, lintechni, wrightBPDN)
* its dual slack  s = c + F F^T z,  c = [tau - A^T b; tau + A^T b]
                                                      (Sec. 3, Eq. dualquadraticBPDN)
* the residuals f_z = s - c - F F^T z, f_s = sigma*mu*e - Z S e, mu = z^T s/(2n)
                                                      (Sec. 3, Eq. fzfs)
* the Newton direction from the reduced system
  (Theta^-1 + F F^T) dz = f_z + Z^-1 f_s,  ds = Z^-1 f_s - Theta^-1 dz,
  Theta = S^-1 Z                                      (Sec. 3, Eqs. redNewtonA, redNewtonB)
  solved EXACTLY: Cholesky of the 2n x 2n matrix, or of the m x m matrix
  I + A (Theta_u + Theta_v) A^T through the Sherman-Morrison-Woodbury identity
  (the paper's own direct-solver variant of the IPM, Sec. 5.7)
* the single-centrality-corrector primal-dual IPM loop  (Sec. 5.1, Algorithm
  "Single-Corrector Primal-Dual Matrix-Free IPM", parameters sigma1=0.1,
  sigma2=0.5, sigma3=0.8, alpha_bar=0.5, alpha_tilde=0.1)
* the paper's preconditioner P and a plain PCG on the 2n system
                                                      (Sec. 4, Eqs. eq:ne2_H, eq:ne2_P)
  used by the pins (Theorem thm:ne2_prec) and to count PCG work; the oracle's
  solve itself never uses PCG.
* certificates: the prox (KKT) residual of the l1 problem and an l1 duality-gap
  certificate.
* the operators: dense A, m rows of the orthonormal DCT-II (Sec. 2, Eq.
  eq:orthonormality) and m rows of the orthonormal Haar matrix (Sec. 2), each
  written out from its definition.

Readings where the paper is silent or ambiguous:
  R1 objective has the 1/2 factor (the QP of Eq. wrightBPDN) although Eq.
     formulationsnoisy1 prints it without;
  R2 rho = ||A||_F^2 / n (the Frobenius-closest multiple of I to A^T A; equals
     the printed m/n when A A^T = I);
  R3 z0 = s0 = 1;
  R4 step to the boundary alpha = min(1, eta*min_{dz_i<0} -z_i/dz_i),
     eta = 0.995 (Algorithm asks for the largest alpha keeping z > 0, which is
     not attained);
  R5 separate primal and dual step lengths as in the Algorithm;
  R6 corrector: right-hand side from Eq. fzfs at the trial point with sigma3 and
     the trial point's mu; the matrix Theta and Z^-1 stay those of the current
     iterate; the combined direction is stepped from the current iterate;
  R7 termination on the relative duality gap  z^T s / (1 + |P(z)|) <= tol
     (Sec. 5.1 "Duality Gap", Sec. 5.4 "tol");
  R8 sigma = sigma2 on iterations k != 1 whose previous step had
     alpha_P <= alpha_bar or alpha_D <= alpha_bar, else sigma1;
  R19 multiple centrality correctors (the variant Sec. 5.1 describes as the original method
     and sets aside; the paper gives no formulas): after the predictor, up to mcc correctors
     with right-hand side (0, t), t the correction of the trial point's complementarity
     products toward [beta_min, beta_max] * sigma*mu, trial point at the aspiration steps
     alpha + delta, accepted while the smaller step grows by gamma * delta (beta_min 0.1,
     beta_max 10, delta 0.1, gamma 0.1).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Optional

import numpy as np
import scipy.fft
import scipy.linalg

# Paper parameters (Sec. 5.1, after the Algorithm; Sec. 5.4).
SIGMA1, SIGMA2, SIGMA3 = 0.1, 0.5, 0.8
ALPHA_BAR, ALPHA_TILDE = 0.5, 0.1
MAXITERS = 100
MXITERPCG = 200


# --------------------------------------------------------------------------------------
# Operators
# --------------------------------------------------------------------------------------
def dct_matrix_rows(n: int, rows) -> np.ndarray:
    """Rows of the orthonormal n x n DCT-II matrix, from its definition
    C[j,k] = alpha_j cos(pi j (2k+1) / (2n)), alpha_0 = sqrt(1/n), alpha_j = sqrt(2/n)
    (Sec. 2: partial DCT with orthonormal rows, Eq. eq:orthonormality)."""
    rows = np.asarray(rows, dtype=np.int64)
    j = rows[:, None].astype(np.float64)
    k = np.arange(n, dtype=np.float64)[None, :]
    alpha = np.where(rows == 0, math.sqrt(1.0 / n), math.sqrt(2.0 / n))[:, None]
    # (j*(2k+1)) mod 4n keeps the cosine argument small and exact in float64
    arg = np.mod(rows[:, None] * (2 * np.arange(n, dtype=np.int64)[None, :] + 1), 4 * n)
    return alpha * np.cos(np.pi * arg.astype(np.float64) / (2.0 * n))


def haar_matrix_rows(n: int, rows) -> np.ndarray:
    """Rows of the orthonormal n x n Haar matrix (n a power of two), from its definition:
    row 0 is the constant 1/sqrt(n); row 2^j + k (0 <= j < log2 n, 0 <= k < 2^j) is the
    wavelet of scale j and position k, +2^(j/2)/sqrt(n) on [k n/2^j, (k + 1/2) n/2^j) and
    -2^(j/2)/sqrt(n) on [(k + 1/2) n/2^j, (k + 1) n/2^j), zero elsewhere.  Sec. 2 names
    Haar wavelets among the orthonormal systems whose random rows form CS matrices with
    orthonormal rows (A A^T = I) and O(n) products."""
    rows = np.asarray(rows, dtype=np.int64)
    H = np.zeros((len(rows), n))
    for r, i in enumerate(rows):
        if i == 0:
            H[r, :] = 1.0 / math.sqrt(n)
            continue
        j = int(i).bit_length() - 1
        k = int(i) - (1 << j)
        w = n >> j                      # support length n / 2^j
        h = 2.0 ** (j / 2.0) / math.sqrt(n)
        H[r, k * w: k * w + w // 2] = h
        H[r, k * w + w // 2: (k + 1) * w] = -h
    return H


def dct_rows_apply(x: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """A x for the partial DCT via the library DCT (large-n certificates only)."""
    return scipy.fft.dct(np.asarray(x, dtype=np.float64), type=2, norm="ortho")[rows]


def dct_rows_apply_t(y: np.ndarray, rows: np.ndarray, n: int) -> np.ndarray:
    full = np.zeros(n)
    full[rows] = y
    return scipy.fft.idct(full, type=2, norm="ortho")


class Operator:
    """A as the two products x -> A x and y -> A^T y (Sec. 1: A used only as an operator)."""

    def __init__(self, m: int, n: int, mv: Callable, rmv: Callable, dense: Optional[np.ndarray] = None):
        self.m, self.n, self.mv, self.rmv, self.dense = m, n, mv, rmv, dense

    @staticmethod
    def from_dense(A: np.ndarray) -> "Operator":
        A = np.asarray(A, dtype=np.float64)
        return Operator(A.shape[0], A.shape[1], lambda x: A @ x, lambda y: A.T @ y, A)

    @staticmethod
    def from_haar_rows(n: int, rows) -> "Operator":
        return Operator.from_dense(haar_matrix_rows(n, rows))

    @staticmethod
    def from_dct_rows(n: int, rows, explicit: bool = True) -> "Operator":
        rows = np.asarray(rows, dtype=np.int64)
        if explicit:
            return Operator.from_dense(dct_matrix_rows(n, rows))
        return Operator(len(rows), n, lambda x: dct_rows_apply(x, rows),
                        lambda y: dct_rows_apply_t(y, rows, n))


# --------------------------------------------------------------------------------------
# Problem quantities (Sec. 1 and Sec. 3)
# --------------------------------------------------------------------------------------
def soft_threshold(y: np.ndarray, tau: float) -> np.ndarray:
    return np.sign(y) * np.maximum(np.abs(y) - tau, 0.0)


def objective(op: Operator, b, tau, x) -> float:
    """tau*||x||_1 + 1/2||Ax-b||^2 (reading R1)."""
    r = op.mv(x) - b
    return tau * float(np.abs(x).sum()) + 0.5 * float(r @ r)


def c_vector(op: Operator, b, tau) -> np.ndarray:
    """c = [tau*1 - A^T b; tau*1 + A^T b]  (Sec. 3, below Eq. dualquadraticBPDN)."""
    atb = op.rmv(b)
    return np.concatenate([tau - atb, tau + atb])


def FFt_apply(op: Operator, z: np.ndarray) -> np.ndarray:
    """F F^T z with F^T = [A, -A]  (Sec. 1, Eq. wrightBPDN; block form Eq. eq:ne2_H)."""
    n = op.n
    t = op.rmv(op.mv(z[:n] - z[n:]))
    return np.concatenate([t, -t])


def primal_value(op: Operator, b, tau, z) -> float:
    """P(z) = tau*1^T z + 1/2||F^T z - b||^2  (Eq. wrightBPDN)."""
    n = op.n
    r = op.mv(z[:n] - z[n:]) - b
    return tau * float(z.sum()) + 0.5 * float(r @ r)


def residuals(op: Operator, b, tau, z, s, c):
    """f_z = s - c - F F^T z and mu = z^T s / (2n)  (Sec. 3, Eq. fzfs)."""
    fz = s - c - FFt_apply(op, z)
    mu = float(z @ s) / z.size
    return fz, mu


def complementarity_rhs(z, s, sigma, mu):
    """f_s = sigma*mu*e - Z S e  (Eq. fzfs); it vanishes on the central path z o s = mu e
    when sigma = 1 (Sec. 4: the IPM perturbs z_j s_j = mu)."""
    return sigma * mu - z * s


def newton_rhs(fz, fs, z):
    """Right-hand side of the reduced Newton system  f_z + Z^-1 f_s  (Eq. redNewtonA)."""
    return fz + fs / z


def recover_ds(fs, z, d, dz):
    """ds = Z^-1 f_s - Theta^-1 dz,  Theta^-1 = Z^-1 S = d  (Eq. redNewtonB)."""
    return fs / z - d * dz


def centrality_target(v, mu_t, beta_min, beta_max):
    """Correction of the complementarity products v = z~ o s~ toward the box
    [beta_min mu_t, beta_max mu_t] around the target barrier mu_t (multiple centrality
    correctors, reading R19): t_i = beta_min mu_t - v_i below the box,
    max(beta_max mu_t - v_i, -beta_max mu_t) above it, 0 inside."""
    lo, hi = beta_min * mu_t, beta_max * mu_t
    t = np.zeros_like(v)
    below, above = v < lo, v > hi
    t[below] = lo - v[below]
    t[above] = np.maximum(hi - v[above], -hi)
    return t


def centrality_correctors(z, s, d, dz, ds, aP, aD, mu_t, p, solve, steps):
    """Up to p.mcc centrality correctors after the predictor (dz, ds) with steps (aP, aD)
    (reading R19).  Each takes the trial point of the current direction at the aspiration
    steps min(1, alpha + delta), the correction t of its complementarity products toward the
    box around mu_t, and solves the Newton system of Eq. sepregaugeq with right-hand side
    (f_z, f_s) = (0, t): (Theta^-1 + F F^T) dz~ = Z^-1 t, ds~ = Z^-1 t - Theta^-1 dz~
    (Eqs. redNewtonA/B).  The sum is kept when its smaller step grows by at least
    gamma * delta; the first rejected corrector ends the sequence.
    Returns (dz, ds, aP, aD, accepted)."""
    acc = 0
    for _ in range(p.mcc):
        if min(aP, aD) >= 1.0:
            break
        aPt, aDt = min(1.0, aP + p.mcc_delta), min(1.0, aD + p.mcc_delta)
        t = centrality_target((z + aPt * dz) * (s + aDt * ds), mu_t, p.mcc_beta_min, p.mcc_beta_max)
        dzc = solve(d, newton_rhs(np.zeros_like(t), t, z))
        dsc = recover_ds(t, z, d, dzc)
        aPn, aDn = steps(dz + dzc, ds + dsc)
        if min(aPn, aDn) < min(aP, aD) + p.mcc_gamma * p.mcc_delta:
            break
        dz, ds, aP, aD = dz + dzc, ds + dsc, aPn, aDn
        acc += 1
    return dz, ds, aP, aD, acc


def corrector_direction(op: "Operator", b, tau, c, z, s, d, zt, st, sigma3, solve):
    """The corrector of the Algorithm (Sec. 5.1), reading R6: the right-hand side of
    Eq. fzfs is evaluated at the trial point (zt, st) = (z + alpha_P dz, s + alpha_D ds) with
    sigma3 and the trial point's mu,
        f_z~ = st - c - F F^T zt,   f_s~ = sigma3 mu~ e - Zt St e,   mu~ = zt^T st / (2n),
    while the Newton matrix (through d = Theta^-1 = s / z) and the Z^-1 of Eqs.
    redNewtonA/B stay those of the current iterate (z, s).  Returns (dz~, ds~); the Algorithm adds them to
    the predictor and steps the sum from (z, s)."""
    fzt, mut = residuals(op, b, tau, zt, st, c)
    fst = complementarity_rhs(zt, st, sigma3, mut)
    dz2 = solve(d, newton_rhs(fzt, fst, z))
    ds2 = recover_ds(fst, z, d, dz2)
    return dz2, ds2


# --------------------------------------------------------------------------------------
# Exact solves of (Theta^-1 + F F^T) dz = r   (Sec. 5.7 direct variant)
# --------------------------------------------------------------------------------------
def newton_matrix(op: Operator, d: np.ndarray) -> np.ndarray:
    """H = Theta^-1 + F F^T as an explicit 2n x 2n matrix (Eq. eq:ne2_matrix / eq:ne2_H)."""
    A = op.dense
    K = A.T @ A
    H = np.block([[K, -K], [-K, K]])
    H[np.diag_indices_from(H)] += d
    return H


def solve_full_cholesky(op: Operator, d, r):
    H = newton_matrix(op, d)
    cf = scipy.linalg.cho_factor(H, lower=True, check_finite=False)
    return scipy.linalg.cho_solve(cf, r, check_finite=False)


def solve_woodbury(op: Operator, d, r):
    """(D + F F^T)^-1 r = D^-1 r - D^-1 F (I_m + F^T D^-1 F)^-1 F^T D^-1 r,
    F^T D^-1 F = A (Theta_u + Theta_v) A^T; Cholesky of the m x m matrix."""
    A = op.dense
    n = op.n
    theta = 1.0 / d
    th_sum = theta[:n] + theta[n:]
    M = (A * th_sum[None, :]) @ A.T
    M[np.diag_indices_from(M)] += 1.0
    Dr = theta * r
    t = A @ (Dr[:n] - Dr[n:])
    cf = scipy.linalg.cho_factor(M, lower=True, check_finite=False)
    y = scipy.linalg.cho_solve(cf, t, check_finite=False)
    aty = A.T @ y
    return Dr - theta * np.concatenate([aty, -aty])


def solve_newton_direct(op: Operator, d, r, method: str = "auto"):
    if method == "auto":
        method = "cholesky" if 2 * op.n <= 2048 else "woodbury"
    return solve_full_cholesky(op, d, r) if method == "cholesky" else solve_woodbury(op, d, r)


# --------------------------------------------------------------------------------------
# The paper's preconditioner and PCG (Sec. 4)
# --------------------------------------------------------------------------------------
def rho_of(op: Operator) -> float:
    """rho: the scalar of the Frobenius-closest rho*I to A^T A (reading R2):
    rho = ||A||_F^2 / n  (= m/n when A A^T = I, Eq. eq:ne2_P)."""
    if op.dense is not None:
        return float((op.dense ** 2).sum()) / op.n
    return op.m / op.n


def precond_matrix(d: np.ndarray, rho: float) -> np.ndarray:
    """P = [[Theta_u^-1 + rho I, -rho I], [-rho I, Theta_v^-1 + rho I]]  (Eq. eq:ne2_P)."""
    n = d.size // 2
    I = np.eye(n)
    return np.block([[np.diag(d[:n]) + rho * I, -rho * I], [-rho * I, np.diag(d[n:]) + rho * I]])


def precond_apply(d: np.ndarray, rho: float, r: np.ndarray) -> np.ndarray:
    """P^-1 r, one 2x2 block per index i (blocks [[du+rho, -rho], [-rho, dv+rho]])."""
    n = d.size // 2
    du, dv, ru, rv = d[:n], d[n:], r[:n], r[n:]
    det = (du + rho) * (dv + rho) - rho * rho
    return np.concatenate([((dv + rho) * ru + rho * rv) / det, (rho * ru + (du + rho) * rv) / det])


def H_apply(op: Operator, d, p):
    """H p = Theta^-1 p + F F^T p  (Eq. eq:ne2_matrix)."""
    return d * p + FFt_apply(op, p)


def pcg(op: Operator, d, rhs, rho, tol, maxiter=MXITERPCG):
    """Textbook preconditioned conjugate gradients on H dz = rhs from dz = 0 (Sec. 4).
    Stops when sqrt(r^T P^-1 r) <= tol * sqrt(rhs^T P^-1 rhs).  Breakdown guard (the paper
    does not say what PCG does when rounding destroys positive definiteness, which happens
    when Theta^-1 spans ~30 orders of magnitude): a search direction with p^T H p not
    positive and finite, or a step alpha that is not finite, ends the solve with the last
    iterate.  Returns (dz, iterations)."""
    x = np.zeros_like(rhs)
    r = rhs.copy()
    zz = precond_apply(d, rho, r)
    p = zz.copy()
    rz = float(r @ zz)
    rz0 = rz
    it = 0
    while it < maxiter and rz > tol * tol * rz0:
        q = H_apply(op, d, p)
        pq = float(p @ q)
        if not (pq > 0.0 and math.isfinite(pq) and math.isfinite(rz / pq)):
            break
        alpha = rz / pq
        x += alpha * p
        r -= alpha * q
        zz = precond_apply(d, rho, r)
        rz_new = float(r @ zz)
        p = zz + (rz_new / rz) * p
        rz = rz_new
        it += 1
    return x, it


# --------------------------------------------------------------------------------------
# Step lengths and the IPM (Sec. 5.1)
# --------------------------------------------------------------------------------------
def step_to_boundary(v: np.ndarray, dv: np.ndarray, eta: float) -> float:
    """alpha = min(1, eta * min_{dv_i < 0} (-v_i / dv_i)); 1 if no component decreases (R4)."""
    neg = dv < 0
    if not neg.any():
        return 1.0
    return min(1.0, eta * float(np.min(-v[neg] / dv[neg])))


@dataclasses.dataclass
class OracleParams:
    tol: float = 1e-12
    max_iter: int = MAXITERS
    sigma1: float = SIGMA1
    sigma2: float = SIGMA2
    sigma3: float = SIGMA3
    alpha_bar: float = ALPHA_BAR
    alpha_tilde: float = ALPHA_TILDE
    eta: float = 0.995
    equal_steps: bool = False
    solver: str = "auto"        # "auto" | "cholesky" | "woodbury" | "pcg"
    tol_pcg: float = 1e-2       # only for solver="pcg"
    # multiple centrality correctors (the method Sec. 5.1 starts from; reading R19): up to mcc
    # correctors per iteration in place of the single conditional one; 0 = the Algorithm
    mcc: int = 0
    mcc_beta_min: float = 0.1
    mcc_beta_max: float = 10.0
    mcc_delta: float = 0.1      # aspiration: trial steps alpha + delta
    mcc_gamma: float = 0.1      # acceptance: min step grows by at least gamma * delta


@dataclasses.dataclass
class OracleResult:
    x: np.ndarray
    z: np.ndarray
    s: np.ndarray
    iters: int
    correctors: int
    pcg_iters: int
    rel_gap: float
    dual_res: float
    converged: bool
    history: list


def ipm(op: Operator, b, tau, params: Optional[OracleParams] = None) -> OracleResult:
    """Single-corrector primal-dual IPM (Sec. 5.1, Algorithm) with the Newton systems of
    Eq. redNewton solved exactly (Sec. 5.7), in float64."""
    p = params or OracleParams()
    n = op.n
    N2 = 2 * n
    c = c_vector(op, b, tau)
    cnorm = float(np.linalg.norm(c))
    rho = rho_of(op)
    z = np.ones(N2)                       # R3
    s = np.ones(N2)
    aP_prev = aD_prev = 1.0
    corr = 0
    pcg_total = 0
    hist = []

    def solve(d, r):
        nonlocal pcg_total
        if p.solver == "pcg":
            dz, it = pcg(op, d, r, rho, p.tol_pcg)
            pcg_total += it
            return dz
        return solve_newton_direct(op, d, r, p.solver)

    def steps(dz, ds):
        aP = step_to_boundary(z, dz, p.eta)
        aD = step_to_boundary(s, ds, p.eta)
        if p.equal_steps:
            aP = aD = min(aP, aD)
        return aP, aD

    converged = False
    k = 0
    rel_gap = dual_res = float("inf")
    for k in range(1, p.max_iter + 1):
        fz, mu = residuals(op, b, tau, z, s, c)
        P = primal_value(op, b, tau, z)
        rel_gap = float(z @ s) / (1.0 + abs(P))
        dual_res = float(np.linalg.norm(fz)) / (1.0 + cnorm)
        hist.append(dict(k=k, mu=mu, rel_gap=rel_gap, dual_res=dual_res, alpha_p=aP_prev, alpha_d=aD_prev))
        if rel_gap <= p.tol:                                                     # R7
            converged = True
            break
        if k != 1 and (aP_prev <= p.alpha_bar or aD_prev <= p.alpha_bar):        # R8
            sigma = p.sigma2
        else:
            sigma = p.sigma1
        # predictor
        fs = complementarity_rhs(z, s, sigma, mu)
        d = s / z
        dz = solve(d, newton_rhs(fz, fs, z))
        ds = recover_ds(fs, z, d, dz)
        aP, aD = steps(dz, ds)
        if p.mcc > 0:                                                            # R19
            dz, ds, aP, aD, acc = centrality_correctors(z, s, d, dz, ds, aP, aD, sigma * mu, p, solve, steps)
            corr += acc
        # corrector (R6)
        elif aP <= p.alpha_tilde or aD <= p.alpha_tilde:
            corr += 1
            dz2, ds2 = corrector_direction(op, b, tau, c, z, s, d, z + aP * dz, s + aD * ds, p.sigma3, solve)
            dz = dz + dz2
            ds = ds + ds2
            aP, aD = steps(dz, ds)
        z = z + aP * dz
        s = s + aD * ds
        aP_prev, aD_prev = aP, aD
    else:
        k = p.max_iter
    x = z[:n] - z[n:]
    return OracleResult(x, z, s, k, corr, pcg_total, rel_gap, dual_res, converged, hist)


# --------------------------------------------------------------------------------------
# Certificates
# --------------------------------------------------------------------------------------
def gradient(op: Operator, b, x):
    """g(x) = A^T (A x - b)."""
    return op.rmv(op.mv(x) - b)


def kkt_rel(op: Operator, b, tau, x) -> float:
    """||x - S_tau(x - g(x))||_2 / (1 + ||x||_2): zero exactly at the minimiser."""
    g = gradient(op, b, x)
    return float(np.linalg.norm(x - soft_threshold(x - g, tau))) / (1.0 + float(np.linalg.norm(x)))


def optimality_violation(op: Operator, b, tau, x, support_tol: float):
    """Largest violation of the l1 optimality conditions: g_i = -tau*sign(x_i) where
    |x_i| > support_tol, |g_i| <= tau elsewhere.  Returns (on-support, off-support)."""
    g = gradient(op, b, x)
    on = np.abs(x) > support_tol
    v_on = float(np.max(np.abs(g[on] + tau * np.sign(x[on])))) if on.any() else 0.0
    v_off = float(np.max(np.maximum(np.abs(g[~on]) - tau, 0.0))) if (~on).any() else 0.0
    return v_on, v_off


def dual_point(op: Operator, b, tau, x):
    """A dual-feasible point of the l1 problem built from x (the construction of the l1_ls
    method the paper cites in Sec. 1): the residual r = A x - b scaled into the dual
    feasible set {nu : ||A^T nu||_inf <= tau},  nu = r * min(1, tau / ||A^T r||_inf)."""
    r = op.mv(x) - b
    gi = float(np.abs(op.rmv(r)).max()) if r.size else 0.0
    return r * (min(1.0, tau / gi) if gi > 0 else 1.0)


def dual_gap_certificate(op: Operator, b, tau, x):
    """Duality gap of the l1 problem at the dual-feasible point nu = dual_point(x):
    D(nu) = -1/2||nu||^2 - b^T nu is a lower bound on P* (weak duality), so
    0 <= P(x) - P* <= P(x) - D(nu).  Returns (P(x), D(nu))."""
    r = op.mv(x) - b
    nu = dual_point(op, b, tau, x)
    P = tau * float(np.abs(x).sum()) + 0.5 * float(r @ r)
    D = -0.5 * float(nu @ nu) - float(b @ nu)
    return P, D


# --------------------------------------------------------------------------------------
# Derivatives of the solution map (b, tau, A) -> x*  (the paper has none; they follow from
# differentiating the perturbed KKT conditions of Eq. fzfs at fixed mu)
# --------------------------------------------------------------------------------------
def adjoint_kkt(op: Operator, b, tau, z, s, grad_x):
    """Reverse-mode derivative at an interior iterate (z, s): with
    H = Theta^-1 + F F^T (Eq. eq:ne2_matrix) and J = [I; -I], dz = -H^-1 dc - H^-1 dQ z,
    so for L with dL/dx = grad_x:  y = H^-1 J grad_x,  w = J^T y,
      dL/db = A w,   dL/dtau = -1^T y,   dL/dA = r w^T - (A w) x^T,  r = b - A x.
    H y = J grad_x is solved exactly by eliminating y_u + y_v (the reduction behind Theorem
    thm:ne2_prec): ((Theta_u + Theta_v)^-1 + A^T A) w = grad_x, then
    y_u = d_v w / (d_u + d_v), y_v = -d_u w / (d_u + d_v) with d = Theta^-1 = s/z.  Near the
    solution Theta spans ~1e+-12 and this n x n system stays well conditioned where the
    m x m Woodbury matrix I + A (Theta_u + Theta_v) A^T does not.
    Returns (grad_b, grad_tau, grad_A or None)."""
    n = op.n
    d = s / z
    du, dv = d[:n], d[n:]
    A = op.dense
    K = A.T @ A
    K[np.diag_indices_from(K)] += du * dv / (du + dv)
    cf = scipy.linalg.cho_factor(K, lower=True, check_finite=False)
    w = scipy.linalg.cho_solve(cf, grad_x, check_finite=False)
    y_u = dv * w / (du + dv)
    y_v = -du * w / (du + dv)
    aw = op.mv(w)
    grad_tau = -float(np.sum(y_u + y_v))
    grad_A = None
    if op.dense is not None:
        x = z[:n] - z[n:]
        r = b - op.mv(x)
        grad_A = np.outer(r, w) - np.outer(aw, x)
    return aw, grad_tau, grad_A


def adjoint_support(A: np.ndarray, b, tau, x, grad_x, support_tol: float = 1e-7):
    """The same derivatives from the closed form on the support S of x* (valid under strict
    complementarity): x_S = (A_S^T A_S)^-1 (A_S^T b - tau sign(x_S)), x = 0 off S, so with
    w_S = (A_S^T A_S)^-1 grad_x_S (w = 0 off S):  dL/db = A w,
    dL/dtau = -sign(x_S)^T w_S,  dL/dA = r w^T - (A w) x^T."""
    S = np.abs(x) > support_tol
    AS = A[:, S]
    wS = np.linalg.solve(AS.T @ AS, grad_x[S])
    w = np.zeros_like(x)
    w[S] = wS
    aw = A @ w
    r = b - A @ x
    return aw, -float(np.sign(x[S]) @ wS), np.outer(r, w) - np.outer(aw, x)
