"""Seeded synthetic inputs for the l1-regularised least-squares problems.

This module only draws random problem data; it contains none of the solver's
arithmetic.  Both the CPU oracle (``oracle/``) and the CUDA path (tests,
``bench.py``) take their inputs from here, so the two sides always see the
same problems.

Problem:  min_x  tau*||x||_1 + 1/2*||A x - b||_2^2            (Sec. 1, Eq. formulationsnoisy1;
                                                              the 1/2 form of Eq. wrightBPDN)
with b = A x_hat + e,  e_i ~ N(0, sigma^2)                    (Eq. incomplsysnoisy)

Operators:
  * dense Gaussian ensemble, i.i.d. N(0, 1/m) entries         (Sec. 2, Table tbl:RIP; Table sparcocollect "gausspike")
  * partial orthonormal DCT-II: m distinct rows of the n x n orthonormal DCT-II matrix,
    chosen uniformly without replacement and sorted           (Sec. 2, Eq. eq:orthonormality; Sec. 5.8)
  * the dense ensemble quantised to bf16 with one per-tensor scale: the problem's matrix is
    exactly  a_scale * bf16(A / a_scale)

The named workloads mirror the benchmark configurations of this project
(sizes in the docstrings of ``WORKLOADS``).  Random streams: numpy PCG64 seeded
with the SeedSequence ``[seed, j]`` for problem ``j`` of a workload.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
import scipy.fft

__all__ = [
    "Problem", "dense_problem", "dct_problem", "bf16_dense_problems", "WORKLOADS",
    "make_workload", "bf16_round", "dct_apply", "dct_apply_t", "phase_cells", "phase_problems",
    "scaling_problems", "haar_apply", "haar_apply_t", "haar_problem",
]


@dataclasses.dataclass
class Problem:
    """One seeded l1-LS instance.  ``A`` (dense, row-major m x n float64) or
    ``rows`` (partial DCT, sorted int64 row indices) describes the operator."""
    kind: str                      # "dense" | "dct" | "haar"
    m: int
    n: int
    b: np.ndarray                  # (m,) float64
    tau: float
    x_hat: np.ndarray              # (n,) float64, the sparse signal b was made from
    A: Optional[np.ndarray] = None     # dense: (m, n) float64 (already the exact problem matrix)
    rows: Optional[np.ndarray] = None  # dct, haar: (m,) int64 ascending
    a_bf16: Optional[np.ndarray] = None  # bf16-quantised dense: (m, n) uint16 bit patterns
    a_scale: float = 1.0
    seed: tuple = ()


def _rng(seed: int, j: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(j)])))


def dct_apply(x: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """A x for the partial orthonormal DCT-II (library DCT; used only to synthesise b)."""
    return scipy.fft.dct(x, type=2, norm="ortho")[rows]


def dct_apply_t(y: np.ndarray, rows: np.ndarray, n: int) -> np.ndarray:
    """A^T y for the partial orthonormal DCT-II (library inverse DCT)."""
    full = np.zeros(n)
    full[rows] = y
    return scipy.fft.idct(full, type=2, norm="ortho")


def _sparse_signal(rng, n, k, values):
    x = np.zeros(n)
    pos = rng.choice(n, size=k, replace=False)
    if values == "pm1":
        x[pos] = rng.choice(np.array([-1.0, 1.0]), size=k)
    else:
        x[pos] = rng.standard_normal(k)
    return x


def dense_problem(m: int, n: int, k: int, seed: int, j: int = 0, sigma: float = 1e-3,
                  tau_frac: float = 0.01, values: str = "pm1") -> Problem:
    """Gaussian A with N(0,1/m) entries, k-sparse x_hat (+-1 or N(0,1) values at uniform
    positions), b = A x_hat + N(0, sigma^2), tau = tau_frac*||A^T b||_inf."""
    rng = _rng(seed, j)
    A = rng.standard_normal((m, n)) / np.sqrt(m)
    x_hat = _sparse_signal(rng, n, k, values)
    b = A @ x_hat + sigma * rng.standard_normal(m)
    tau = tau_frac * float(np.abs(A.T @ b).max())
    return Problem("dense", m, n, b, tau, x_hat, A=A, seed=(seed, j))


def dct_problem(n: int, m: int, k: int, seed: int, j: int = 0, sigma: float = 1e-3,
                tau_frac: float = 0.01, values: str = "normal") -> Problem:
    """Partial orthonormal DCT-II with m of n rows (uniform, without replacement, sorted)."""
    rng = _rng(seed, j)
    rows = np.sort(rng.choice(n, size=m, replace=False)).astype(np.int64)
    x_hat = _sparse_signal(rng, n, k, values)
    b = dct_apply(x_hat, rows) + sigma * rng.standard_normal(m)
    tau = tau_frac * float(np.abs(dct_apply_t(b, rows, n)).max())
    return Problem("dct", m, n, b, tau, x_hat, rows=rows, seed=(seed, j))


def haar_apply(x: np.ndarray) -> np.ndarray:
    """Orthonormal Haar coefficients of x (n a power of two), in the order: scaling
    coefficient, then scale j = 0, 1, ... with positions k = 0 .. 2^j - 1 (index 2^j + k).
    Pyramid of pairwise sums and differences / sqrt(2); used only to synthesise b."""
    a = np.asarray(x, dtype=np.float64).copy()
    details = []
    while a.size > 1:
        even, odd = a[0::2], a[1::2]
        details.append((even - odd) / np.sqrt(2.0))
        a = (even + odd) / np.sqrt(2.0)
    return np.concatenate([a] + details[::-1])


def haar_problem(n: int, m: int, k: int, seed: int, j: int = 0, sigma: float = 1e-3,
                 tau_frac: float = 0.01, values: str = "normal") -> Problem:
    """m random rows of the orthonormal n x n Haar matrix (uniform without replacement,
    sorted), k-sparse x_hat, b = A x_hat + N(0, sigma^2), tau = tau_frac ||A^T b||_inf."""
    rng = _rng(seed, j)
    rows = np.sort(rng.choice(n, size=m, replace=False)).astype(np.int64)
    x_hat = _sparse_signal(rng, n, k, values)
    b = haar_apply(x_hat)[rows] + sigma * rng.standard_normal(m)
    # A^T b: coefficients b at the sampled rows, inverse transform
    full = np.zeros(n)
    full[rows] = b
    atb = haar_apply_t(full)
    tau = tau_frac * float(np.abs(atb).max())
    return Problem("haar", m, n, b, tau, x_hat, rows=rows, seed=(seed, j))


def haar_apply_t(c: np.ndarray) -> np.ndarray:
    """Inverse of haar_apply (the synthesis pyramid; the orthonormal Haar matrix transposed)."""
    a = c[:1].copy()
    pos = 1
    while pos < c.size:
        d = c[pos: 2 * pos]
        out = np.empty(2 * pos)
        out[0::2] = (a + d) / np.sqrt(2.0)
        out[1::2] = (a - d) / np.sqrt(2.0)
        a = out
        pos *= 2
    return a


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float64 -> bfloat16 (round to nearest even) and return the uint16 bit patterns."""
    f = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    lsb = (f >> 16) & 1
    rounded = (f + 0x7FFF + lsb) >> 16
    return rounded.astype(np.uint16)


def bf16_to_f64(bits: np.ndarray) -> np.ndarray:
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def bf16_dense_problems(m: int, n: int, k: int, nrhs: int, seed: int, sigma: float = 1e-3,
                        tau_frac: float = 0.01, first: int = 0):
    """One shared Gaussian A stored as bf16 with a per-tensor scale (a_scale = 1/sqrt(m)),
    and ``nrhs`` right-hand sides from k-sparse +-1 signals.  The problem matrix is exactly
    a_scale * bf16(A/a_scale); b and tau are computed with that exact matrix."""
    rng = _rng(seed, 0)
    a_scale = 1.0 / np.sqrt(m)
    bits = bf16_round(rng.standard_normal((m, n)))
    A = a_scale * bf16_to_f64(bits)
    probs = []
    for j in range(first, first + nrhs):
        r = _rng(seed, 1 + j)
        x_hat = _sparse_signal(r, n, k, "pm1")
        b = A @ x_hat + sigma * r.standard_normal(m)
        tau = tau_frac * float(np.abs(A.T @ b).max())
        probs.append(Problem("dense", m, n, b, tau, x_hat, A=A, a_bf16=bits, a_scale=a_scale,
                             seed=(seed, j)))
    return probs


# The five benchmark workloads (sizes and distributions of this project's configurations).
WORKLOADS = {
    # Gaussian 256 x 1024 (the shape of Sparco "gausspike", Table sparcocollect), k=20 +-1 spikes
    "dense_fp64_256x1024": dict(kind="dense", m=256, n=1024, k=20, values="pm1", seed=1001, count=1),
    # partial DCT n=65536, m=16384, k=655 N(0,1) values
    "dct_65536": dict(kind="dct", n=65536, m=16384, k=655, values="normal", seed=1002, count=1),
    # 256 partial-DCT problems, n uniform in {2^12..2^16}, m=n/4, k uniform in [n/100, n/20]
    "dct_batch_256": dict(kind="dct_batch", count=256, seed=1003),
    # shared bf16 Gaussian 4096 x 16384, 64 right-hand sides, k=164 +-1 spikes
    "bf16_4096x16384_64rhs": dict(kind="bf16", m=4096, n=16384, k=164, nrhs=64, seed=1004),
    # 32 partial-DCT problems n=2^20, m=2^18, k=n/100 N(0,1)
    "dct_adjoint_32x1M": dict(kind="dct", n=1 << 20, m=1 << 18, k=(1 << 20) // 100, values="normal",
                              seed=1005, count=32),
    # the empirical phase transition of Sec. 5.8: noiseless partial DCT of the paper's n = 1000
    # (the mixed-radix chain: n/2 = 2^2 5^3), m = 100..900 step 100, k = 1..m step 1, +-1
    # spikes; one problem per (m, k) cell per trial (4500 per trial), tau = 1e-6
    # ||A^T b||_inf (the paper states no tau for this experiment; see phase_problems); solver
    # tolerance 1e-12: with objectives near tau ||x_hat||_1 ~ 1e-5, a relative gap of 1e-10
    # against 1 + |P| leaves x errors close to the 1e-5 success radius
    "phase_transition_1000": dict(kind="phase", n=1000, seed=1006, trials=100, tau_frac=1e-6, tol=1e-12),
    # the same grid at n = 1024 (the power-of-two chain of the persistent kernel's clusters)
    "phase_transition_1024": dict(kind="phase", n=1024, seed=1006, trials=100, tau_frac=1e-6, tol=1e-12),
    # the uneven batch of dct_batch_256 (same sizes and spikes) on partial Haar rows (Sec. 2)
    "haar_batch_256": dict(kind="haar_batch", count=256, seed=1003),
    # PCG against a direct solver (Sec. 5.7): Gaussian A, n = 2^5..2^12, m = n/4, k = ceil(m/20)
    # N(0,1) values, noiseless b, tau = 1e-3; one problem per size
    "pcg_vs_direct": dict(kind="scaling", seed=1007, log2n=(5, 12), tau=1e-3),
}


def scaling_problems(seed: int, log2n=(5, 12), tau: float = 1e-3, trial: int = 0):
    """One Gaussian problem per n = 2^e (e in log2n, inclusive): A ~ N(0, 1/m), m = n/4,
    k = ceil(m/20) N(0,1) spikes, b = A x_hat exactly, tau fixed.  Problem e of trial t draws
    from the stream [seed, 100 t + e]."""
    out = []
    for e in range(log2n[0], log2n[1] + 1):
        n = 1 << e
        m = n // 4
        k = -(-m // 20)
        p = dense_problem(m, n, k, seed, 100 * trial + e, sigma=0.0, values="normal")
        out.append(dataclasses.replace(p, tau=float(tau)))
    return out


def phase_cells():
    """(m, k) of every cell of the phase-transition grid, m-major."""
    return [(m, k) for m in range(100, 901, 100) for k in range(1, m + 1)]


def phase_problems(n: int, seed: int, trial: int, tau_frac: float, count: Optional[int] = None):
    """Trial ``trial`` of every phase-transition cell: m random rows of the orthonormal n-point
    DCT-II, k-sparse +-1 x_hat at random positions, b = A x_hat exactly (no noise).  Problem j
    of trial t draws from the stream [seed, t * 4500 + j]."""
    cells = phase_cells()[: count or None]
    base = trial * len(phase_cells())
    return [dct_problem(n, m, k, seed, base + j, sigma=0.0, tau_frac=tau_frac, values="pm1")
            for j, (m, k) in enumerate(cells)]


def batch_sizes(count: int, seed: int):
    """(n, m, k) for each problem of the uneven partial-DCT batch."""
    rng = _rng(seed, 10**6)
    ns = rng.choice(np.array([4096, 8192, 16384, 32768, 65536]), size=count)
    out = []
    for n in ns:
        n = int(n)
        k = int(rng.integers(n // 100, n // 20 + 1))
        out.append((n, n // 4, k))
    return out


def make_workload(name: str, count: Optional[int] = None, scale_n: Optional[int] = None, offset: int = 0):
    """Return the list of Problems of a named workload.  ``count`` truncates the batch;
    ``scale_n`` (DCT only) replaces n by a smaller power of two with the same m/n and k/n
    ratios, for oracle-sized cases.  ``offset`` shifts the random stream of every problem
    (sizes, and the shared bf16 matrix, stay those of the workload): another shard of the
    same workload for another GPU."""
    w = WORKLOADS[name]
    if w["kind"] == "dense":
        return [dense_problem(w["m"], w["n"], w["k"], w["seed"], offset + j, values=w["values"])
                for j in range(count or w["count"])]
    if w["kind"] == "dct":
        n, m, k = w["n"], w["m"], w["k"]
        if scale_n:
            m = m * scale_n // n
            k = max(1, k * scale_n // n)
            n = scale_n
        return [dct_problem(n, m, k, w["seed"], offset + j, values=w["values"]) for j in range(count or w["count"])]
    if w["kind"] == "dct_batch":
        sizes = batch_sizes(w["count"], w["seed"])[: (count or w["count"])]
        return [dct_problem(n, m, k, w["seed"], offset + j) for j, (n, m, k) in enumerate(sizes)]
    if w["kind"] == "haar_batch":
        sizes = batch_sizes(w["count"], w["seed"])[: (count or w["count"])]
        return [haar_problem(n, m, k, w["seed"], offset + j) for j, (n, m, k) in enumerate(sizes)]
    if w["kind"] == "bf16":
        return bf16_dense_problems(w["m"], w["n"], w["k"], count or w["nrhs"], w["seed"], first=offset)
    if w["kind"] == "scaling":
        return scaling_problems(w["seed"], w["log2n"], w["tau"], offset)[: count or None]
    if w["kind"] == "phase":
        # offset selects the trial (another GPU's shard is another set of trials)
        return phase_problems(w["n"], w["seed"], offset, w["tau_frac"], count)
    raise KeyError(name)
