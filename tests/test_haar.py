"""Pins of the oracle's partial-Haar operator (orthonormal Haar matrix rows, Sec. 2) and of
the Haar workload generator, each against something other than the oracle itself."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import mfipm_oracle as O


def pyramid(x):
    """Haar analysis written out here: repeated pairwise (sum, difference) / sqrt(2) of the
    running averages; coefficients ordered scaling, then scale 0, 1, ... (coarse to fine)."""
    levels = []
    a = list(map(float, x))
    while len(a) > 1:
        s = [(a[2 * i] + a[2 * i + 1]) / math.sqrt(2) for i in range(len(a) // 2)]
        d = [(a[2 * i] - a[2 * i + 1]) / math.sqrt(2) for i in range(len(a) // 2)]
        levels.append(d)
        a = s
    out = a
    for d in reversed(levels):
        out = out + d
    return np.array(out)


@pytest.mark.parametrize("n", [2, 8, 64, 1024])
def test_orthonormal_rows(n):
    H = O.haar_matrix_rows(n, np.arange(n))
    assert np.abs(H @ H.T - np.eye(n)).max() < 1e-13


def test_closed_forms():
    n = 256
    H = O.haar_matrix_rows(n, np.arange(n))
    # a constant signal has only the scaling coefficient sqrt(n)
    c = H @ np.ones(n)
    assert c[0] == pytest.approx(math.sqrt(n)) and np.abs(c[1:]).max() < 1e-12
    # a unit impulse at 0: the first column, 2^(j/2)/sqrt(n) at position k = 0 of every scale
    e = H[:, 0]
    want = np.zeros(n)
    want[0] = 1 / math.sqrt(n)
    for j in range(8):
        want[1 << j] = 2 ** (j / 2) / math.sqrt(n)
    assert np.abs(e - want).max() < 1e-14


@pytest.mark.parametrize("n", [4, 32, 512])
def test_pyramid_equals_matrix(n):
    x = np.random.default_rng(n).standard_normal(n)
    H = O.haar_matrix_rows(n, np.arange(n))
    assert np.abs(H @ x - pyramid(x)).max() < 1e-12
    assert np.abs(W.haar_apply(x) - pyramid(x)).max() < 1e-12


def test_square_haar_problem_is_soft_thresholding():
    """m = n: A orthonormal and square, so the minimiser is S_tau(A^T b)."""
    n = 64
    rng = np.random.default_rng(5)
    H = O.haar_matrix_rows(n, np.arange(n))
    b = rng.standard_normal(n)
    tau = 0.3 * np.abs(H.T @ b).max()
    res = O.ipm(O.Operator.from_haar_rows(n, np.arange(n)), b, tau)
    assert np.abs(res.x - O.soft_threshold(H.T @ b, tau)).max() < 1e-8


def test_haar_problem_generator():
    p = W.haar_problem(1024, 256, 10, 7, 3, sigma=0.0)
    assert p.kind == "haar" and p.m == 256 and np.all(np.diff(p.rows) > 0)
    H = O.haar_matrix_rows(p.n, p.rows)
    assert np.abs(H @ p.x_hat - p.b).max() < 1e-12
    assert p.tau == pytest.approx(0.01 * np.abs(H.T @ p.b).max())


def _mutant(kind):
    """haar_matrix_rows with one plausible mistake planted."""
    def rows_fn(n, rows):
        H = np.zeros((len(rows), n))
        for r, i in enumerate(rows):
            if i == 0:
                H[r, :] = 1.0 / math.sqrt(n)
                continue
            j = int(i).bit_length() - 1
            k = int(i) - (1 << j)
            if kind == "position" and j > 0:
                k = (k + 1) % (1 << j)
            w = n >> j
            h = (2.0 ** j if kind == "scale" else 2.0 ** (j / 2.0)) / math.sqrt(n)
            sgn = -1.0 if (kind == "sign" and j == 2) else 1.0
            H[r, k * w: k * w + w // 2] = sgn * h
            H[r, k * w + w // 2: (k + 1) * w] = -sgn * h
        return H
    return rows_fn


@pytest.mark.parametrize("kind", ["scale", "sign", "position"])
def test_pins_catch_planted_mistakes(kind, monkeypatch):
    """Each planted mistake in the Haar rows fails at least one of the pins above."""
    monkeypatch.setattr(O, "haar_matrix_rows", _mutant(kind))
    caught = 0
    for pin in (lambda: test_orthonormal_rows(64), test_closed_forms, lambda: test_pyramid_equals_matrix(32)):
        try:
            pin()
        except AssertionError:
            caught += 1
    assert caught >= 1, kind
