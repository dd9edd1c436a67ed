"""The phase-transition workload (Sec. 5.8) on the CPU: its generator, and two facts about l1
recovery that pin the oracle on it.  Below the mutual-coherence bound k < (1 + 1/mu)/2 the
k-sparse signal is the unique basis-pursuit solution (Donoho and Elad's coherence theorem), so
with the workload's tiny tau the minimiser lies within the 1e-5 success radius of x_hat; with
k = m random +-1 spikes and m < n the signal is not the l1 minimiser and the solve fails the
radius by far."""
import numpy as np
import pytest
import scipy.fft

import workloads as W
from oracle import mfipm_oracle as O

N = W.WORKLOADS["phase_transition_1024"]["n"]


def test_grid_and_problems():
    cells = W.phase_cells()
    assert len(cells) == 4500
    assert [m for m in range(100, 901, 100)] == sorted({m for m, _ in cells})
    assert all(1 <= k <= m for m, k in cells)
    probs = W.make_workload("phase_transition_1024", count=120)
    for (m, k), p in zip(cells, probs):
        assert (p.m, p.n) == (m, N) and np.count_nonzero(p.x_hat) == k
        assert set(np.unique(p.x_hat[p.x_hat != 0])) <= {-1.0, 1.0}
        assert np.all(np.diff(p.rows) > 0) and p.rows[-1] < N
        # noiseless: b is exactly A x_hat
        assert np.allclose(W.dct_apply(p.x_hat, p.rows), p.b, rtol=0, atol=1e-12)
        assert p.tau == pytest.approx(1e-6 * np.abs(W.dct_apply_t(p.b, p.rows, N)).max())
    # trials are independent draws of the same cells
    t1 = W.make_workload("phase_transition_1024", count=3, offset=1)
    assert not np.array_equal(t1[2].rows, probs[2].rows)


def coherence(rows):
    """Largest |cosine| between two distinct columns of the partial DCT."""
    A = scipy.fft.dct(np.eye(N), type=2, norm="ortho", axis=0)[rows]
    A = A / np.linalg.norm(A, axis=0)
    G = np.abs(A.T @ A)
    np.fill_diagonal(G, 0.0)
    return float(G.max())


def _re(p, x):
    return float(np.linalg.norm(x - p.x_hat) / np.linalg.norm(p.x_hat))


@pytest.mark.parametrize("m", [400, 900])
def test_recovery_below_the_coherence_bound(m):
    """The cell (m, k) with the largest k under the coherence bound of its own rows."""
    cells = W.phase_cells()
    k = 1
    while True:  # the bound depends on the rows, which depend on the cell's random stream
        p = W.make_workload("phase_transition_1024", count=cells.index((m, k)) + 1)[-1]
        bound = (1 + 1 / coherence(p.rows)) / 2
        if k + 1 >= bound:
            break
        k += 1
    assert k < bound
    res = O.ipm(O.Operator.from_dct_rows(p.n, p.rows), p.b, p.tau, O.OracleParams(tol=1e-10))
    assert _re(p, res.x) <= 1e-5


def test_no_recovery_at_k_equal_m():
    cells = W.phase_cells()
    probs = W.make_workload("phase_transition_1024", count=cells.index((100, 100)) + 1)
    p = probs[-1]
    res = O.ipm(O.Operator.from_dct_rows(p.n, p.rows), p.b, p.tau, O.OracleParams(tol=1e-10))
    assert _re(p, res.x) > 1e-2
