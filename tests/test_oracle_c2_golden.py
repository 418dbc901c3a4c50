"""The stored exhaustive oracle result of the d = 3 headline workload
(n = 1000, m = 1000: all 166,167,000 tuples fitted, Sec. 2.4) against cheap
independent checks: its SSEs re-computed tuple by tuple, LAPACK least squares
on a few rows, the order, and the planted descriptor first."""

import numpy as np

import oracle
from c2_golden import load
from workloads import make_config


def test_c2_golden_consistent():
    prob, d, k = make_config("C2")
    t, sse, rmse = load()
    assert t.shape == (128, 3)
    assert np.all(t[:, 0] < t[:, 1]) and np.all(t[:, 1] < t[:, 2])
    assert len({tuple(r) for r in t.tolist()}) == 128
    assert tuple(t[0]) == tuple(sorted(prob.planted[0]))
    # ascending by (SSE, lexicographic)
    keys = list(zip(sse.tolist(), [tuple(r) for r in t.tolist()]))
    assert keys == sorted(keys)
    got, rho = oracle.score(prob.X, prob.y, t)
    np.testing.assert_allclose(got[:, 0], sse, rtol=1e-13)
    np.testing.assert_allclose(rmse, np.sqrt(sse / prob.n_total), rtol=1e-15)
    assert np.all(rho[:, 0] >= oracle.RHO_MIN)
    for r in (0, 1, 57, 99, 127):
        A = np.column_stack([np.ones(prob.n_total)] + [prob.X[j] for j in t[r]])
        beta, *_ = np.linalg.lstsq(A, prob.y, rcond=None)
        res = prob.y - A @ beta
        assert abs(float(res @ res) - sse[r]) <= 1e-9 * sse[r]
