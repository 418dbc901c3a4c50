"""GPU parity of the SHARED multi-task mode (one descriptor for all tasks,
ranked by the pooled mean SSE sum_t SSE_t / N; ineligible when rank
deficient in any task) against the CPU oracle, in both precisions."""

import math

import numpy as np
import pytest

import oracle
import paper_2502_20072_gb300 as l0
from l0_testutil import RMSE_RTOL, TIE_GAP
from workloads import make_problem

pytestmark = pytest.mark.gpu


def _check_shared(prob, d, k, precision):
    ref = oracle.fit(prob.X, prob.y, d, k, offsets=prob.offsets, mode=oracle.SHARED)
    with l0.Handle(precision=precision, task_mode=l0.SHARED) as h:
        t, r = h.fit(prob.X, prob.y, d, k, offsets=prob.offsets)
        st = h.stats()
    assert t.shape == (1, k, d)

    def score_fn(tuples):
        if len(tuples) == 0:
            return []
        sse, _ = oracle.score(prob.X, prob.y, np.array(tuples, dtype=np.int32),
                              offsets=prob.offsets)
        return sse.sum(axis=1) / prob.n_total

    ok, msg = oracle.agreement(ref["tuples"][0], ref["score"][0], t[0], rel_gap=TIE_GAP,
                               score_fn=score_fn)
    assert ok, msg
    fin = np.isfinite(ref["rmse"][0])
    np.testing.assert_allclose(r[0][fin], ref["rmse"][0][fin], rtol=RMSE_RTOL)
    assert st["certified"] == 1
    return t, r


@pytest.mark.parametrize("precision", [l0.FP64, l0.MIXED_BF16X3])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_shared_matches_oracle(precision, d):
    prob = make_problem([40, 75, 130, 60], 90, seed=301 + d, n_planted=2, sigma=0.03)
    _check_shared(prob, d, 25, precision)


@pytest.mark.parametrize("precision", [l0.FP64, l0.MIXED_BF16X3])
def test_shared_c3_shape_small(precision):
    # C3-like: uneven task sizes, each task with its own planted pair
    prob = make_problem([50, 120, 300, 500], 160, seed=311, n_planted=2, sigma=0.02,
                        distinct=False)
    _check_shared(prob, 2, 30, precision)


def test_shared_rank_deficient_in_one_task_is_ineligible():
    prob = make_problem([40, 60], 30, seed=321, n_planted=2, sigma=0.05)
    X = prob.X.copy()
    # columns 4 and 9 identical on task 0's rows only
    X[9, :40] = X[4, :40]
    k = math.comb(30, 2) - 1
    ref = oracle.fit(X, prob.y, 2, k, offsets=prob.offsets, mode=oracle.SHARED)
    with l0.Handle(task_mode=l0.SHARED) as h:
        t, r = h.fit(X, prob.y, 2, k, offsets=prob.offsets)
    got = {tuple(x) for x in t[0] if x[0] >= 0}
    assert (4, 9) not in got
    assert int(ref["n_eligible"][0]) == k
    assert np.isfinite(r[0]).sum() == k
