"""Failure paths made on the host, with no GPU fault: the host-side deadline
(ETIMEOUT) and an allocation that reports out-of-memory (ENOMEM, injected by
the library's test hook without exhausting the device).  After either, the
same handle must return the oracle's result on its next call."""

import numpy as np
import pytest

import oracle
import paper_2502_20072_gb300 as l0
from l0_testutil import RMSE_RTOL, TIE_GAP, score_fn
from workloads import make_config, make_problem

pytestmark = pytest.mark.gpu


def _check(prob, d, ref, t, r):
    ok, msg = oracle.agreement(ref["tuples"][0], ref["score"][0], t[0], rel_gap=TIE_GAP,
                               score_fn=score_fn(prob.X, prob.y))
    assert ok, msg
    np.testing.assert_allclose(r[0], ref["rmse"][0], rtol=RMSE_RTOL)


def test_deadline_returns_etimeout_then_the_handle_recovers():
    prob, d, k = make_config("C2")
    k = 20
    ref = oracle.fit(prob.X, prob.y, d, k)
    # the FP64 search of this workload keeps the GPU busy for milliseconds:
    # a one-microsecond host deadline expires while it runs
    with l0.Handle(precision=l0.FP64, timeout_seconds=1e-6) as h:
        with pytest.raises(l0.L0Error) as e:
            h.fit(prob.X, prob.y, d, k)
        assert e.value.code == l0.ETIMEOUT
        h.set_timeout(300.0)
        t, r = h.fit(prob.X, prob.y, d, k)
        _check(prob, d, ref, t, r)


@pytest.mark.parametrize("after", [0, 3, 9, 20])
@pytest.mark.parametrize("precision", [l0.FP64, l0.MIXED_BF16X3])
def test_allocation_failure_returns_enomem_then_the_handle_recovers(after, precision):
    prob = make_problem(150, 160, seed=801, n_planted=3, sigma=0.02)
    ref = oracle.fit(prob.X, prob.y, 3, 15)
    with l0.Handle(precision=precision, use_graph=1) as h:
        l0.debug_fail_allocation(after)
        try:
            h.fit(prob.X, prob.y, 3, 15)
            failed = None
        except l0.L0Error as e:
            failed = e.code
        finally:
            l0.debug_fail_allocation(-1)
        # a fit makes more than `after` allocations on a fresh handle
        assert failed == l0.ENOMEM
        t, r = h.fit(prob.X, prob.y, 3, 15)
        _check(prob, 3, ref, t, r)
        t, r = h.fit(prob.X, prob.y, 3, 15)   # and again (graph captured now)
        _check(prob, 3, ref, t, r)
