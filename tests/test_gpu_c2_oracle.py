"""The headline d = 3 workload (n = 1000, m = 1000, k = 100) against the
oracle's exhaustive result over all C(1000, 3) tuples (stored by
tests/golden/make_c2_top.py, which calls only the oracle): every one of the
100 tuples under the tie rule and every RMSE to 1e-10, for the plain FP64
path and the mixed-precision path, each with and without graph replay."""

import numpy as np
import pytest

import oracle
import paper_2502_20072_gb300 as l0
from c2_golden import load
from l0_testutil import RMSE_RTOL, TIE_GAP, score_fn
from workloads import make_config

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [l0.FP64, l0.MIXED_BF16X3])
def test_c2_top100_equals_exhaustive_oracle(precision):
    prob, d, k = make_config("C2")
    ref_t, ref_sse, ref_rmse = load()
    ref_t, ref_sse, ref_rmse = ref_t[:k], ref_sse[:k], ref_rmse[:k]
    with l0.Handle(precision=precision, use_graph=1) as h:
        for _ in range(2):          # the second call replays the captured graph
            t, r = h.fit(prob.X, prob.y, d, k)
            st = h.stats()
            assert st["certified"] == 1
            ok, msg = oracle.agreement(ref_t, ref_sse, t[0], rel_gap=TIE_GAP,
                                       score_fn=score_fn(prob.X, prob.y))
            assert ok, msg
            np.testing.assert_allclose(r[0], ref_rmse, rtol=RMSE_RTOL, atol=0)
