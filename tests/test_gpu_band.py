"""Mixed precision on workloads whose best scores the FP32 search cannot
rank: the first FP32 pass is followed by a band pass that scores every tuple
below its k-th re-fitted score + 8 delta in FP64, instead of a full FP64
rerun.  The results must be the oracle's (small case, exhaustive) or the
plain FP64 GPU path's (the batched multi-task and the d = 4 workloads, at
full size), with no FP64 rerun."""

import numpy as np
import pytest

import oracle
import paper_2502_20072_gb300 as l0
from l0_testutil import RMSE_RTOL, TIE_GAP, check_against_oracle, score_fn
from workloads import make_config, make_problem

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("v", [0, 2, 3])
def test_band_pass_on_a_low_noise_target(v):
    # sigma 1e-5: the best relative SSEs (~1e-11) are far below FP32's resolution
    prob = make_problem(400, 180, seed=901, n_planted=2, sigma=1e-5)
    _, _, st = check_against_oracle(prob.X, prob.y, 3, 40, precision=l0.MIXED_BF16X3,
                                    tuple_kernel=v)
    assert st["band_pass"] == 1 and st["fp64_rerun"] == 0 and st["certified"] == 1


def _vs_fp64(prob, reqs, **kw):
    with l0.Handle(precision=l0.MIXED_BF16X3, **kw) as h:
        got = h.fit_multi(prob.X, prob.y, reqs, offsets=prob.offsets)
        st = h.stats()
    with l0.Handle(precision=l0.FP64) as h:
        ref = h.fit_multi(prob.X, prob.y, reqs, offsets=prob.offsets)
    for (tg, rg), (tf, rf) in zip(got, ref):
        for task in range(prob.n_tasks):
            lo, hi = prob.offsets[task], prob.offsets[task + 1]
            fin = np.isfinite(rf[task])
            ok, msg = oracle.agreement(tf[task][fin], rf[task][fin] ** 2 * (hi - lo),
                                       tg[task][fin], rel_gap=TIE_GAP,
                                       score_fn=score_fn(prob.X, prob.y, prob.offsets, task))
            assert ok, (task, msg)
            np.testing.assert_allclose(rg[task][fin], rf[task][fin], rtol=RMSE_RTOL)
    return st


def test_band_pass_batched_multitask_workload():
    prob, dims, k = make_config("C3")
    st = _vs_fp64(prob, [(2, k), (3, k)], use_graph=1)
    print("C3 band stats", {q: st[q] for q in ("certified", "band_pass", "fp64_rerun",
                                               "candidate_pool", "fp64_fallback_tuples")})
    assert st["fp64_rerun"] == 0 and st["certified"] == 1


def test_band_pass_d4_near_collinear_workload():
    prob, d, k = make_config("C4")
    st = _vs_fp64(prob, [(d, k)])
    print("C4 band stats", {q: st[q] for q in ("certified", "band_pass", "fp64_rerun",
                                               "candidate_pool", "fp64_fallback_tuples")})
    assert st["fp64_rerun"] == 0 and st["certified"] == 1
