"""GPU parity of every tuple-kernel shape of the FP32 search (the general
kernel, 0, and the d = 2/3 kernel's shapes 1, 2, 3) against the CPU oracle:
the reported tuples must be the oracle's (tie rule), RMSE to 1e-10.  Cases:
d = 2 and 3, sizes that leave ragged tiles (m not a multiple of 64 or 128),
several tasks of uneven size, duplicated columns (exactly rank deficient),
near-collinear columns (FP32 pivots below the redo ratio, FP64 redo), the
full-size headline workload against the stored exhaustive oracle result, and
both d in one call."""

import math

import numpy as np
import pytest

import oracle
import paper_2502_20072_gb300 as l0
from c2_golden import load
from l0_testutil import RMSE_RTOL, TIE_GAP, check_against_oracle, score_fn
from workloads import make_config, make_problem

pytestmark = pytest.mark.gpu
SHAPES = [0, 1, 2, 3]


def _opts(v):
    return dict(precision=l0.MIXED_BF16X3, tuple_kernel=v)


@pytest.mark.parametrize("v", SHAPES)
@pytest.mark.parametrize("n,m,d,k", [
    (70, 150, 3, 30),
    (90, 197, 3, 45),      # ragged: 197 = 3 * 64 + 5, one k tile of 69 columns
    (60, 131, 2, 40),
    (300, 400, 3, 60),
])
def test_shapes_match_oracle(v, n, m, d, k):
    prob = make_problem(n, m, seed=700 + m + d, n_planted=min(d, 3), sigma=0.05)
    _, _, st = check_against_oracle(prob.X, prob.y, d, k, **_opts(v))
    assert st["certified"] == 1
    if v and d <= 3:
        assert st["tuple_kernel"] == v


@pytest.mark.parametrize("v", SHAPES)
def test_shapes_multitask(v):
    prob = make_problem([45, 80, 133], 140, seed=731, n_planted=2, sigma=0.03)
    check_against_oracle(prob.X, prob.y, 3, 25, offsets=prob.offsets, **_opts(v))


@pytest.mark.parametrize("v", SHAPES)
def test_shapes_duplicates_and_near_collinear(v):
    prob = make_problem(260, 120, seed=741, n_planted=3, sigma=0.01, replace_frac=0.2)
    X = prob.X.copy()
    X[50] = X[7]          # exact duplicates: ineligible
    X[101] = X[33]
    _, _, st = check_against_oracle(X, prob.y, 3, 50, **_opts(v))
    assert st["fp64_fallback_tuples"] > 0


@pytest.mark.parametrize("v", SHAPES)
def test_shapes_both_d_in_one_call(v):
    prob = make_problem(120, 170, seed=751, n_planted=2, sigma=0.02)
    ref2 = oracle.fit(prob.X, prob.y, 2, 20)
    ref3 = oracle.fit(prob.X, prob.y, 3, 30)
    with l0.Handle(**_opts(v)) as h:
        (t2, r2), (t3, r3) = h.fit_multi(prob.X, prob.y, [(2, 20), (3, 30)])
        st = h.stats()
    for ref, t, r in ((ref2, t2, r2), (ref3, t3, r3)):
        ok, msg = oracle.agreement(ref["tuples"][0], ref["score"][0], t[0], rel_gap=TIE_GAP,
                                   score_fn=score_fn(prob.X, prob.y))
        assert ok, msg
        np.testing.assert_allclose(r[0], ref["rmse"][0], rtol=RMSE_RTOL)
    if v:
        assert st["tuple_kernel"] == v


@pytest.mark.parametrize("v", [1, 2, 3])
def test_shapes_headline_against_exhaustive_oracle(v):
    prob, d, k = make_config("C2")
    ref_t, ref_sse, ref_rmse = load()
    with l0.Handle(**_opts(v)) as h:
        t, r = h.fit(prob.X, prob.y, d, k)
        st = h.stats()
    assert st["certified"] == 1 and st["tuple_kernel"] == v
    ok, msg = oracle.agreement(ref_t[:k], ref_sse[:k], t[0], rel_gap=TIE_GAP,
                               score_fn=score_fn(prob.X, prob.y))
    assert ok, msg
    np.testing.assert_allclose(r[0], ref_rmse[:k], rtol=RMSE_RTOL)
