"""The batched multi-task workload (8 tasks of 50..2000 samples, 2000 shared
columns with duplicates, d = 2 and d = 3 in one pass) and the d = 4 workload
with near-collinear columns (5000 samples, 400 columns), at full size.

The oracle cannot search these exhaustively in test time, so each is pinned
three ways: the oracle re-fits the GPU's reported tuples (RMSE to 1e-10 and
eligibility), the exhaustive order is checked on a sub-block of columns the
oracle can search, and the properties the workload plants (the planted
descriptor first, FP64 redo of near-collinear blocks) hold."""

import numpy as np
import pytest

import oracle
import paper_2502_20072_gb300 as l0
from workloads import make_config

from l0_testutil import RMSE_RTOL, TIE_GAP, score_fn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c3():
    prob, dims, k = make_config("C3")
    return prob, dims, k


@pytest.fixture(scope="module")
def c4():
    return make_config("C4")


def _refit_matches(X, y, offsets, tuples, rmse, task):
    lo, hi = int(offsets[task]), int(offsets[task + 1])
    ok = tuples[:, 0] >= 0
    sse, rho = oracle.score(X, y, tuples[ok], offsets=offsets)
    assert np.all(rho[:, task] >= oracle.RHO_MIN)
    ref = np.sqrt(sse[:, task] / (hi - lo))
    np.testing.assert_allclose(rmse[ok], ref, rtol=RMSE_RTOL, atol=0)
    assert np.all(np.diff(rmse[ok]) >= -1e-12 * rmse[ok][1:])   # ranked


def _same_values(X, a, b):
    """Tuples a and b hold the same columns up to value-identical copies."""
    A = sorted(X[int(i)].tobytes() for i in a)
    B = sorted(X[int(i)].tobytes() for i in b)
    return A == B


def test_c3_batched_both_dims_one_pass(c3):
    prob, dims, k = c3
    reqs = [(2, k), (3, k)]
    with l0.Handle(precision=l0.MIXED_BF16X3, use_graph=1, autotune=1) as h:
        out = h.fit_multi(prob.X, prob.y, reqs, offsets=prob.offsets)
        st = h.stats()
        again = h.fit_multi(prob.X, prob.y, reqs, offsets=prob.offsets)
        st2 = h.stats()
    print("C3 stats", {q: st[q] for q in ("certified", "candidate_pool", "pool_enlargements",
                                          "max_pool_rel_error", "fp64_fallback_tuples",
                                          "fp64_rerun")})
    for (t1, r1), (t2, r2) in zip(out, again):
        np.testing.assert_array_equal(t1, t2)
        np.testing.assert_array_equal(r1, r2)
    (t2d, r2d), (t3d, r3d) = out
    for task in range(prob.n_tasks):
        # the planted two-term descriptor (or a value-identical copy) is first
        assert _same_values(prob.X, t2d[task, 0], prob.planted[task]), task
        _refit_matches(prob.X, prob.y, prob.offsets, t2d[task], r2d[task], task)
        _refit_matches(prob.X, prob.y, prob.offsets, t3d[task], r3d[task], task)
    assert st["certified"] == 1


def test_c3_sub_block_exhaustive_order(c3):
    prob, dims, k = c3
    cols = np.arange(80)
    X = np.ascontiguousarray(prob.X[cols])
    with l0.Handle(precision=l0.MIXED_BF16X3) as h:
        out = h.fit_multi(X, prob.y, [(2, 30), (3, 30)], offsets=prob.offsets)
    for (tg, rg), d in zip(out, (2, 3)):
        ref = oracle.fit(X, prob.y, d, 30, offsets=prob.offsets)
        for task in range(prob.n_tasks):
            ok, msg = oracle.agreement(ref["tuples"][task], ref["score"][task], tg[task],
                                       rel_gap=TIE_GAP, score_fn=score_fn(X, prob.y, prob.offsets, task))
            assert ok, (d, task, msg)
            fin = np.isfinite(ref["rmse"][task])
            np.testing.assert_allclose(rg[task][fin], ref["rmse"][task][fin], rtol=RMSE_RTOL)


def test_c3_shared_sub_block(c3):
    prob, dims, k = c3
    X = np.ascontiguousarray(prob.X[:60])
    ref = oracle.fit(X, prob.y, 2, 25, offsets=prob.offsets, mode=oracle.SHARED)
    with l0.Handle(precision=l0.MIXED_BF16X3, task_mode=l0.SHARED) as h:
        tg, rg = h.fit(X, prob.y, 2, 25, offsets=prob.offsets)

    def pooled(tuples):
        if len(tuples) == 0:
            return []
        sse, _ = oracle.score(X, prob.y, np.array(tuples, dtype=np.int32), offsets=prob.offsets)
        return sse.sum(axis=1) / prob.n_total
    ok, msg = oracle.agreement(ref["tuples"][0], ref["score"][0], tg[0], rel_gap=TIE_GAP,
                               score_fn=pooled)
    assert ok, msg
    np.testing.assert_allclose(rg[0], ref["rmse"][0], rtol=RMSE_RTOL)


def test_c4_mixed_equals_fp64_and_refits(c4):
    prob, d, k = c4
    with l0.Handle(precision=l0.MIXED_BF16X3) as h:
        tm, rm = h.fit(prob.X, prob.y, d, k)
        st = h.stats()
        if st["fp64_rerun"] == 1:
            # the same inputs again: straight to FP64, same result
            tm2, rm2 = h.fit(prob.X, prob.y, d, k)
            assert h.stats()["fp64_rerun"] == 2
            np.testing.assert_array_equal(tm2, tm)
            np.testing.assert_array_equal(rm2, rm)
    with l0.Handle(precision=l0.FP64) as h:
        tf, rf = h.fit(prob.X, prob.y, d, k)
    print("C4 stats", {q: st[q] for q in ("certified", "candidate_pool", "pool_enlargements",
                                          "max_pool_rel_error", "fp64_fallback_tuples",
                                          "fp64_rerun")})
    assert st["fp64_fallback_tuples"] > 0 or st["fp64_rerun"] == 1          # near-collinear blocks went to FP64
    ok, msg = oracle.agreement(tf[0], rf[0] ** 2 * prob.n_total, tm[0], rel_gap=TIE_GAP,
                               score_fn=score_fn(prob.X, prob.y))
    assert ok, msg
    np.testing.assert_allclose(rm[0], rf[0], rtol=RMSE_RTOL)
    _refit_matches(prob.X, prob.y, prob.offsets, tm[0], rm[0], 0)
    # the best 4-tuple beats every completion of the planted triple
    pl = list(prob.planted[0])
    rest = [c for c in range(prob.n_sis) if c not in pl]
    comp = np.sort(np.array([pl + [c] for c in rest], dtype=np.int32), axis=1)
    sse, rho = oracle.score(prob.X, prob.y, comp)
    best = np.min(sse[rho[:, 0] >= oracle.RHO_MIN, 0])
    assert rm[0, 0] ** 2 * prob.n_total <= best * (1 + 1e-12)
    assert st["certified"] == 1


def test_c4_sub_block_with_collinear_pairs(c4):
    prob, d, k = c4
    rep = prob.replaced[:10]
    cols = np.unique(np.concatenate([rep[:, 0], rep[:, 1], np.arange(10)]))
    X = np.ascontiguousarray(prob.X[cols])
    ref = oracle.fit(X, prob.y, d, 40)
    for prec in (l0.MIXED_BF16X3, l0.FP64):
        with l0.Handle(precision=prec) as h:
            tg, rg = h.fit(X, prob.y, d, 40)
        ok, msg = oracle.agreement(ref["tuples"][0], ref["score"][0], tg[0], rel_gap=TIE_GAP,
                                   score_fn=score_fn(X, prob.y))
        assert ok, (prec, msg)
        np.testing.assert_allclose(rg[0], ref["rmse"][0], rtol=RMSE_RTOL)
