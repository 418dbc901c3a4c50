"""Batched searches (several tuple sizes over the same data in one persistent
launch), CUDA-graph replay and the launch autotuner, checked against the CPU
oracle and against the single-request path."""

import os

import numpy as np
import pytest

import oracle
import paper_2502_20072_gb300 as l0
from l0_testutil import RMSE_RTOL, TIE_GAP, score_fn
from workloads import make_problem

pytestmark = pytest.mark.gpu


def _check_list(prob, d, k, t, r, task=0):
    lo, hi = prob.offsets[task], prob.offsets[task + 1]
    X, y = prob.X[:, lo:hi], prob.y[lo:hi]
    ref = oracle.fit(X, y, d, k)
    ok, msg = oracle.agreement(ref["tuples"][0], ref["score"][0], t, rel_gap=TIE_GAP,
                               score_fn=score_fn(X, y))
    assert ok, msg
    fin = np.isfinite(ref["rmse"][0])
    np.testing.assert_allclose(r[fin], ref["rmse"][0][fin], rtol=RMSE_RTOL)


@pytest.mark.parametrize("precision", [l0.FP64, l0.MIXED_BF16X3])
def test_multi_request_one_pass_matches_oracle(precision):
    # C3 shape, scaled down: uneven tasks, d = 2 and d = 3 (and d = 1) in one pass
    prob = make_problem([50, 120, 300, 500], 120, seed=401, n_planted=2, sigma=0.02,
                        distinct=False)
    with l0.Handle(precision=precision) as h:
        outs = h.fit_multi(prob.X, prob.y, [(2, 20), (3, 30), (1, 5)], offsets=prob.offsets)
        st = h.stats()
    assert st["certified"] == 1
    for (d, k), (t, r) in zip([(2, 20), (3, 30), (1, 5)], outs):
        assert t.shape == (4, k, d)
        for task in range(4):
            _check_list(prob, d, k, t[task], r[task], task)


def test_multi_request_equals_single_requests():
    prob = make_problem([80, 140], 150, seed=402, n_planted=2, sigma=0.02)
    with l0.Handle(precision=l0.MIXED_BF16X3) as h:
        outs = h.fit_multi(prob.X, prob.y, [(2, 25), (4, 25), (3, 25)], offsets=prob.offsets)
        for (d, k), (t, r) in zip([(2, 25), (4, 25), (3, 25)], outs):
            t1, r1 = h.fit(prob.X, prob.y, d, k, offsets=prob.offsets)
            np.testing.assert_array_equal(t, t1)
            np.testing.assert_allclose(r, r1, rtol=1e-12)


def test_multi_request_rejects_wide_tuple_size_spread():
    prob = make_problem(60, 40, seed=403, n_planted=2, sigma=0.02)
    with l0.Handle() as h:
        with pytest.raises(l0.L0Error) as e:
            h.fit_multi(prob.X, prob.y, [(2, 5), (6, 5)])
        assert e.value.code == l0.EUNSUPPORTED


@pytest.mark.parametrize("precision", [l0.FP64, l0.MIXED_BF16X3])
def test_graph_replay_gives_identical_results(precision):
    import torch
    prob = make_problem([70, 90], 130, seed=404, n_planted=3, sigma=0.02)
    X = torch.from_numpy(prob.X).cuda()
    y = torch.from_numpy(prob.y).cuda()
    with l0.Handle(precision=precision, use_graph=1) as h:
        t0, r0 = h.fit(X, y, 3, 30, offsets=prob.offsets)
        s0 = h.stats()
        t1, r1 = h.fit(X, y, 3, 30, offsets=prob.offsets)
        s1 = h.stats()
    assert s0["graph_replayed"] == 0 and s1["graph_replayed"] == 1
    np.testing.assert_array_equal(t0, t1)
    np.testing.assert_array_equal(r0, r1)
    with l0.Handle(precision=precision) as h:
        t2, r2 = h.fit(X, y, 3, 30, offsets=prob.offsets)
    np.testing.assert_array_equal(t0, t2)
    np.testing.assert_allclose(r0, r2, rtol=1e-12)


def test_autotuner_choice_is_persisted_and_results_unchanged(tmp_path):
    prob = make_problem(300, 260, seed=405, n_planted=3, sigma=0.02)
    cache = str(tmp_path / "tune.txt")
    with l0.Handle(precision=l0.MIXED_BF16X3, autotune=1, autotune_cache_path=cache) as h:
        t0, r0 = h.fit(prob.X, prob.y, 3, 40)
        st = h.stats()
    assert st["tuned_items_factor"] in (1, 2, 4, 8, 16)
    assert st["tuned_ctas_per_sm"] in (1, 2)
    lines = open(cache).read().split("\n")
    assert any(line.strip() for line in lines)
    # a new handle reads the cache and reproduces the search
    with l0.Handle(precision=l0.MIXED_BF16X3, autotune=1, autotune_cache_path=cache) as h:
        t1, r1 = h.fit(prob.X, prob.y, 3, 40)
        st1 = h.stats()
    assert (st1["tuned_items_factor"], st1["tuned_ctas_per_sm"], st1["tuple_kernel"]) == \
        (st["tuned_items_factor"], st["tuned_ctas_per_sm"], st["tuple_kernel"])
    np.testing.assert_array_equal(t0, t1)
    _check_list(prob, 3, 40, t0[0], r0[0])
    # each line: key, items per CTA factor, CTAs per SM, kernel shape (the shape
    # the fit ran: the d <= 3 FP32 kernel's shapes are among the candidates)
    rec = [ln.split() for ln in lines if ln.strip()]
    assert all(len(f) == 4 for f in rec)
    assert (int(rec[-1][1]), int(rec[-1][3])) == (st["tuned_items_factor"], st["tuple_kernel"])
    assert st["tuple_kernel"] in (0, 1, 2, 3)


@pytest.mark.parametrize("v", [0, 1, 2, 3])
def test_forced_kernel_shape_is_the_one_tuned_and_run(tmp_path, v):
    # with a fixed shape the autotuner only times launch configurations of it
    prob = make_problem(200, 190, seed=406, n_planted=3, sigma=0.02)
    with l0.Handle(precision=l0.MIXED_BF16X3, autotune=1, tuple_kernel=v,
                   autotune_cache_path=str(tmp_path / "t.txt")) as h:
        t, r = h.fit(prob.X, prob.y, 3, 30)
        st = h.stats()
    assert st["tuple_kernel"] == v
    _check_list(prob, 3, 30, t[0], r[0])
