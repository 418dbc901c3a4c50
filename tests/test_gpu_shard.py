"""Sharded search on one GPU: the shards run one after the other (as
separate workers would), their candidate pools are merged, and the result
equals the unsharded search and the oracle."""

import numpy as np
import pytest

import oracle
import paper_2502_20072_gb300 as l0
from paper_2502_20072_gb300.shard import fit_sharded
from workloads import make_config, make_problem

from l0_testutil import RMSE_RTOL, TIE_GAP, score_fn

pytestmark = pytest.mark.gpu


def _sharded(h, X, y, d, k, n_shards):
    keys, sse, bounds, deltas = [], [], [], []
    for s in range(n_shards):
        kk, ss, b, dl = h.fit_shard(X, y, d, k, s, n_shards)
        keys.append(kk)
        sse.append(ss)
        bounds.append(b)
        deltas.append(dl)
    return h.merge_shards(X.shape[0], d, k, X.shape[1], np.concatenate(keys),
                          np.concatenate(sse), np.array(bounds), np.array(deltas))


@pytest.mark.parametrize("precision", [l0.FP64, l0.MIXED_BF16X3])
@pytest.mark.parametrize("n_shards", [1, 2, 3, 8])
def test_shards_merge_to_the_unsharded_result(precision, n_shards):
    p = make_problem(n_samples=300, n_sis=150, seed=9, n_planted=3, sigma=0.02)
    with l0.Handle(precision=precision) as h:
        ref_t, ref_r = h.fit(p.X, p.y, 3, 50)
        t, r, cert = _sharded(h, p.X, p.y, 3, 50, n_shards)
    assert cert
    np.testing.assert_array_equal(t, ref_t[0])
    np.testing.assert_array_equal(r, ref_r[0])


@pytest.mark.parametrize("d", [2, 4])
def test_shards_match_oracle(d):
    p = make_problem(n_samples=80, n_sis=24, seed=10, n_planted=2, sigma=0.05)
    k = 20
    ref = oracle.fit(p.X, p.y, d, k)
    with l0.Handle(precision=l0.MIXED_BF16X3) as h:
        t, r, cert = _sharded(h, p.X, p.y, d, k, 3)
    assert cert
    ok, msg = oracle.agreement(ref["tuples"][0], ref["score"][0], t, rel_gap=TIE_GAP,
                               score_fn=score_fn(p.X, p.y))
    assert ok, msg
    np.testing.assert_allclose(r, ref["rmse"][0], rtol=RMSE_RTOL)


def test_fit_sharded_single_process_is_the_plain_search():
    prob, d, k = make_config("C1")
    with l0.Handle(precision=l0.FP64) as h:
        t, r, cert = fit_sharded(h, prob.X, prob.y, d, k)
        ref_t, ref_r = h.fit(prob.X, prob.y, d, k)
    assert cert
    np.testing.assert_array_equal(t, ref_t[0])
    np.testing.assert_array_equal(r, ref_r[0])
