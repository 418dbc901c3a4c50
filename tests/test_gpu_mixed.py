"""GPU parity of the mixed-precision path (split-BF16 tensor-core Gram,
FP32 tuple search, FP64 redo of near-singular tuples, FP64 re-fit) against
the CPU oracle.  The reported tuples must be the oracle's (tie rule) and the
RMSEs, which come from the FP64 re-fit, must match to 1e-10 relative."""

import math

import numpy as np
import pytest

import oracle
import paper_2502_20072_gb300 as l0
from l0_testutil import RMSE_RTOL, TIE_GAP, check_against_oracle
from workloads import make_config, make_problem

pytestmark = pytest.mark.gpu
MIXED = dict(precision=l0.MIXED_BF16X3)


@pytest.mark.parametrize("n,m,d,k", [
    (60, 150, 2, 25),
    (80, 150, 3, 40),
    (50, 70, 4, 30),
    (40, 30, 5, 20),
    (200, 300, 3, 50),     # three Gram tiles per side, ragged
])
def test_mixed_fit_matches_oracle(n, m, d, k):
    prob = make_problem(n, m, seed=200 + m + d, n_planted=min(d, 3), sigma=0.05)
    _, _, st = check_against_oracle(prob.X, prob.y, d, k, **MIXED)
    assert st["certified"] == 1


def test_mixed_multitask():
    prob = make_problem([40, 75, 130], 90, seed=231, n_planted=2, sigma=0.03)
    check_against_oracle(prob.X, prob.y, 3, 20, offsets=prob.offsets, **MIXED)


def test_mixed_c1():
    prob, d, k = make_config("C1")
    t, _, _ = check_against_oracle(prob.X, prob.y, d, k, **MIXED)
    assert tuple(t[0, 0]) == (16, 102)


def test_mixed_near_collinear_columns_use_fp64_redo():
    # columns replaced by f_src * (1 + N(0, 1e-4)): FP32 pivots collapse,
    # the FP64 redo must still score them (they are eligible in FP64)
    prob = make_problem(300, 60, seed=241, n_planted=3, sigma=0.01, replace_frac=0.2)
    _, _, st = check_against_oracle(prob.X, prob.y, 3, 40, **MIXED)
    assert st["fp64_fallback_tuples"] > 0


def test_mixed_duplicates_are_ineligible():
    prob = make_problem(50, 40, seed=243, n_planted=2, sigma=0.05)
    X = prob.X.copy()
    X[7] = X[3]
    k = math.comb(40, 2) - 1
    t, r, _ = check_against_oracle(X, prob.y, 2, k, **MIXED)
    assert (3, 7) not in {tuple(x) for x in t[0]}


def test_mixed_agrees_with_fp64_path():
    prob = make_problem(150, 200, seed=251, n_planted=3, sigma=0.02)
    with l0.Handle() as h:
        t64, r64 = h.fit(prob.X, prob.y, 3, 60)
    with l0.Handle(**MIXED) as h:
        t32, r32 = h.fit(prob.X, prob.y, 3, 60)
    np.testing.assert_array_equal(t32, t64)
    np.testing.assert_allclose(r32, r64, rtol=1e-12)


def test_mixed_c2_full_size_sampled_against_oracle():
    prob, d, k = make_config("C2")
    with l0.Handle(**MIXED) as h:
        t, r = h.fit(prob.X, prob.y, d, k)
        st = h.stats()
    assert st["certified"] == 1
    assert tuple(t[0, 0]) == tuple(prob.planted[0])
    sse, _ = oracle.score(prob.X, prob.y, t[0])
    np.testing.assert_allclose(r[0], np.sqrt(sse[:, 0] / prob.n_total), rtol=RMSE_RTOL)
    rng = np.random.default_rng(17)
    samp = np.sort(np.array([rng.choice(prob.n_sis, d, replace=False) for _ in range(4000)]), axis=1)
    ssamp, _ = oracle.score(prob.X, prob.y, samp.astype(np.int32))
    listed = {tuple(x) for x in t[0]}
    for tup, s in zip(samp, ssamp[:, 0]):
        if tuple(tup) not in listed:
            assert s >= sse[-1, 0] * (1 - TIE_GAP)
    # the mixed and FP64 paths return the same list on the headline workload
    with l0.Handle() as h:
        t64, _ = h.fit(prob.X, prob.y, d, k)
    np.testing.assert_array_equal(t, t64)
