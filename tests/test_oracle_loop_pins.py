"""Pins of the dimension-loop oracle (CPU only): LAPACK least squares for the
residuals, brute-force multi-target screening, the closed form of the
one-dimensional loop, and recovery of a planted two-term descriptor that only
the residual-driven screening can find."""

import itertools

import numpy as np

from oracle import loop as oloop
from oracle import sis as osis


def _data(seed, n=60, nf=40):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(nf, n)) + rng.uniform(-2, 2, size=(nf, 1))
    y = 1.5 * X[3] - 0.7 * X[11] + 0.3 * rng.normal(size=n) + 4.0
    return X, y


def test_residuals_match_lstsq_and_are_orthogonal():
    X, y = _data(1)
    tuples = [(3,), (3, 11), (0, 5, 7)]
    res = oloop.residuals(X, y, tuples)
    for r, tup in zip(res, tuples):
        A = np.column_stack([np.ones(len(y))] + [X[t] for t in tup])
        beta = np.linalg.lstsq(A, y, rcond=None)[0]
        np.testing.assert_allclose(r, y - A @ beta, atol=1e-10 * np.abs(y).max())
        # orthogonal to the intercept and to every column of the model
        np.testing.assert_allclose(A.T @ r, 0.0, atol=1e-8 * np.abs(A).max() * np.abs(y).max())


def test_sis_multi_is_brute_force_max_abs_r():
    X, y = _data(2)
    res = oloop.residuals(X, y, [(3,), (11,), (3, 11)])
    m = 7
    idx, r = oloop.sis_multi(X, res, m, exclude=[5, 9])
    n_feat = X.shape[0]
    score = np.empty(n_feat)
    first = np.empty(n_feat)
    for j in range(n_feat):
        cs = [np.corrcoef(X[j], t)[0, 1] for t in res]
        a = [abs(c) for c in cs]
        score[j] = max(a)
        first[j] = cs[a.index(max(a))]
    cand = [j for j in range(n_feat) if j not in (5, 9)]
    want = sorted(cand, key=lambda j: (-score[j], j))[:m]
    assert list(idx) == want
    np.testing.assert_allclose(r, first[want], rtol=1e-12)
    # one target: the plain screening
    i1, r1 = oloop.sis_multi(X, y, m)
    i2, r2 = osis.sis(X, y, m)
    assert list(i1) == list(i2)
    np.testing.assert_allclose(r1, r2, rtol=1e-14)


def test_one_dimension_loop_is_best_single_correlation():
    X, y = _data(3)
    out = oloop.dimension_loop(X, y, m=6, D=1, k=3, n_res=2)
    r = osis.pearson(X, y)
    best = sorted(range(len(r)), key=lambda j: (-abs(r[j]), j))
    assert list(out[0]["S"]) == best[:6]
    assert out[0]["tuples"][0, 0] == best[0]
    syy = float(((y - y.mean()) ** 2).sum())
    np.testing.assert_allclose(out[0]["rmse"][0] ** 2 * len(y), syy * (1 - r[best[0]] ** 2),
                               rtol=1e-10)


def test_residual_screening_finds_planted_second_term():
    """y = 3 x_a + 0.4 x_b with x_b independent of x_a and weakly correlated
    with y: it is outside the first screening but tops the residual one."""
    rng = np.random.default_rng(4)
    n, nf = 80, 60
    X = rng.normal(size=(nf, n))
    a, b = 17, 42
    # features 0..9 correlated with x_a, so they crowd the first screening
    for j in range(10):
        X[j] = X[a] + 0.3 * rng.normal(size=n)
    y = 3.0 * X[a] + 0.4 * X[b]
    out = oloop.dimension_loop(X, y, m=8, D=2, k=5, n_res=3)
    assert b not in out[0]["S"]
    assert b in out[1]["S"][8:]
    assert tuple(out[1]["tuples"][0]) == (a, b)
    assert out[1]["rmse"][0] < 1e-12 * np.abs(y).max()
    # S grows by m per dimension, without repeats
    assert len(set(out[1]["S"].tolist())) == 16
    # the 2-D search is exhaustive over S: brute force over all pairs of S
    S = out[1]["S"]
    best = None
    for i, j in itertools.combinations(range(len(S)), 2):
        A = np.column_stack([np.ones(n), X[S[i]], X[S[j]]])
        rr = y - A @ np.linalg.lstsq(A, y, rcond=None)[0]
        sse = float(rr @ rr)
        if best is None or sse < best[0]:
            best = (sse, tuple(sorted((int(S[i]), int(S[j])))))
    assert best[1] == (a, b)


def test_loop_never_reselects_and_takes_all_models_when_fewer_than_n_res():
    X, y = _data(5, n=50, nf=30)
    out = oloop.dimension_loop(X, y, m=4, D=3, k=2, n_res=10)
    S = out[-1]["S"].tolist()
    assert len(S) == 12 and len(set(S)) == 12
    # each dimension's S extends the previous one
    for a, b in zip(out, out[1:]):
        assert b["S"][:len(a["S"])].tolist() == a["S"].tolist()
    # dimension 2 screens against the residuals of both (k = 2 < n_res) 1-D models
    res = oloop.residuals(X, y, out[0]["tuples"])
    idx, _ = oloop.sis_multi(X, res, 4, exclude=out[0]["S"])
    assert out[1]["S"][4:].tolist() == idx.tolist()
