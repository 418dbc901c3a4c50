"""SIS screening on the GPU against the oracle (Pearson r of every feature,
the m largest |r|, ties by index)."""

import numpy as np
import pytest

import paper_2502_20072_gb300 as l0
from oracle import sis as osis
from workloads import make_problem

pytestmark = pytest.mark.gpu


def _check(X, y, m, idx, r, tol=1e-11):
    ref_idx, ref_r = osis.sis(X, y, m)
    full = osis.pearson(X, y)
    # r of the selected features to FP64 rounding (shifted one-pass sums vs
    # the oracle's two passes), or to FP32 rounding of the centred products
    np.testing.assert_allclose(r, full[idx], rtol=tol, atol=tol * 1e-2)
    # same selection, except among features whose |r| differ by < 1e-11
    # (their order is decided by rounding)
    a = np.abs(full)
    cut = a[ref_idx[-1]]
    sure = set(np.nonzero(a > cut * (1 + tol))[0].tolist())
    assert sure <= set(idx.tolist())
    assert all(a[j] >= cut * (1 - tol) for j in idx)
    # the ordering is by |r| descending
    assert np.all(np.diff(np.abs(r)) <= 1e-12)
    # position by position, up to groups of near-equal |r| (value-identical
    # or ulp-different copies of one column), whose order rounding decides
    ra = a[ref_idx]
    i = 0
    while i < m:
        j = i + 1
        while j < m and ra[j - 1] - ra[j] <= tol * ra[j - 1]:
            j += 1
        if j < m:       # a group ending before the cut must match as a set
            assert set(idx[i:j].tolist()) == set(ref_idx[i:j].tolist()), (i, j)
        i = j


@pytest.mark.parametrize("precision,tol", [(l0.FP64, 1e-11), (l0.MIXED_BF16X3, 2e-6)])
def test_sis_matches_oracle_small(precision, tol):
    p = make_problem(n_samples=300, n_sis=5000, seed=41, n_planted=3, sigma=0.1, distinct=True,
                     factors=4)
    with l0.Handle(precision=precision) as h:
        idx, r = h.sis(p.X, p.y, 100)
    _check(p.X, p.y, 100, idx, r, tol)
    # a planted column is among the best
    assert set(p.planted[0]) & set(idx.tolist())


def test_sis_ties_by_index_and_constants():
    rng = np.random.default_rng(5)
    X = rng.normal(size=(500, 64))
    X[10] = X[200]          # exact duplicates: equal |r|, smaller index first
    X[20] = 3.0             # constant: r = 0
    y = X[200] + 0.5 * rng.normal(size=64)
    with l0.Handle() as h:
        idx, r = h.sis(X, y, 50)
    assert idx[0] == 10 and idx[1] == 200
    assert r[0] == r[1]
    assert 20 not in idx.tolist()
    _check(X, y, 50, idx, r)


def test_sis_large_device_input():
    torch = pytest.importorskip("torch")
    p = make_problem(n_samples=500, n_sis=200000, seed=42, n_planted=3, sigma=0.05,
                     distinct=False, factors=4)
    X = torch.from_numpy(p.X).cuda()
    y = torch.from_numpy(p.y).cuda()
    for precision, tol in ((l0.FP64, 1e-11), (l0.MIXED_BF16X3, 2e-6)):
        with l0.Handle(precision=precision) as h:
            idx, r = h.sis(X, y, 1000)
        _check(p.X, p.y, 1000, idx, r, tol)


def test_sis_errors():
    X = np.ones((10, 5))
    y = np.arange(5.0)
    with l0.Handle() as h:
        with pytest.raises(l0.L0Error) as e:
            h.sis(X, y, 11)
        assert e.value.code == l0.EINVAL
        X2 = np.random.default_rng(0).normal(size=(10, 5))
        X2[3, 2] = np.nan
        with pytest.raises(l0.L0Error) as e:
            h.sis(X2, y, 3)
        assert e.value.code == l0.ENONFINITE
