"""Pins of the SIS-screening oracle (CPU only): numpy's correlation
routine, invariances, exact correlations, and brute-force selection."""

import numpy as np
import pytest

from oracle import sis as os_


def test_pearson_matches_numpy_corrcoef():
    rng = np.random.default_rng(0)
    X = rng.normal(size=(40, 75)) * rng.uniform(0.1, 10, size=(40, 1)) + rng.normal(size=(40, 1))
    y = rng.normal(size=75)
    r = os_.pearson(X, y)
    ref = np.array([np.corrcoef(X[j], y)[0, 1] for j in range(40)])
    np.testing.assert_allclose(r, ref, rtol=1e-12, atol=1e-14)


def test_pearson_invariances_and_exact_values():
    rng = np.random.default_rng(1)
    x = rng.uniform(0.5, 2.0, size=50)
    y = 3.0 * x - 1.0 + 0.0 * x
    X = np.stack([x, -2.0 * x + 5.0, np.full(50, 3.0), 7.0 * x + 1.0])
    r = os_.pearson(X, y)
    assert r[0] == pytest.approx(1.0, abs=1e-14)
    assert r[1] == pytest.approx(-1.0, abs=1e-14)
    assert r[2] == 0.0                       # constant column
    assert r[3] == pytest.approx(r[0], abs=1e-14)   # affine invariance
    # shifting y changes nothing
    np.testing.assert_allclose(os_.pearson(X, y + 100.0), r, atol=1e-13)


def test_sis_selection_is_brute_force_top_m():
    rng = np.random.default_rng(2)
    X = rng.normal(size=(60, 30))
    X[7] = X[3]                               # an exact tie: index order decides
    y = rng.normal(size=30)
    idx, r = os_.sis(X, y, 12)
    full = os_.pearson(X, y)
    # brute force: a feature is selected iff fewer than 12 beat it under
    # (|r| desc, index asc)
    sel = []
    for j in range(60):
        better = sum(1 for q in range(60)
                     if abs(full[q]) > abs(full[j]) or (abs(full[q]) == abs(full[j]) and q < j))
        if better < 12:
            sel.append((better, j))
    assert [j for _, j in sorted(sel)] == idx.tolist()
    np.testing.assert_array_equal(r, full[idx])
    if 3 in idx and 7 in idx:
        assert list(idx).index(3) < list(idx).index(7)
