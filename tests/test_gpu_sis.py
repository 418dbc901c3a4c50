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


def _sis(X, y, m):
    """Both scans: the FP64 one and the pre-screened one must agree bit for
    bit (the pre-screen only decides which features the FP64 routine scores)."""
    with l0.Handle(precision=l0.FP64) as h:
        idx64, r64 = h.sis(X, y, m)
    with l0.Handle(precision=l0.MIXED_BF16X3) as h:
        idx, r = h.sis(X, y, m)
        st = h.stats()
    np.testing.assert_array_equal(idx, idx64)
    np.testing.assert_array_equal(r, r64)
    return idx, r, st


def test_sis_matches_oracle_small():
    p = make_problem(n_samples=300, n_sis=5000, seed=41, n_planted=3, sigma=0.1, distinct=True,
                     factors=4)
    idx, r, st = _sis(p.X, p.y, 100)
    _check(p.X, p.y, 100, idx, r)
    # a planted column is among the best
    assert set(p.planted[0]) & set(idx.tolist())
    # the pre-screen sends few features past the m selected to FP64
    assert 100 <= st["fp64_fallback_tuples"] <= 400


def test_sis_ties_by_index_and_constants():
    rng = np.random.default_rng(5)
    X = rng.normal(size=(500, 64))
    X[10] = X[200]          # exact duplicates: equal |r|, smaller index first
    X[20] = 3.0             # constant: r = 0
    y = X[200] + 0.5 * rng.normal(size=64)
    idx, r, _ = _sis(X, y, 50)
    assert idx[0] == 10 and idx[1] == 200
    assert r[0] == r[1]
    assert 20 not in idx.tolist()
    _check(X, y, 50, idx, r)


def test_sis_hard_scales():
    """Features the FP32 pre-screen cannot take (out of its exponent range,
    subnormal, huge offsets, sparse zeros, one outlier) and an offset target:
    the selection is still the FP64 scan's."""
    rng = np.random.default_rng(9)
    n, nf = 200, 3000
    y = 1e8 + rng.normal(size=n)
    X = rng.normal(size=(nf, n)) + 0.05 * (y - 1e8)
    X[0:100] *= 1e30                         # above 2^61
    X[100:200] *= 1e-30                      # below 2^-60
    X[200:300] += 1e6                        # offset 1e6 sigma
    X[300:400] = np.where(rng.random((100, n)) < 0.9, 0.0, X[300:400])   # sparse
    X[400:500, 7] = 1e12                     # one outlier each
    X[500:510] = 5e-320 * rng.integers(1, 100, size=(10, n))            # subnormal
    X[510:520] = X[600:610]                  # duplicates
    X[520:530] = 0.0
    # values below 2^-60 beside values of order one (flushed by the pre-screen)
    X[530:540] = 1e-25 * rng.normal(size=(10, n)) + (rng.random((10, n)) < 0.5) + 0.02 * y
    for m in (1, 250, 1000, nf):
        idx, r, _ = _sis(X, y, m)
        _check(X, y, m, idx, r)


def test_sis_many_ties_at_cut():
    """More tied candidates than the rank sort takes: the one-block sort
    orders them by index."""
    rng = np.random.default_rng(3)
    n, nf = 32, 70000
    col = rng.normal(size=n)
    X = np.tile(col, (nf, 1))
    y = col + 0.1 * rng.normal(size=n)
    idx, r, _ = _sis(X, y, 100)
    np.testing.assert_array_equal(idx, np.arange(100, dtype=np.int32))
    assert np.all(r == r[0])


@pytest.mark.parametrize("n,nf,m", [(1001, 3000, 50), (2500, 700, 20), (1025, 333, 333),
                                    (3, 5000, 10), (4097, 65, 7)])
def test_sis_shapes(n, nf, m):
    """Rows that start on odd samples, rows of several staged segments, a
    last segment of one sample, three samples."""
    rng = np.random.default_rng(n)
    y = rng.normal(size=n)
    X = rng.normal(size=(nf, n)) + rng.uniform(0, 0.3, size=(nf, 1)) * y
    idx, r, _ = _sis(X, y, m)
    _check(X, y, m, idx, r)


def test_sis_unaligned_device_input():
    """X at an 8-byte (not 16-byte) offset: the register-staged pre-screen."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(17)
    n, nf, m = 1000, 5000, 100
    y = rng.normal(size=n)
    Xn = rng.normal(size=(nf, n)) + rng.uniform(0, 0.2, size=(nf, 1)) * y
    buf = torch.empty(nf * n + 1, dtype=torch.float64, device="cuda")
    buf[1:] = torch.from_numpy(Xn.reshape(-1)).cuda()
    Xv = buf[1:].view(nf, n)
    assert Xv.data_ptr() % 16 == 8
    idx, r, _ = _sis(Xv, torch.from_numpy(y).cuda(), m)
    idx2, r2, _ = _sis(Xn, y, m)
    np.testing.assert_array_equal(idx, idx2)
    np.testing.assert_array_equal(r, r2)
    _check(Xn, y, m, idx, r)


def test_sis_large_device_input():
    torch = pytest.importorskip("torch")
    p = make_problem(n_samples=500, n_sis=200000, seed=42, n_planted=3, sigma=0.05,
                     distinct=False, factors=4)
    X = torch.from_numpy(p.X).cuda()
    y = torch.from_numpy(p.y).cuda()
    idx, r, st = _sis(X, y, 1000)
    _check(p.X, p.y, 1000, idx, r)
    assert st["fp64_fallback_tuples"] < 5000


def test_sis_errors():
    X = np.ones((10, 5))
    y = np.arange(5.0)
    for precision in (l0.FP64, l0.MIXED_BF16X3):
        with l0.Handle(precision=precision) as h:
            with pytest.raises(l0.L0Error) as e:
                h.sis(X, y, 11)
            assert e.value.code == l0.EINVAL
            X2 = np.random.default_rng(0).normal(size=(10, 5))
            X2[3, 2] = np.nan
            with pytest.raises(l0.L0Error) as e:
                h.sis(X2, y, 3)
            assert e.value.code == l0.ENONFINITE
            y2 = y.copy()
            y2[1] = np.inf
            with pytest.raises(l0.L0Error) as e:
                h.sis(np.random.default_rng(0).normal(size=(10, 5)), y2, 3)
            assert e.value.code == l0.ENONFINITE
