"""The dimension loop on the GPU against the oracle: residuals of the best
models, SIS against several residuals with exclusions, and the whole loop
(SIS -> l0 -> residuals -> SIS ...)."""

import numpy as np
import pytest

import paper_2502_20072_gb300 as l0
from oracle import loop as oloop

pytestmark = pytest.mark.gpu


def _planted(seed, n=200, nf=3000):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(nf, n)) + rng.uniform(-3, 3, size=(nf, 1))
    a, b, c = 123, 2001, 777
    for j in range(40):                     # decoys crowding the first screening
        X[j] = X[a] + 0.4 * rng.normal(size=n)
    y = 2.0 * X[a] + 0.6 * X[b] - 0.4 * X[c] + 0.02 * rng.normal(size=n) + 5.0
    return X, y, (a, b, c)


def test_residuals_match_oracle():
    X, y, _ = _planted(1)
    models = np.array([[123, 5, 9], [2001, 777, 40], [0, 1, 2]], dtype=np.int32)
    with l0.Handle() as h:
        got = h.residuals(X, y, models)
        ref = oloop.residuals(X, y, models)
        np.testing.assert_allclose(got, ref, atol=1e-10 * np.abs(y - y.mean()).max())
        # one feature, four features
        for mm in ([[123]], [[1, 2, 3, 4]]):
            np.testing.assert_allclose(h.residuals(X, y, mm), oloop.residuals(X, y, mm),
                                       atol=1e-10 * np.abs(y - y.mean()).max())
        # a dependent column leaves the residual of the independent ones
        X2 = X.copy()
        X2[10] = 2.5 * X2[123] - 1.0
        np.testing.assert_allclose(h.residuals(X2, y, [[123, 10]]), oloop.residuals(X, y, [[123]]),
                                   atol=1e-9 * np.abs(y - y.mean()).max())


@pytest.mark.parametrize("R", [1, 3, 10])
def test_sis_multi_matches_oracle_and_paths_agree(R):
    X, y, _ = _planted(2)
    models = [[123], [40], [7], [2001], [777], [3], [4], [5], [6], [8]][:R]
    Y = oloop.residuals(X, y, models)
    ex = [123, 40, 7, 2500]
    m = 60
    with l0.Handle(precision=l0.FP64) as h:
        i64, r64 = h.sis_multi(X, Y, m, exclude=ex)
    with l0.Handle(precision=l0.MIXED_BF16X3) as h:
        i32, r32 = h.sis_multi(X, Y, m, exclude=ex)
        st = h.stats()
    np.testing.assert_array_equal(i32, i64)
    np.testing.assert_array_equal(r32, r64)
    ref_i, ref_r = oloop.sis_multi(X, Y, m, exclude=ex)
    np.testing.assert_array_equal(i64, ref_i)
    np.testing.assert_allclose(r64, ref_r, rtol=1e-11, atol=1e-13)
    assert not set(ex) & set(i64.tolist())
    assert m <= st["fp64_fallback_tuples"] <= 8 * m


def test_sis_multi_long_rows():
    """Rows longer than the fused multi-target pre-screen takes (one pass
    per target): same selection as the FP64 scan and the oracle."""
    X, y, _ = _planted(6, n=1500)
    Y = oloop.residuals(X, y, [[123], [2001], [40], [7]])
    with l0.Handle(precision=l0.FP64) as h:
        i64, r64 = h.sis_multi(X, Y, 30, exclude=[123])
    with l0.Handle(precision=l0.MIXED_BF16X3) as h:
        i32, r32 = h.sis_multi(X, Y, 30, exclude=[123])
    np.testing.assert_array_equal(i32, i64)
    np.testing.assert_array_equal(r32, r64)
    ref_i, ref_r = oloop.sis_multi(X, Y, 30, exclude=[123])
    np.testing.assert_array_equal(i64, ref_i)
    np.testing.assert_allclose(r64, ref_r, rtol=1e-11, atol=1e-13)


def test_sis_multi_errors():
    X, y, _ = _planted(3)
    nf = X.shape[0]
    with l0.Handle() as h:
        for kw in (dict(exclude=[5, 5]), dict(exclude=[-1]), dict(exclude=[nf])):
            with pytest.raises(l0.L0Error) as e:
                h.sis_multi(X, y, 10, **kw)
            assert e.value.code == l0.EINVAL
        with pytest.raises(l0.L0Error) as e:
            h.sis_multi(X, y, nf - 1, exclude=[1, 2])
        assert e.value.code == l0.EINVAL
        with pytest.raises(l0.L0Error) as e:
            h.sis_multi(X, np.tile(y, (17, 1)), 10)
        assert e.value.code == l0.EINVAL


@pytest.mark.parametrize("precision", [l0.FP64, l0.MIXED_BF16X3])
def test_dimension_loop_matches_oracle(precision):
    X, y, (a, b, c) = _planted(4)
    m, D, k, n_res = 12, 3, 10, 5
    ref = oloop.dimension_loop(X, y, m, D, k, n_res)
    with l0.Handle(precision=precision) as h:
        got = h.dimension_loop(X, y, m, D, k, n_res)
    for n in range(D):
        np.testing.assert_array_equal(got[n]["S"], ref[n]["S"])
        np.testing.assert_array_equal(got[n]["tuples"], ref[n]["tuples"])
        np.testing.assert_allclose(got[n]["rmse"], ref[n]["rmse"], rtol=1e-10)
    # the planted descriptor is the best 3-D model, found through the residuals
    assert tuple(got[2]["tuples"][0]) == tuple(sorted((a, b, c)))
    assert b not in got[0]["S"] or c not in got[0]["S"]


def test_dimension_loop_device_inputs():
    torch = pytest.importorskip("torch")
    X, y, _ = _planted(5, n=300, nf=20000)
    m, D, k, n_res = 20, 2, 8, 10
    ref = oloop.dimension_loop(X, y, m, D, k, n_res)
    with l0.Handle(precision=l0.MIXED_BF16X3) as h:
        got = h.dimension_loop(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), m, D, k,
                               n_res)
    for n in range(D):
        np.testing.assert_array_equal(got[n]["S"], ref[n]["S"])
        np.testing.assert_array_equal(got[n]["tuples"], ref[n]["tuples"])
        np.testing.assert_allclose(got[n]["rmse"], ref[n]["rmse"], rtol=1e-10)
