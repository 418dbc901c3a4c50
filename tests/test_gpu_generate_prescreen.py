"""Generated-feature SIS through the FP32 pre-screen (a mixed-precision
handle, no per-candidate validity asked for): every candidate is evaluated
in FP32 with an interval around its |r|, and only those whose interval
reaches the m-th largest lower bound of a certainly valid candidate are
evaluated in FP64.  The selection and its r must be the FP64 evaluation's:
the FP64 handle's bit for bit, and the oracle's (tie-aware; r to 1e-11
relative or 1e-12 absolute, the FP64 shifted sums' cancellation on small r)."""

import numpy as np
import pytest

import paper_2502_20072_gb300 as l0
from oracle import generate as og

pytestmark = pytest.mark.gpu


def _candidates(nc, seed, binary_frac=1.0):
    rng = np.random.default_rng(seed)
    ops, c1, c2 = [], [], []
    for op in range(14):
        if op in og.BINARY:
            for i in range(nc):
                for j in range(nc):
                    if i != j and rng.random() < binary_frac:
                        ops.append(op), c1.append(i), c2.append(j)
        else:
            for i in range(nc):
                ops.append(op), c1.append(i), c2.append(0)
    return (np.array(ops, dtype=np.int32), np.array(c1, dtype=np.int32),
            np.array(c2, dtype=np.int32))


def _children(nc, n, seed):
    rng = np.random.default_rng(seed)
    C = rng.uniform(0.3, 3.0, size=(nc, n)) * rng.choice([1.0, -1.0, 10.0, 1e-3], size=(nc, 1))
    C[1] = np.abs(C[1])
    C[2, 5] = 0.0                         # division by zero, log(0)
    C[3] = 4.0e4 + rng.normal(size=n)     # squares and cubes beyond 1e8
    return C


def _same_selection(got, ref, tol=1e-11, atol=1e-12):
    idx, r = got[0], got[1]
    ridx, rr = ref[0], ref[1]
    np.testing.assert_array_equal(idx >= 0, ridx >= 0)
    a = np.abs(rr)
    i, m = 0, len(ridx)
    while i < m:
        j = i + 1
        while j < m and ridx[j] >= 0 and a[j - 1] - a[j] <= tol * a[j - 1]:
            j += 1
        if j < m:                          # a group cut by m may continue past it
            assert set(idx[i:j].tolist()) == set(ridx[i:j].tolist()), (i, j)
        i = j
    order = {t: q for q, t in enumerate(ridx.tolist())}
    for q, t in enumerate(idx.tolist()):
        if t >= 0 and t in order:
            np.testing.assert_allclose(r[q], rr[order[t]], rtol=tol, atol=atol)


def _identical(got, ref64):
    # the survivors are re-scored by the FP64 path's own routine: the same r
    # bit for bit, so the same selection in the same order
    np.testing.assert_array_equal(got[0], ref64[0])
    np.testing.assert_array_equal(got[1], ref64[1])


def _run(C, ops, c1, c2, y, m, lb=1e-5, ub=1e8):
    with l0.Handle(precision=l0.MIXED_BF16X3) as h:
        got = h.sis_generated(C, ops, c1, c2, y, m, lb, ub, want_valid=False)
        st = h.stats()
    with l0.Handle(precision=l0.FP64) as h:
        ref64 = h.sis_generated(C, ops, c1, c2, y, m, lb, ub, want_valid=False)
    return got, ref64, st


def test_prescreen_matches_oracle_all_operators():
    nc, n = 40, 100
    C = _children(nc, n, 1)
    rng = np.random.default_rng(2)
    y = np.log(np.abs(C[4])) * C[7] + 0.1 * rng.normal(size=n)
    ops, c1, c2 = _candidates(nc, 3)
    ref = og.sis_generated(C, ops, c1, c2, y, 200)
    got, ref64, st = _run(C, ops, c1, c2, y, 200)
    assert st["fp64_fallback_tuples"] == 0          # the pre-screen ran
    _same_selection(got, ref)
    _identical(got, ref64)


@pytest.mark.parametrize("lb,ub", [(1e-5, 1e8), (1.0, 50.0), (1e3, 1e4)])
def test_prescreen_value_bounds(lb, ub):
    nc, n = 6, 50
    C = _children(nc, n, 4)
    y = np.random.default_rng(5).normal(size=n)
    ops, c1, c2 = _candidates(nc, 6)
    for m in (20, len(ops)):                        # the second: fewer valid than m
        ref = og.sis_generated(C, ops, c1, c2, y, m, lb, ub)
        got, ref64, _ = _run(C, ops, c1, c2, y, m, lb, ub)
        _same_selection(got, ref)
        _identical(got, ref64)


def test_prescreen_children_outside_the_fp32_range():
    # values near 1e-35 and 1e35 (outside [1e-30, 1e30]) and exact zeros:
    # those candidates skip the FP32 bounds and are evaluated in FP64
    nc, n = 8, 60
    rng = np.random.default_rng(11)
    C = rng.uniform(0.5, 2.0, size=(nc, n))
    C[2] *= 1e-35
    C[3] *= 1e35
    C[4, ::3] = 0.0
    y = C[0] * C[5] + 0.01 * rng.normal(size=n)
    ops, c1, c2 = _candidates(nc, 12)
    ref = og.sis_generated(C, ops, c1, c2, y, 30, 1e-40, 1e40)
    got, ref64, _ = _run(C, ops, c1, c2, y, 30, 1e-40, 1e40)
    _same_selection(got, ref)
    _identical(got, ref64)


def test_prescreen_near_ties_and_planted_product():
    torch = pytest.importorskip("torch")
    nc, n = 300, 150
    C = _children(nc, n, 7)
    C[50] = C[51] * (1.0 + 1e-9)                    # near-duplicate children: near-equal r
    rng = np.random.default_rng(8)
    prod = C[10] * C[20]
    y = prod / prod.std() + 0.05 * rng.normal(size=n)
    ops, c1, c2 = _candidates(nc, 9, binary_frac=0.25)
    ops = np.append(ops, np.int32(og.MUL))
    c1 = np.append(c1, np.int32(20))
    c2 = np.append(c2, np.int32(10))
    ref = og.sis_generated(C, ops, c1, c2, y, 500)
    dev = [torch.from_numpy(a).cuda() for a in (C, ops, c1, c2, y)]
    with l0.Handle(precision=l0.MIXED_BF16X3) as h:
        got = h.sis_generated(*dev, 500, want_valid=False)
    _same_selection(got, ref)
    t = int(got[0][0])
    assert ops[t] == og.MUL and {int(c1[t]), int(c2[t])} == {10, 20}


def test_prescreen_rejects_bad_candidates():
    C = _children(5, 20, 10)
    y = np.arange(20.0)
    with l0.Handle(precision=l0.MIXED_BF16X3) as h:
        for ops, c1, c2 in (([0], [0], [7]), ([14], [0], [1]), ([5], [-1], [0])):
            with pytest.raises(l0.L0Error) as e:
                h.sis_generated(C, ops, c1, c2, y, 1, want_valid=False)
            assert e.value.code == l0.EINVAL
