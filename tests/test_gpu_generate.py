"""On-the-fly feature generation fused with SIS on the GPU against the
oracle: validity of every candidate, the selected candidates and their r."""

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


def _compare(got, ref, tol=1e-11):
    idx, r, valid = got
    ridx, rr, rvalid = ref
    np.testing.assert_array_equal(valid.astype(bool), rvalid)
    # same selection up to groups of near-equal |r| (order decided by rounding)
    a = np.abs(rr)
    i = 0
    m = len(ridx)
    while i < m:
        j = i + 1
        while j < m and ridx[j] >= 0 and a[j - 1] - a[j] <= tol * a[j - 1]:
            j += 1
        if j < m:
            assert set(idx[i:j].tolist()) == set(ridx[i:j].tolist()), (i, j)
        i = j
    ok = ridx >= 0
    np.testing.assert_array_equal(idx >= 0, ok)
    order = {t: q for q, t in enumerate(ridx.tolist())}
    for q, t in enumerate(idx.tolist()):
        if t >= 0 and t in order:
            np.testing.assert_allclose(r[q], rr[order[t]], rtol=tol, atol=1e-14)


def test_generated_matches_oracle_all_operators():
    nc, n = 40, 100
    C = _children(nc, n, 1)
    rng = np.random.default_rng(2)
    y = np.log(np.abs(C[4])) * C[7] + 0.1 * rng.normal(size=n)
    ops, c1, c2 = _candidates(nc, 3)
    ref = og.sis_generated(C, ops, c1, c2, y, 200)
    with l0.Handle() as h:
        got = h.sis_generated(C, ops, c1, c2, y, 200)
    _compare(got, ref)
    assert 0 < ref[2].sum() < len(ops)            # both kinds present


def test_generated_bounds_and_few_valid():
    nc, n = 6, 50
    C = _children(nc, n, 4)
    y = np.random.default_rng(5).normal(size=n)
    ops, c1, c2 = _candidates(nc, 6)
    for lb, ub in ((1e-5, 1e8), (1.0, 50.0), (1e3, 1e4)):
        m = 20
        ref = og.sis_generated(C, ops, c1, c2, y, m, lb, ub)
        with l0.Handle() as h:
            got = h.sis_generated(C, ops, c1, c2, y, m, lb, ub)
        _compare(got, ref)
    # fewer valid candidates than m: -1 slots
    m = len(ops)
    ref = og.sis_generated(C, ops, c1, c2, y, m, 1e3, 1e4)
    with l0.Handle() as h:
        got = h.sis_generated(C, ops, c1, c2, y, m, 1e3, 1e4)
    assert (got[0] < 0).sum() == (ref[0] < 0).sum() > 0
    _compare(got, ref)


def test_generated_device_inputs_larger():
    torch = pytest.importorskip("torch")
    nc, n = 300, 150
    C = _children(nc, n, 7)
    rng = np.random.default_rng(8)
    prod = C[10] * C[20]
    y = prod / prod.std() + 0.05 * rng.normal(size=n)
    ops, c1, c2 = _candidates(nc, 9, binary_frac=0.25)
    ops = np.append(ops, np.int32(og.MUL))
    c1 = np.append(c1, np.int32(20))
    c2 = np.append(c2, np.int32(10))
    ref = og.sis_generated(C, ops, c1, c2, y, 500)
    with l0.Handle() as h:
        got = h.sis_generated(torch.from_numpy(C).cuda(), torch.from_numpy(ops).cuda(),
                              torch.from_numpy(c1).cuda(), torch.from_numpy(c2).cuda(),
                              torch.from_numpy(y).cuda(), 500)
    _compare(got, ref)
    # the planted product is the best candidate
    t = int(got[0][0])
    assert ops[t] == og.MUL and {int(c1[t]), int(c2[t])} == {10, 20}


def test_generated_rejects_bad_candidates():
    C = _children(5, 20, 10)
    y = np.arange(20.0)
    with l0.Handle() as h:
        for ops, c1, c2 in (([0], [0], [7]), ([14], [0], [1]), ([5], [-1], [0])):
            with pytest.raises(l0.L0Error) as e:
                h.sis_generated(C, ops, c1, c2, y, 1)
            assert e.value.code == l0.EINVAL
        # a unary operator ignores c2, whatever it holds
        idx, r, valid = h.sis_generated(C, [og.SQ, og.ADD], [1, 0], [99, 1], y, 2)
        ref = og.sis_generated(C, [og.SQ, og.ADD], [1, 0], [99, 1], y, 2)
        _compare((idx, r, valid), ref)
