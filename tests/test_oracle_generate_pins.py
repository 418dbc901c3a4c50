"""Pins of the feature-generation oracle (CPU only): each operator against
Python's math module sample by sample, each value rule on a constructed
case, and the fused screening against explicitly built features."""

import math

import numpy as np

from oracle import generate as og
from oracle import sis as osis

_MATH = {
    og.ADD: lambda a, b: a + b, og.SUB: lambda a, b: a - b, og.MUL: lambda a, b: a * b,
    og.DIV: lambda a, b: a / b, og.ABS_DIFF: lambda a, b: abs(a - b),
    og.LOG: lambda a, b: math.log(a), og.EXP: lambda a, b: math.exp(a),
    og.NEG_EXP: lambda a, b: math.exp(-a), og.ABS: lambda a, b: abs(a),
    og.SQRT: lambda a, b: math.sqrt(a), og.CBRT: lambda a, b: math.copysign(abs(a) ** (1 / 3), a),
    og.SQ: lambda a, b: a * a, og.CUBE: lambda a, b: a * a * a, og.INV: lambda a, b: 1.0 / a,
}


def test_operators_match_math_module():
    rng = np.random.default_rng(0)
    a = rng.uniform(0.5, 3.0, size=50)
    b = rng.uniform(0.5, 3.0, size=50)
    for op, f in _MATH.items():
        got = og.apply(op, a, b)
        want = np.array([f(x, z) for x, z in zip(a, b)])
        np.testing.assert_allclose(got, want, rtol=1e-14, err_msg=str(op))
    # the cube root keeps the sign
    np.testing.assert_allclose(og.apply(og.CBRT, np.array([-8.0, 27.0])), [-2.0, 3.0])


def test_value_rules():
    a = np.array([1.0, 2.0, 3.0, 4.0])
    b = np.array([2.0, 1.0, 5.0, 3.0])
    assert og.valid(og.apply(og.ADD, a, b), a, b, 1e-5, 1e8)
    # non-finite: log of a negative value, division by zero
    assert not og.valid(og.apply(og.LOG, -a), -a, None, 1e-5, 1e8)
    z = np.array([1.0, 0.0, 2.0, 3.0])
    assert not og.valid(og.apply(og.DIV, a, z), a, z, 1e-5, 1e8)
    # bounds on the largest absolute value
    big = a * 1e7
    assert not og.valid(og.apply(og.MUL, big, a), big, a, 1e-5, 1e8)
    tiny = a * 1e-7
    assert not og.valid(og.apply(og.MUL, tiny, tiny), tiny, tiny, 1e-5, 1e8)
    assert og.valid(og.apply(og.MUL, tiny, a * 1e3), tiny, a * 1e3, 1e-5, 1e8)
    # constant
    assert not og.valid(og.apply(og.SUB, a, a - 1.0), a, a - 1.0, 1e-5, 1e8)
    # identical to a child: |x| of a positive feature
    assert not og.valid(og.apply(og.ABS, a), a, None, 1e-5, 1e8)
    assert og.valid(og.apply(og.ABS, a - 2.5), a - 2.5, None, 1e-5, 1e8)


def test_sis_generated_equals_screening_of_built_features():
    rng = np.random.default_rng(1)
    n, nc = 40, 12
    C = rng.uniform(0.2, 4.0, size=(nc, n))
    y = np.log(C[3]) * C[7] + 0.05 * rng.normal(size=n)
    ops, c1, c2 = [], [], []
    for op in range(14):
        for i in range(nc):
            if op in og.BINARY:
                for j in range(nc):
                    if i != j:
                        ops.append(op), c1.append(i), c2.append(j)
            else:
                ops.append(op), c1.append(i), c2.append(0)
    # a few invalid ones
    C[5, 4] = -1.0          # log, sqrt of a negative value
    idx, r, ok = og.sis_generated(C, ops, c1, c2, y, 25)
    built = []
    keep = []
    for t, (op, i, j) in enumerate(zip(ops, c1, c2)):
        f = _MATH[op]
        try:
            v = np.array([f(C[i, s], C[j, s]) for s in range(n)])
        except (ValueError, ZeroDivisionError):
            continue
        if not np.all(np.isfinite(v)) or np.all(v == v[0]):
            continue
        mx = np.abs(v).max()
        if mx > 1e8 or mx < 1e-5 or np.array_equal(v, C[i]) or (op in og.BINARY and np.array_equal(v, C[j])):
            continue
        built.append(v)
        keep.append(t)
    assert sorted(keep) == np.nonzero(ok)[0].tolist()
    rb = osis.pearson(np.array(built), y)
    order = sorted(range(len(keep)), key=lambda q: (-abs(rb[q]), keep[q]))[:25]
    assert list(idx) == [keep[q] for q in order]
    np.testing.assert_allclose(r, rb[order], rtol=1e-10)
    # the generating expression, log(x3) * x7, is not a single operator of two
    # children, but its factor log(x3) is among the best
    assert any(ops[t] == og.LOG and c1[t] == 3 for t in idx)


def test_fewer_valid_than_m():
    C = np.array([[1.0, 2.0, 3.0], [2.0, 2.0, 2.0]])
    y = np.array([1.0, 0.0, 2.0])
    idx, r, ok = og.sis_generated(C, [og.SQ, og.SQ, og.LOG], [0, 1, 1], [0, 0, 0], y, 3)
    assert list(ok) == [True, False, False]
    assert list(idx) == [0, -1, -1]


def test_bounds_are_inclusive():
    """max |value| equal to either bound is valid; just beyond is not."""
    a = np.array([1.0, 2.0, 4.0])
    for lb, ub, ok in ((4.0, 8.0, True), (1.0, 4.0, True), (np.nextafter(4.0, 5.0), 8.0, False),
                       (1.0, np.nextafter(4.0, 0.0), False)):
        assert og.valid(a, a + 1.0, None, lb, ub) is ok


def test_unary_operators_ignore_the_second_child():
    rng = np.random.default_rng(3)
    C = rng.uniform(0.5, 2.0, size=(4, 30))
    y = rng.normal(size=30)
    unary = [op for op in range(14) if op not in og.BINARY]
    i1, r1, v1 = og.sis_generated(C, unary, [1] * len(unary), [0] * len(unary), y, 5)
    i2, r2, v2 = og.sis_generated(C, unary, [1] * len(unary), [3] * len(unary), y, 5)
    assert list(i1) == list(i2) and list(v1) == list(v2)
    np.testing.assert_array_equal(r1, r2)
