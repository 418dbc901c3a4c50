"""CPU FP64 oracle for on-the-fly feature generation fused with SIS (test
infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import this module.  It shares no code with the CUDA path.

Feature creation (paper Sec. 2) applies operators to pairs of child
features; the GPU evaluates the values of candidate (operator, child pair)
combinations, applies the value-based rules and, for the last rung, feeds
the values straight into the SIS projection score instead of storing them
(Sec. 2.3; Sec. 3 runs the last rung on the fly).  The operator set is the
one of Sec. 3: addition, subtraction, multiplication, division, absolute
difference, logarithm, exponential, negative exponential, absolute value,
square root, cube root, square, cube and inverse.  Readings where the paper
gives no formula:

* a candidate is valid when every value is finite, the largest absolute
  value lies in [l_bound, u_bound] (Sec. 3: "maximum absolute value ...
  between 1e-5 and 1e8"), the values are not all equal, and they are not
  identical, sample by sample, to a child's values;
* unary operators read child 1 only;
* the score is Eq. 1's |r| against y; the m valid candidates of largest |r|
  are selected, ties to the smaller candidate index; slots beyond the valid
  count hold -1.
"""

from __future__ import annotations

import numpy as np

from oracle import sis as osis

ADD, SUB, MUL, DIV, ABS_DIFF, LOG, EXP, NEG_EXP, ABS, SQRT, CBRT, SQ, CUBE, INV = range(14)
BINARY = (ADD, SUB, MUL, DIV, ABS_DIFF)


def apply(op, a, b=None):
    """Values of op(a, b) (b unused for unary operators), FP64."""
    a = np.asarray(a, dtype=np.float64)
    with np.errstate(all="ignore"):
        if op == ADD:
            return a + b
        if op == SUB:
            return a - b
        if op == MUL:
            return a * b
        if op == DIV:
            return a / b
        if op == ABS_DIFF:
            return np.abs(a - b)
        if op == LOG:
            return np.log(a)
        if op == EXP:
            return np.exp(a)
        if op == NEG_EXP:
            return np.exp(-a)
        if op == ABS:
            return np.abs(a)
        if op == SQRT:
            return np.sqrt(a)
        if op == CBRT:
            return np.cbrt(a)
        if op == SQ:
            return a * a
        if op == CUBE:
            return a * a * a
        if op == INV:
            return 1.0 / a
    raise ValueError("unknown operator %d" % op)


def valid(v, a, b, l_bound, u_bound):
    """The value-based rules."""
    if not np.all(np.isfinite(v)):
        return False
    mx = float(np.max(np.abs(v)))
    if mx > u_bound or mx < l_bound:
        return False
    if np.all(v == v[0]):
        return False
    if np.array_equal(v, a) or (b is not None and np.array_equal(v, b)):
        return False
    return True


def evaluate(C, ops, c1, c2, l_bound=1e-5, u_bound=1e8):
    """Values [n_cand, n] and validity [n_cand] of the candidates."""
    C = np.asarray(C, dtype=np.float64)
    vals = np.empty((len(ops), C.shape[1]))
    ok = np.zeros(len(ops), dtype=bool)
    for t, (op, i, j) in enumerate(zip(ops, c1, c2)):
        a = C[i]
        b = C[j] if op in BINARY else None
        v = apply(op, a, b)
        vals[t] = v
        ok[t] = valid(v, a, b, l_bound, u_bound)
    return vals, ok


def sis_generated(C, ops, c1, c2, y, m, l_bound=1e-5, u_bound=1e8):
    """(idx [m] candidate indices, r [m], valid [n_cand]) of the screening of
    the generated candidates."""
    vals, ok = evaluate(C, ops, c1, c2, l_bound, u_bound)
    r = np.zeros(len(ops))
    if ok.any():
        r[ok] = osis.pearson(vals[ok], y)
    order = sorted(np.nonzero(ok)[0].tolist(), key=lambda t: (-abs(r[t]), t))[:m]
    idx = np.full(m, -1, dtype=np.int32)
    rr = np.zeros(m)
    idx[:len(order)] = order
    rr[:len(order)] = r[order]
    return idx, rr, ok
