"""Pins for the CPU FP64 oracle against facts fixed by the paper and by
mathematics, independent of the oracle's own code.

* d = 1: SSE = S_yy (1 - r^2) with r the Pearson coefficient of Eq. 1.
* tiny inputs: exact rational normal equations (fractions.Fraction).
* random tuples: LAPACK least squares (numpy.linalg.lstsq) with an explicit
  intercept column.
* planted noise-free descriptor: exact recovery, ranks first.
* invariants: nesting, column permutation, affine column maps, target shift,
  0 <= SSE <= S_yy, orthogonal columns in closed form.
* enumeration: all C(m, n) combinations, the counts the paper prints.
* multi-task, rank deficiency and tie order.
"""

import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from workloads import make_problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed):
    return np.random.default_rng(seed)


def _pearson_eq1(x, y):
    """Eq. 1, written out: centred cross sum over the root of both centred
    sums of squares (two-pass means)."""
    xm = sum(x) / len(x)
    ym = sum(y) / len(y)
    num = sum((a - xm) * (b - ym) for a, b in zip(x, y))
    den = math.sqrt(sum((a - xm) ** 2 for a in x) * sum((b - ym) ** 2 for b in y))
    return num / den


# ----------------------------------------------------------------- d = 1 --
def test_d1_matches_pearson_closed_form():
    rng = _rng(11)
    n, m = 57, 23
    X = rng.normal(3.0, 1.5, size=(m, n))      # nonzero means: the intercept matters
    y = 2.0 + 0.3 * X[4] + rng.normal(size=n)
    res = oracle.fit(X, y, 1, m)
    yl = list(y)
    ym = sum(yl) / n
    syy = sum((v - ym) ** 2 for v in yl)
    expect = {}
    for j in range(m):
        r = _pearson_eq1(list(X[j]), yl)
        expect[j] = syy * (1.0 - r * r)
    got = {int(t[0]): s for t, s in zip(res["tuples"][0], res["score"][0])}
    assert set(got) == set(range(m))
    for j in range(m):
        assert abs(got[j] - expect[j]) <= 1e-13 * expect[j], (j, got[j], expect[j])
    # ranking is by SSE ascending, i.e. by |r| descending
    order = sorted(range(m), key=lambda j: (expect[j], j))
    assert [int(t[0]) for t in res["tuples"][0]] == order


# --------------------------------------------------- exact rational pins --
def _exact_sse(cols, y):
    """Exact SSE of the least-squares fit of y on [1, cols] by rational
    Gaussian elimination on the normal equations."""
    n = len(y)
    A = [[Fraction(1)] + [Fraction(c[i]) for c in cols] for i in range(n)]
    Y = [Fraction(v) for v in y]
    p = len(A[0])
    M = [[sum(A[i][a] * A[i][b] for i in range(n)) for b in range(p)] for a in range(p)]
    r = [sum(A[i][a] * Y[i] for i in range(n)) for a in range(p)]
    # Gauss-Jordan
    for c in range(p):
        piv = next(i for i in range(c, p) if M[i][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        r[c], r[piv] = r[piv], r[c]
        for i in range(p):
            if i != c and M[i][c] != 0:
                f = M[i][c] / M[c][c]
                M[i] = [a - f * b for a, b in zip(M[i], M[c])]
                r[i] = r[i] - f * r[c]
    beta = [r[i] / M[i][i] for i in range(p)]
    res = [Y[i] - sum(A[i][a] * beta[a] for a in range(p)) for i in range(n)]
    return sum(v * v for v in res)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_exact_rational_normal_equations(d):
    rng = _rng(100 + d)
    n, m = 9, 6
    X = rng.normal(size=(m, n))
    y = rng.normal(size=n)
    tuples = list(itertools.combinations(range(m), d))
    exact = {t: _exact_sse([X[j] for j in t], y) for t in tuples}
    res = oracle.fit(X, y, d, len(tuples))
    got = {tuple(int(v) for v in t): s for t, s in zip(res["tuples"][0], res["score"][0])}
    for t in tuples:
        e = float(exact[t])
        assert abs(got[t] - e) <= 1e-12 * e, (t, got[t], e)
    # exact order (the exact SSEs have no ties here)
    order = sorted(tuples, key=lambda t: (exact[t], t))
    assert [tuple(int(v) for v in t) for t in res["tuples"][0]] == order


# ------------------------------------------------------- LAPACK cross-check --
def test_lstsq_random_tuples():
    rng = _rng(7)
    n, m, d = 60, 14, 3
    X = rng.normal(size=(m, n))
    y = rng.normal(size=n) + X[2] - 0.5 * X[9]
    tuples = np.array(sorted({tuple(sorted(rng.choice(m, d, replace=False))) for _ in range(40)}),
                      dtype=np.int32)
    sse, rho = oracle.score(X, y, tuples)
    for q, t in enumerate(tuples):
        A = np.column_stack([np.ones(n)] + [X[j] for j in t])
        beta, *_ = np.linalg.lstsq(A, y, rcond=None)
        r = y - A @ beta
        ref = float(r @ r)
        assert abs(sse[q, 0] - ref) <= 1e-11 * ref, (t, sse[q, 0], ref)
        assert rho[q, 0] > 1e-3


# ------------------------------------------------------ planted recovery --
def test_planted_noise_free_recovered_first():
    prob = make_problem(80, 30, seed=21, n_planted=3, sigma=0.0, intercept=0.1)
    res = oracle.fit(prob.X, prob.y, 3, 5)
    planted = tuple(prob.planted[0])
    assert tuple(int(v) for v in res["tuples"][0, 0]) == planted
    syy = float(((prob.y - prob.y.mean()) ** 2).sum())
    assert res["score"][0, 0] <= 1e-20 * syy
    c = oracle.coefs(prob.X, prob.y, planted)
    assert abs(c[0] - 0.1) <= 1e-10 * max(1.0, abs(c[0]))
    for got, want in zip(c[1:], prob.beta[0]):
        assert abs(got - want) <= 1e-10 * max(1.0, abs(want))


def test_c1_shape_planted_pair_first_noise_free():
    prob = make_problem(100, 200, seed=1, planted=[[16, 102]], beta=[[2.3, -0.7]], sigma=0.0)
    res = oracle.fit(prob.X, prob.y, 2, 3)
    assert tuple(int(v) for v in res["tuples"][0, 0]) == (16, 102)


# ------------------------------------------------------------- invariants --
def _random_problem(seed, n=40, m=10):
    rng = _rng(seed)
    X = rng.normal(1.0, 2.0, size=(m, n))
    y = rng.normal(size=n) + 0.7 * X[1 % m] - 1.3 * X[5 % m] + 0.2 * X[7 % m]
    return X, y


def test_nesting_and_bounds():
    X, y = _random_problem(31)
    m = X.shape[0]
    syy = float(((y - y.mean()) ** 2).sum())
    t3 = np.array(list(itertools.combinations(range(m), 3)), dtype=np.int32)
    s3, _ = oracle.score(X, y, t3)
    t2 = {t: s for t, s in zip(itertools.combinations(range(m), 2),
                                oracle.score(X, y, np.array(list(itertools.combinations(range(m), 2)),
                                                            dtype=np.int32))[0][:, 0])}
    for q, t in enumerate(t3):
        s = s3[q, 0]
        assert -1e-12 * syy <= s <= syy * (1 + 1e-12)
        for drop in range(3):
            sub = tuple(int(v) for i, v in enumerate(t) if i != drop)
            assert s <= t2[sub] + 1e-12 * syy


def test_permutation_affine_and_shift_invariance():
    X, y = _random_problem(41)
    m = X.shape[0]
    rng = _rng(42)
    perm = rng.permutation(m)          # new column c holds old column perm[c]
    inv = np.argsort(perm)
    a = rng.uniform(0.5, 3.0, size=m) * rng.choice([-1.0, 1.0], size=m)
    b = rng.normal(size=m) * 10
    X2 = (X[perm] * a[perm, None]) + b[perm, None]
    y2 = y + 123.0
    tuples = np.array(list(itertools.combinations(range(m), 3)), dtype=np.int32)
    s1, _ = oracle.score(X, y, tuples)
    mapped = np.sort(inv[tuples], axis=1).astype(np.int32)
    s2, _ = oracle.score(X2, y2, mapped)
    np.testing.assert_allclose(s2[:, 0], s1[:, 0], rtol=1e-10)


def test_orthogonal_columns_closed_form():
    rng = _rng(51)
    n, m = 50, 6
    M = np.column_stack([np.ones(n), rng.normal(size=(n, m))])
    Q, _ = np.linalg.qr(M)
    cols = Q[:, 1:].T * rng.uniform(0.5, 4.0, size=(m, 1)) + rng.normal(size=(m, 1))
    y = rng.normal(size=n)
    yc = y - y.mean()
    syy = float(yc @ yc)
    tuples = np.array(list(itertools.combinations(range(m), 3)), dtype=np.int32)
    sse, _ = oracle.score(cols, y, tuples)
    for q, t in enumerate(tuples):
        expect = syy
        for j in t:
            a = cols[j] - cols[j].mean()
            expect -= float(a @ yc) ** 2 / float(a @ a)
        assert abs(sse[q, 0] - expect) <= 1e-12 * syy


# ----------------------------------------------------------- enumeration --
@pytest.mark.parametrize("m,d", [(7, 1), (7, 2), (8, 3), (9, 4)])
def test_enumerates_all_combinations(m, d):
    X, y = _random_problem(61 + m + d, n=20, m=m)
    k = math.comb(m, d)
    res = oracle.fit(X, y, d, k)
    got = [tuple(int(v) for v in t) for t in res["tuples"][0]]
    assert len(set(got)) == k
    assert set(got) == set(itertools.combinations(range(m), d))
    assert int(res["n_eligible"][0]) == k
    assert all(all(a < b for a, b in zip(t, t[1:])) for t in got)


def test_paper_tuple_counts_are_binomials():
    rows = []
    with open(os.path.join(GOLDEN, "paper_tuple_counts.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                parts = line.split()
                rows.append((int(parts[0]), int(parts[1]), int(parts[2])))
    assert rows
    for m, n, count in rows:
        assert math.comb(m, n) == count


def test_padding_when_fewer_eligible_than_k():
    X, y = _random_problem(71, n=12, m=4)
    res = oracle.fit(X, y, 2, 10)
    assert int(res["n_eligible"][0]) == 6
    assert np.all(res["tuples"][0, 6:] == -1)
    assert np.all(np.isinf(res["score"][0, 6:]))


# ------------------------------------------------------------- multi-task --
def test_per_task_equals_single_task_runs():
    prob = make_problem([30, 45, 25], 12, seed=81, n_planted=2, sigma=0.05)
    res = oracle.fit(prob.X, prob.y, 2, 8, offsets=prob.offsets)
    for t in range(3):
        lo, hi = prob.offsets[t], prob.offsets[t + 1]
        single = oracle.fit(prob.X[:, lo:hi], prob.y[lo:hi], 2, 8)
        np.testing.assert_array_equal(res["tuples"][t], single["tuples"][0])
        np.testing.assert_array_equal(res["score"][t], single["score"][0])


def test_shared_mode_two_identical_tasks():
    X, y = _random_problem(91, n=30, m=9)
    X2 = np.concatenate([X, X], axis=1)
    y2 = np.concatenate([y, y])
    off = np.array([0, 30, 60], dtype=np.int64)
    shared = oracle.fit(X2, y2, 2, 10, offsets=off, mode=oracle.SHARED)
    single = oracle.fit(X, y, 2, 10)
    np.testing.assert_array_equal(shared["tuples"][0], single["tuples"][0])
    # pooled mean SSE = 2 SSE / 60 = SSE / 30
    np.testing.assert_allclose(shared["score"][0], single["score"][0] / 30.0, rtol=1e-15)
    np.testing.assert_allclose(shared["rmse"][0], single["rmse"][0], rtol=1e-15)


def test_shared_mode_pools_sse_over_unequal_tasks():
    """SHARED score = sum_t SSE_t / sum_t n_t, each task with its own
    intercept and coefficients (Sec. 3.1), against LAPACK per task.  The
    tasks differ in size and in data, so the pooled mean differs from the
    mean of the per-task MSEs (a wrong weighting fails here)."""
    rng = _rng(93)
    sizes = [12, 31, 57]
    m, d = 8, 2
    X = rng.normal(1.0, 2.0, size=(m, sum(sizes)))
    y = np.empty(sum(sizes))
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    for t in range(3):
        lo, hi = off[t], off[t + 1]
        # a different descriptor per task and a task-dependent noise level
        y[lo:hi] = (t + 1.0) * X[t, lo:hi] - 0.5 * X[t + 3, lo:hi] \
            + (0.3 + 0.7 * t) * rng.standard_normal(hi - lo)
    k = math.comb(m, d)
    res = oracle.fit(X, y, d, k, offsets=off, mode=oracle.SHARED)
    assert res["tuples"].shape[0] == 1
    expect = {}
    mean_of_mse = {}
    for tup in itertools.combinations(range(m), d):
        sse = []
        for t in range(3):
            lo, hi = off[t], off[t + 1]
            A = np.column_stack([np.ones(hi - lo)] + [X[j, lo:hi] for j in tup])
            beta, *_ = np.linalg.lstsq(A, y[lo:hi], rcond=None)
            r = y[lo:hi] - A @ beta
            sse.append(float(r @ r))
        expect[tup] = sum(sse) / float(sum(sizes))
        mean_of_mse[tup] = sum(e / n for e, n in zip(sse, sizes)) / 3.0
    got = {tuple(int(v) for v in t): sc for t, sc in zip(res["tuples"][0], res["score"][0])}
    assert set(got) == set(expect)
    for tup, v in expect.items():
        assert abs(got[tup] - v) <= 1e-11 * v, (tup, got[tup], v)
        # the two weightings really differ on this input
        assert abs(mean_of_mse[tup] - v) > 1e-3 * v
    order = sorted(expect, key=lambda t: (expect[t], t))
    assert [tuple(int(v) for v in t) for t in res["tuples"][0]] == order
    np.testing.assert_allclose(res["rmse"][0], np.sqrt([expect[t] for t in order]), rtol=1e-11)


def test_shared_mode_ineligible_in_any_task():
    """A tuple rank deficient in one task only is ineligible for the pooled
    ranking (the shared descriptor must be fitted in every task)."""
    rng = _rng(94)
    sizes = [20, 25]
    m = 6
    X = rng.normal(size=(m, sum(sizes)))
    X[4, :20] = 3.0 * X[1, :20] - 2.0          # columns 1 and 4 collinear in task 0 only
    y = rng.normal(size=sum(sizes))
    off = np.array([0, 20, 45], dtype=np.int64)
    res = oracle.fit(X, y, 2, math.comb(m, 2), offsets=off, mode=oracle.SHARED)
    got = [tuple(int(v) for v in t) for t in res["tuples"][0] if t[0] >= 0]
    assert (1, 4) not in got
    assert len(got) == math.comb(m, 2) - 1
    per_task = oracle.fit(X, y, 2, math.comb(m, 2), offsets=off)
    t1 = [tuple(int(v) for v in t) for t in per_task["tuples"][1] if t[0] >= 0]
    assert (1, 4) in t1


def test_agreement_handles_padding():
    """Padded positions (+inf scores) form one tie group; a list that agrees
    on its finite part and pads the rest agrees, and no NaN is formed."""
    ref_t = np.array([[0, 1], [0, 2], [-1, -1], [-1, -1]])
    ref_s = np.array([1.0, 2.0, np.inf, np.inf])
    import warnings
    with warnings.catch_warnings():
        warnings.simplefilter("error")
        ok, msg = oracle.agreement(ref_t, ref_s, ref_t.copy())
        assert ok, msg
        bad = ref_t.copy()
        bad[2] = [1, 2]
        ok, _ = oracle.agreement(ref_t, ref_s, bad)
        assert not ok
        # a finite score next to an infinite one is never a tie
        ok, _ = oracle.agreement(ref_t[:3], ref_s[:3], np.array([[0, 1], [-1, -1], [0, 2]]))
        assert not ok


# ------------------------------------------------- rank deficiency, ties --
def test_exact_duplicate_is_ineligible_near_duplicate_is_not():
    X, y = _random_problem(101, n=40, m=8)
    Xd = X.copy()
    Xd[6] = Xd[2]                                   # exact duplicate
    rng = _rng(102)
    Xd[7] = Xd[3] * (1.0 + 1e-4 * rng.standard_normal(40))   # near duplicate
    k = math.comb(8, 2)
    res = oracle.fit(Xd, y, 2, k)
    got = [tuple(int(v) for v in t) for t in res["tuples"][0] if t[0] >= 0]
    assert (2, 6) not in got
    assert (3, 7) in got
    assert int(res["n_eligible"][0]) == k - 1


def test_ties_ordered_lexicographically():
    X, y = _random_problem(111, n=40, m=8)
    Xd = X.copy()
    Xd[5] = Xd[1]                                   # column 5 duplicates column 1
    res = oracle.fit(Xd, y, 2, math.comb(8, 2))
    tl = [tuple(int(v) for v in t) for t in res["tuples"][0]]
    sc = list(res["score"][0])
    for j in (0,):
        a, b = tl.index((j, 1)), tl.index((j, 5))
        assert sc[a] == sc[b]
        assert a < b
    a, b = tl.index((1, 7)), tl.index((5, 7))
    assert sc[a] == sc[b] and a < b


def test_agreement_helper():
    ref = [(0, 1), (0, 2), (1, 2), (2, 3)]
    sc = [1.0, 2.0, 2.0 + 1e-12, 3.0]
    ok, _ = oracle.agreement(ref, sc, [(0, 1), (1, 2), (0, 2), (2, 3)])
    assert ok
    ok, _ = oracle.agreement(ref, sc, [(0, 1), (1, 2), (0, 3), (2, 3)])
    assert not ok
    ok, _ = oracle.agreement(ref, sc, [(0, 1), (0, 2), (1, 2), (1, 3)],
                             score_fn=lambda ts: [3.0 for _ in ts])
    assert ok
