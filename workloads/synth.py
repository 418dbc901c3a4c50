"""Synthetic SISSO-shaped inputs (numpy, seeded).

Stand-ins for the paper's two data sets (thermal conductivity, Sec. 3.1.1;
Kaggle (Al,In,Ga)2O3 band gaps, Sec. 3.1.2), which are not used here.  The
recipe:

* primaries x_1..x_8 ~ U(0.5, 2.0) per sample;
* each candidate column f_j = x_a^p * x_b^q with a, b ~ U{1..8} and
  p, q ~ U{-2, -1, 0.5, 1, 2, 3} (with ``factors`` > 2 more factors drawn
  the same way: the two-factor family has only 1128 distinct non-constant
  columns, three factors 16,644, four factors 174,056);
* a column that is the constant 1 (a == b and p + q == 0) is redrawn;
* with ``distinct=True`` a column whose monomial (exponent vector) was already
  drawn is redrawn too, so no two columns are value duplicates;
* optionally a share of columns is replaced by near-collinear copies
  f_src * (1 + N(0, rel_noise^2)) of other columns;
* y = 0.1 + sum(beta * f_planted) + N(0, sigma^2), per task.

Columns are returned feature-major: ``X[j, i]`` is feature j of sample i, so
each column is contiguous.  Rows (samples) are grouped by task; task t owns
samples ``offsets[t] .. offsets[t+1]-1``.
"""

from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np

N_PRIMARIES = 8
EXPONENTS = (-2.0, -1.0, 0.5, 1.0, 2.0, 3.0)
# exponents times two, as integers, for exact monomial keys
_EXP2 = tuple(int(round(2 * e)) for e in EXPONENTS)


@dataclasses.dataclass
class Problem:
    X: np.ndarray                 # float64 [n_sis, n_total], feature-major
    y: np.ndarray                 # float64 [n_total]
    offsets: np.ndarray           # int64 [n_tasks + 1]
    planted: List[List[int]]      # per task: planted column indices (0-based, ascending)
    beta: List[List[float]]       # per task: planted coefficients (same order)
    intercept: float
    sigma: float
    spec: np.ndarray              # int64 [n_sis, 2 * factors]: (a, 2p, b, 2q[, c, 2r]), 0-based
    replaced: np.ndarray          # int64 [n_replaced, 2]: (column, source column)
    seed: int
    name: str = ""

    @property
    def n_tasks(self) -> int:
        return int(len(self.offsets) - 1)

    @property
    def n_sis(self) -> int:
        return int(self.X.shape[0])

    @property
    def n_total(self) -> int:
        return int(self.X.shape[1])


def _monomial_key(idx, e2) -> tuple:
    e = [0] * N_PRIMARIES
    for a, p2 in zip(idx, e2):
        e[a] += p2
    return tuple(e)


def _draw_spec(rng: np.random.Generator, n_sis: int, distinct: bool,
               factors: int = 2) -> np.ndarray:
    """Draw (a, 2p, b, 2q[, c, 2r]) for every column (primary indices first,
    then exponents, from the stream); constants always redrawn."""
    spec = np.zeros((n_sis, 2 * factors), dtype=np.int64)
    seen = set()
    tries = 0
    for j in range(n_sis):
        while True:
            tries += 1
            if tries > 200 * n_sis + 100000:
                raise ValueError("fewer distinct %d-factor monomials than n_sis=%d"
                                 % (factors, n_sis))
            idx = [int(rng.integers(0, N_PRIMARIES)) for _ in range(factors)]
            e2 = [_EXP2[int(rng.integers(0, len(_EXP2)))] for _ in range(factors)]
            key = _monomial_key(idx, e2)
            if all(v == 0 for v in key):
                continue
            if distinct and key in seen:
                continue
            break
        seen.add(key)
        row = []
        for a, p2 in zip(idx, e2):
            row += [a, p2]
        spec[j] = row
    return spec


def _columns(x: np.ndarray, spec: np.ndarray) -> np.ndarray:
    m = spec.shape[0]
    X = np.empty((m, x.shape[1]), dtype=np.float64)
    for j in range(m):
        v = np.power(x[int(spec[j, 0])], spec[j, 1] / 2.0)
        for f in range(1, spec.shape[1] // 2):
            v = v * np.power(x[int(spec[j, 2 * f])], spec[j, 2 * f + 1] / 2.0)
        X[j] = v
    return X


def make_problem(n_samples: Sequence[int] | int, n_sis: int, seed: int, *,
                 n_planted: int = 2, planted: Optional[Sequence[Sequence[int]]] = None,
                 beta: Optional[Sequence[Sequence[float]]] = None,
                 intercept: float = 0.1, sigma: float = 0.01,
                 distinct: bool = True, beta_range: float = 3.0,
                 replace_frac: float = 0.0, replace_rel_noise: float = 1e-4,
                 factors: int = 2, name: str = "") -> Problem:
    """Build one seeded problem.

    ``n_samples`` is an int (one task) or a list of per-task sample counts.
    Planted columns are drawn per task without replacement (and, with
    ``distinct``, are value-distinct by construction) unless given.
    """
    if isinstance(n_samples, (int, np.integer)):
        sizes = [int(n_samples)]
    else:
        sizes = [int(s) for s in n_samples]
    n_total = int(sum(sizes))
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.5, 2.0, size=(N_PRIMARIES, n_total))
    spec = _draw_spec(rng, n_sis, distinct, factors)
    X = _columns(x, spec)

    n_tasks = len(sizes)
    offsets = np.zeros(n_tasks + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)

    # near-collinear replacements (drawn before the planted columns so that
    # planted columns can avoid replaced ones)
    replaced = np.zeros((0, 2), dtype=np.int64)
    n_rep = int(round(replace_frac * n_sis))
    if n_rep > 0:
        cols = rng.permutation(n_sis)
        rep_cols = np.sort(cols[:n_rep])
        keep = np.sort(cols[n_rep:])
        pairs = []
        for j in rep_cols:
            src = int(keep[int(rng.integers(0, len(keep)))])
            X[j] = X[src] * (1.0 + replace_rel_noise * rng.standard_normal(n_total))
            pairs.append((int(j), src))
        replaced = np.asarray(pairs, dtype=np.int64)

    rep_set = set(int(j) for j in replaced[:, 0]) if len(replaced) else set()
    planted_out: List[List[int]] = []
    beta_out: List[List[float]] = []
    y = np.empty(n_total, dtype=np.float64)
    for t in range(n_tasks):
        if planted is not None:
            cols_t = sorted(int(c) for c in planted[t])
        else:
            pool = np.array([j for j in range(n_sis) if j not in rep_set])
            cols_t = sorted(int(c) for c in rng.choice(pool, size=n_planted, replace=False))
        if beta is not None:
            b_t = [float(v) for v in beta[t]]
        else:
            b_t = [float(v) for v in rng.uniform(-beta_range, beta_range, size=len(cols_t))]
        lo, hi = int(offsets[t]), int(offsets[t + 1])
        yt = np.full(hi - lo, intercept, dtype=np.float64)
        for c, bv in zip(cols_t, b_t):
            yt = yt + bv * X[c, lo:hi]
        if sigma > 0:
            yt = yt + sigma * rng.standard_normal(hi - lo)
        y[lo:hi] = yt
        planted_out.append(cols_t)
        beta_out.append(b_t)
    return Problem(X=np.ascontiguousarray(X), y=y, offsets=offsets, planted=planted_out,
                   beta=beta_out, intercept=intercept, sigma=sigma, spec=spec,
                   replaced=replaced, seed=seed, name=name)


# The five workloads: shapes, seeds and noise levels.  C1's planted
# columns f_17 and f_103 are read 1-based like x_1..x_8 (0-based 16, 102).
CONFIGS = {
    "C1": dict(n_samples=100, n_sis=200, n_dim=2, k=10, seed=1,
               planted=[[16, 102]], beta=[[2.3, -0.7]], sigma=0.01, distinct=True),
    "C2": dict(n_samples=1000, n_sis=1000, n_dim=3, k=100, seed=2,
               n_planted=3, sigma=0.01, distinct=True),
    "C3": dict(n_samples=[50, 120, 300, 500, 800, 1200, 1600, 2000], n_sis=2000,
               n_dim=(2, 3), k=100, seed=3, n_planted=2, sigma=0.02, distinct=False),
    "C4": dict(n_samples=5000, n_sis=400, n_dim=4, k=100, seed=4, n_planted=3,
               sigma=0.01, distinct=True, replace_frac=0.2, replace_rel_noise=1e-4),
    "C5": dict(n_samples=2000, n_sis=20000, n_dim=3, k=100, seed=5, n_planted=3,
               sigma=0.01, distinct=False),
    # the learned form's workload with distinct columns: four-factor
    # monomials (the two-factor family repeats each of its 1128 distinct
    # columns ~18 times at n_sis = 20000, and three factors give only 16,644
    # distinct columns); training instances use seeds 1000..1049 at
    # n_sis = 2000 of the same family
    "C5L": dict(n_samples=2000, n_sis=20000, n_dim=3, k=100, seed=5, n_planted=3,
                sigma=0.01, distinct=True, factors=4),
}
C5L_TRAIN = dict(n_samples=2000, n_sis=2000, n_planted=3, sigma=0.01, distinct=True, factors=4)
C5L_TRAIN_SEEDS = tuple(range(1000, 1050))


def make_config(name: str, **overrides) -> tuple:
    """Return (Problem, n_dim, k) for one of the five workloads."""
    cfg = dict(CONFIGS[name])
    cfg.update(overrides)
    n_dim = cfg.pop("n_dim")
    k = cfg.pop("k")
    prob = make_problem(name=name, **cfg)
    return prob, n_dim, k
