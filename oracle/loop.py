"""CPU FP64 oracle for the dimension loop with multi-residual SIS (test
infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import this module.  It shares no code with the CUDA path.

Descriptor identification (paper Sec. 2, Fig. 1b) alternates SIS and l0 per
dimension: the subspace S receives, at dimension 1, the features with the
best projection score against the target and, at dimension n > 1, the best
against the residuals of the (n-1)-dimensional models; the l0 step then
searches all n-tuples of S.  Sec. 3 runs ten residuals per SIS iteration.
Readings where the paper gives no formula:

* residual of a model: y minus its least-squares fit with intercept
  (the fit of Sec. 2.4), for the ``n_res`` best models of the previous
  dimension;
* projection score against several residuals: the largest |r| (Eq. 1) over
  them; the reported r is the signed r of the first residual reaching it;
* a feature already in S is not selected again; ties in the score go to the
  smaller feature index;
* the l0 step at dimension n searches every n-tuple of the whole S
  (|S| = n m), ranked as in ``oracle.fit``.
"""

from __future__ import annotations

import numpy as np

import oracle
from oracle import sis as osis


def residuals(X, y, tuples):
    """[R, n] residuals y - (b0 + sum_i b_i x_{t_i}) of the least-squares fits
    of the R tuples (global feature indices, X feature-major [n_feat, n])."""
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    out = np.empty((len(tuples), len(y)))
    for r, tup in enumerate(tuples):
        tup = [int(t) for t in tup]
        beta = oracle.coefs(X, y, np.array(tup, dtype=np.int32))
        out[r] = y - beta[0] - X[tup].T @ beta[1:]
    return out


def sis_multi(X, targets, m, exclude=()):
    """The m features (not in ``exclude``) of largest max_r |r(x, targets[r])|,
    ordered by that score descending, ties by index.  Returns (idx int32 [m],
    signed r [m] of the first target reaching the maximum)."""
    targets = np.atleast_2d(np.asarray(targets, dtype=np.float64))
    R = np.stack([osis.pearson(X, t) for t in targets])       # [R, n_feat]
    best = np.argmax(np.abs(R), axis=0)
    r = R[best, np.arange(R.shape[1])]
    ex = set(int(e) for e in exclude)
    order = sorted((j for j in range(len(r)) if j not in ex), key=lambda j: (-abs(r[j]), j))[:m]
    idx = np.array(order, dtype=np.int32)
    return idx, r[idx]


def dimension_loop(X, y, m, D, k, n_res):
    """Per dimension n = 1..D: SIS of m new features (against y, then against
    the residuals of the min(n_res, k) best (n-1)-dimensional models), then the
    l0 search of all n-tuples of S.  Returns a list of dicts: S (global
    indices in selection order), tuples [k, n] (global indices, each tuple
    ascending), rmse [k]."""
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    S = []
    out = []
    prev = None
    for n in range(1, D + 1):
        if prev is None:
            targets = y[None, :]
        else:
            targets = residuals(X, y, prev[:min(n_res, len(prev))])
        new, _ = sis_multi(X, targets, m, exclude=S)
        S.extend(int(j) for j in new)
        Sa = np.array(S)
        fit = oracle.fit(X[Sa], y, n, k)
        tl = fit["tuples"][0]
        glob = np.sort(Sa[tl], axis=1)
        out.append(dict(S=Sa.copy(), tuples=glob, rmse=fit["rmse"][0].copy(),
                        local=tl.copy()))
        prev = glob
    return out
