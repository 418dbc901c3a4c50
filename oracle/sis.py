"""CPU FP64 oracle for SIS screening (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import this module.  It shares no code with the CUDA path.

Sure independence screening ranks candidate features by the magnitude of
their Pearson correlation with the target (paper Sec. 2.3, Eq. 1) and keeps
the best m for the l0 step.  Plain definitions:

* pearson(X, y): r_j = sum_i (x_ji - mean_j)(y_i - mean_y) /
  sqrt(sum_i (x_ji - mean_j)^2 * sum_i (y_i - mean_y)^2), two passes in FP64;
  a constant column has r = 0;
* sis(X, y, m): the m features with the largest |r_j|, ties broken by the
  smaller index.
"""

from __future__ import annotations

import numpy as np


def pearson(X, y):
    """Pearson r of every row of X (feature-major [n_feat, n]) with y."""
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    yc = y - y.mean()
    syy = float(yc @ yc)
    out = np.zeros(X.shape[0])
    for j in range(X.shape[0]):
        xc = X[j] - X[j].mean()
        sxx = float(xc @ xc)
        if sxx > 0.0 and syy > 0.0:
            out[j] = float(xc @ yc) / np.sqrt(sxx * syy)
    return out


def sis(X, y, m):
    """Indices (int32 [m]) and r of the m features with the largest |r|,
    ordered by |r| descending, ties by index."""
    r = pearson(X, y)
    order = sorted(range(len(r)), key=lambda j: (-abs(r[j]), j))[:m]
    idx = np.array(order, dtype=np.int32)
    return idx, r[idx]
