"""Reader of the stored oracle top list of the d = 3 headline workload
(n = 1000, m = 1000, seed 2), written by tests/golden/make_c2_top.py."""

import os

import numpy as np

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c2_top128.txt")


def load():
    """(tuples [128, 3] int32, sse [128] float64, rmse [128] float64)."""
    rows = [ln.split() for ln in open(PATH) if ln.strip() and not ln.startswith("#")]
    a = np.array(rows, dtype=object)
    assert [int(v) for v in a[:, 0]] == list(range(len(rows)))
    t = a[:, 1:4].astype(np.int32)
    sse = a[:, 4].astype(np.float64)
    rmse = a[:, 5].astype(np.float64)
    return t, sse, rmse
