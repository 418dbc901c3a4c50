"""CPU FP64 oracle for the SISSO l0-regularization step (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg (and its ``--impl reference`` arm) may import this package.  It shares no
code with the CUDA path: the arithmetic lives in ``oracle.c`` (plain C, FP64,
Householder QR per tuple, paper Sec. 2.4), compiled here with gcc.

Every function here is pinned by ``tests/test_oracle_pins.py``:
closed form at d = 1 (squared Pearson correlation, Eq. 1), exact rational
normal equations on tiny inputs, LAPACK least squares on random tuples,
exact recovery of a planted noise-free descriptor, invariants (nesting,
permutation and affine invariance, bounds, orthogonal columns) and the
tuple counts C(m, n) printed in Sec. 3.1.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lock = threading.Lock()
_lib = None

PER_TASK = 0
SHARED = 1
RHO_MIN = 1e-6  # rank-deficiency cut on min |R_jj| / ||a_j||


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            i64p = ctypes.POINTER(ctypes.c_int64)
            i32p = ctypes.POINTER(ctypes.c_int32)
            lib.oracle_l0_fit.argtypes = [dp, dp, i64p, ctypes.c_int, ctypes.c_int64,
                                          ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_double, ctypes.c_int, i32p, dp, dp, i64p]
            lib.oracle_l0_fit.restype = ctypes.c_int
            lib.oracle_l0_score.argtypes = [dp, dp, i64p, ctypes.c_int, ctypes.c_int64,
                                            ctypes.c_int, ctypes.c_int64, i32p, dp, dp,
                                            ctypes.c_int]
            lib.oracle_l0_score.restype = ctypes.c_int
            lib.oracle_l0_coefs.argtypes = [dp, dp, i64p, ctypes.c_int, ctypes.c_int64,
                                            ctypes.c_int, ctypes.c_int, i32p, dp]
            lib.oracle_l0_coefs.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _prep(X, y, offsets):
    X = np.ascontiguousarray(X, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    if offsets is None:
        offsets = np.array([0, X.shape[1]], dtype=np.int64)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    if X.ndim != 2 or y.shape != (X.shape[1],) or offsets[-1] != X.shape[1]:
        raise ValueError("X must be [n_sis, n_total], y [n_total], offsets[-1] == n_total")
    return X, y, offsets


def fit(X, y, n_dim, k, offsets=None, mode=PER_TASK, rho_min=RHO_MIN, n_threads=0):
    """Exhaustive search.  Returns dict(tuples [n_out,k,d], score [n_out,k],
    rmse [n_out,k], n_eligible [n_out]).  PER_TASK score = SSE_t;
    SHARED score = sum_t SSE_t / N."""
    X, y, offsets = _prep(X, y, offsets)
    n_tasks = len(offsets) - 1
    n_out = 1 if mode == SHARED else n_tasks
    tuples = np.empty((n_out, k, n_dim), dtype=np.int32)
    score = np.empty((n_out, k), dtype=np.float64)
    rmse = np.empty((n_out, k), dtype=np.float64)
    ne = np.empty(n_out, dtype=np.int64)
    rc = _load().oracle_l0_fit(_ptr(X, ctypes.c_double), _ptr(y, ctypes.c_double),
                               _ptr(offsets, ctypes.c_int64), n_tasks, X.shape[0], n_dim,
                               k, int(mode), float(rho_min), int(n_threads),
                               _ptr(tuples, ctypes.c_int32), _ptr(score, ctypes.c_double),
                               _ptr(rmse, ctypes.c_double), _ptr(ne, ctypes.c_int64))
    if rc != 0:
        raise ValueError("oracle_l0_fit failed with status %d" % rc)
    return dict(tuples=tuples, score=score, rmse=rmse, n_eligible=ne)


def score(X, y, tuples, offsets=None, n_threads=0):
    """SSE and rho of explicit tuples: returns (sse [n, n_tasks], rho [n, n_tasks])."""
    X, y, offsets = _prep(X, y, offsets)
    tuples = np.ascontiguousarray(tuples, dtype=np.int32)
    if tuples.ndim == 1:
        tuples = tuples[None, :]
    n, d = tuples.shape
    n_tasks = len(offsets) - 1
    sse = np.empty((n, n_tasks), dtype=np.float64)
    rho = np.empty((n, n_tasks), dtype=np.float64)
    if n == 0:
        return sse, rho
    rc = _load().oracle_l0_score(_ptr(X, ctypes.c_double), _ptr(y, ctypes.c_double),
                                 _ptr(offsets, ctypes.c_int64), n_tasks, X.shape[0], d, n,
                                 _ptr(tuples, ctypes.c_int32), _ptr(sse, ctypes.c_double),
                                 _ptr(rho, ctypes.c_double), int(n_threads))
    if rc != 0:
        raise ValueError("oracle_l0_score failed with status %d" % rc)
    return sse, rho


def coefs(X, y, tup, offsets=None, task=0):
    """Intercept and coefficients of one tuple on one task: [beta_0, beta_1..beta_d]."""
    X, y, offsets = _prep(X, y, offsets)
    tup = np.ascontiguousarray(tup, dtype=np.int32)
    out = np.empty(len(tup) + 1, dtype=np.float64)
    rc = _load().oracle_l0_coefs(_ptr(X, ctypes.c_double), _ptr(y, ctypes.c_double),
                                 _ptr(offsets, ctypes.c_int64), len(offsets) - 1, X.shape[0],
                                 len(tup), int(task), _ptr(tup, ctypes.c_int32),
                                 _ptr(out, ctypes.c_double))
    if rc != 0:
        raise ValueError("oracle_l0_coefs failed with status %d" % rc)
    return out


def agreement(ref_tuples, ref_score, got_tuples, rel_gap=1e-9, score_fn=None):
    """Top-k agreement under the tie rule.

    Reference positions are grouped into tie groups (adjacent reference
    scores within ``rel_gap`` relative).  Each group's tuple set must match.
    The last group may straddle position k: its slots may be filled by any
    tuple whose score (``score_fn(list_of_tuples) -> scores``, the oracle's
    own re-scoring) ties the group's score within ``rel_gap``.
    Returns (ok, message)."""
    ref_t = [tuple(int(v) for v in t) for t in ref_tuples]
    got_t = [tuple(int(v) for v in t) for t in got_tuples]
    s = np.asarray(ref_score, dtype=np.float64)
    k = len(ref_t)
    if len(got_t) != k:
        return False, "length %d != %d" % (len(got_t), k)
    def tied(a, b):
        # padding positions carry +inf: two equal non-finite scores are one
        # tie group; a finite score never ties a non-finite one
        if not (np.isfinite(a) and np.isfinite(b)):
            return bool(a == b)
        return abs(a - b) <= rel_gap * max(abs(a), abs(b))

    groups = []
    start = 0
    for i in range(1, k + 1):
        if i == k or not tied(s[i], s[i - 1]):
            groups.append((start, i))
            start = i
    for (a, b) in groups:
        rs = set(ref_t[a:b])
        gs = set(got_t[a:b])
        if rs == gs:
            continue
        if b == k and score_fn is not None and np.isfinite(s[a]):
            extra = sorted(gs - rs)
            sc = np.asarray(score_fn(extra), dtype=np.float64)
            lo, hi = s[a:b].min(), s[a:b].max()
            tol = rel_gap * max(abs(lo), abs(hi))
            if np.all((sc >= lo - tol) & (sc <= hi + tol)):
                continue
        return False, "group %d..%d differs: ref %s got %s" % (
            a, b, sorted(rs - gs)[:5], sorted(gs - rs)[:5])
    return True, "ok"
