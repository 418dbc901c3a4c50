"""CPU FP64 oracle for the learned proposal scorer (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import this module.  It shares no code with the CUDA path.

The paper's l0 step scores every n-tuple exhaustively (Sec. 2.4).  The
learned form ranks the (d-1)-subsets of a d = 3 search -- feature pairs --
with a small network and fits exactly only the triples reachable from the
best-ranked pairs.  This module states every piece of that from its plain
definition:

* pair features of (i, j), i < j, from the centred, unit-norm columns z and
  the centred, unit-norm target u:  r_i = z_i.u, r_j = z_j.u (Pearson r,
  Eq. 1), C_ij = z_i.z_j, rho_j.i = corr(z_j, u - r_i z_i) (the correlation
  of f_j with the residual of the one-feature fit on f_i), rho_i.j likewise,
  and log(max(SSE(i, j) / S_yy, LABEL_FLOOR)) / 8, the log residual fraction
  1 - R2_ij of the two-feature least-squares fit (Householder QR through
  ``oracle.score``);
* the label of a pair: the best completion, min over k not in {i, j} of
  SSE(i, j, k) / S_yy over eligible triples, as log(clip(., LABEL_FLOOR, 1))
  (0 when no completion is eligible: the worst possible fit);
* a 6-256-256-1 ReLU network whose matrix products take BF16 operands with
  exact (here FP64) accumulation, FP32 master weights, squared-error loss,
  its gradient and an Adam step;
* the exact search restricted to the triples reachable from a pair list.

Rounding points of the network (the same ones the GPU kernels use): the
features, the weights W1, W2, w3, the hidden activations h1, h2 and the
back-propagated dh2 are rounded to BF16 (round to nearest, ties to even);
everything else is exact arithmetic here.
"""

from __future__ import annotations

import numpy as np

from . import RHO_MIN, score as _score

N_IN, N_H = 6, 256
LABEL_FLOOR = 1e-12
N_PARAMS = N_H * N_IN + N_H + N_H * N_H + N_H + N_H + 1


# ------------------------------------------------------------------ BF16 --
def bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as float64.

    BF16 keeps the top 16 bits of an IEEE single: round the single's bit
    pattern at bit 16.  Inputs are first rounded to single precision."""
    a = np.asarray(x, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    out = r.view(np.float32).astype(np.float64)
    nan = np.isnan(a)
    if np.any(nan):
        out = np.where(nan, np.nan, out)
    return out


# ----------------------------------------------------------- pair ranks --
def pair_rank(i, j):
    """Colex rank of the pair i < j: j (j - 1) / 2 + i."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    return j * (j - 1) // 2 + i


def all_pairs(m):
    """Every pair (i, j), i < j, in colex order: array [C(m, 2), 2]."""
    out = np.empty((m * (m - 1) // 2, 2), dtype=np.int32)
    p = 0
    for j in range(1, m):
        out[p:p + j, 0] = np.arange(j)
        out[p:p + j, 1] = j
        p += j
    return out


# -------------------------------------------------------- pair features --
def _unit_columns(X, y):
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    Z = X - X.mean(axis=1, keepdims=True)
    Z = Z / np.linalg.norm(Z, axis=1, keepdims=True)
    u = y - y.mean()
    syy = float(u @ u)
    u = u / np.sqrt(syy)
    return Z, u, syy


def pair_features(X, y, pairs=None):
    """Features [P, 6] = (r_i, r_j, C_ij, rho_j.i, rho_i.j, log(1 - R2_ij) / 8)
    of the pairs (default: all pairs in colex order) of one task."""
    m = np.asarray(X).shape[0]
    if pairs is None:
        pairs = all_pairs(m)
    pairs = np.asarray(pairs, dtype=np.int32)
    Z, u, syy = _unit_columns(X, y)
    r = Z @ u
    out = np.empty((len(pairs), N_IN), dtype=np.float64)
    for q, (i, j) in enumerate(pairs):
        ei = u - r[i] * Z[i]            # residual of y after the fit on f_i
        ej = u - r[j] * Z[j]
        ni, nj = np.linalg.norm(ei), np.linalg.norm(ej)
        out[q, 0] = r[i]
        out[q, 1] = r[j]
        out[q, 2] = Z[i] @ Z[j]
        out[q, 3] = (Z[j] @ ei) / ni if ni > 0 else 0.0
        out[q, 4] = (Z[i] @ ej) / nj if nj > 0 else 0.0
    sse, _ = _score(X, y, pairs)
    out[:, 5] = np.log(np.maximum(sse[:, 0] / syy, LABEL_FLOOR)) / 8.0
    return out


def best_completion(X, y, pairs=None):
    """Per pair: min over k not in the pair of SSE(i, j, k) / S_yy over the
    eligible triples (rho >= RHO_MIN), +inf when none is eligible."""
    m = np.asarray(X).shape[0]
    if pairs is None:
        pairs = all_pairs(m)
    pairs = np.asarray(pairs, dtype=np.int32)
    _, _, syy = _unit_columns(X, y)
    best = np.full(len(pairs), np.inf)
    for q, (i, j) in enumerate(pairs):
        ks = np.array([k for k in range(m) if k != i and k != j], dtype=np.int32)
        tri = np.sort(np.stack([np.full(len(ks), i), np.full(len(ks), j), ks], axis=1), axis=1)
        sse, rho = _score(X, y, tri.astype(np.int32))
        ok = rho[:, 0] >= RHO_MIN
        if np.any(ok):
            best[q] = float(np.min(sse[ok, 0])) / syy
    return best


def labels(X, y, pairs=None):
    """log(clip(best completion, LABEL_FLOOR, 1)) of each pair."""
    b = best_completion(X, y, pairs)
    return np.log(np.clip(b, LABEL_FLOOR, 1.0))


# ------------------------------------------------------------ the network --
def unpack(flat):
    """Split the flat parameter vector: W1 [256,6], b1 [256], W2 [256,256]
    (row = output unit), b2 [256], w3 [256], b3 [1]."""
    flat = np.asarray(flat, dtype=np.float64)
    assert flat.size == N_PARAMS
    o = 0
    parts = {}
    for name, shape in (("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)),
                        ("b2", (N_H,)), ("w3", (N_H,)), ("b3", (1,))):
        n = int(np.prod(shape))
        parts[name] = flat[o:o + n].reshape(shape)
        o += n
    return parts


def pack(parts):
    return np.concatenate([np.asarray(parts[n], dtype=np.float64).ravel()
                           for n in ("W1", "b1", "W2", "b2", "w3", "b3")])


def forward(flat, feats, round_bf16=True):
    """Network output for each row of feats [B, 6] and the intermediates."""
    p = unpack(flat)
    rd = bf16 if round_bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    x = rd(feats)
    W1, W2, w3 = rd(p["W1"]), rd(p["W2"]), rd(p["w3"])
    pre1 = x @ W1.T + p["b1"]
    h1 = rd(np.maximum(pre1, 0.0))
    pre2 = h1 @ W2.T + p["b2"]
    h2 = rd(np.maximum(pre2, 0.0))
    out = h2 @ w3 + p["b3"][0]
    return out, dict(x=x, W1=W1, W2=W2, w3=w3, pre1=pre1, h1=h1, pre2=pre2, h2=h2)


def loss_and_grad(flat, feats, target, round_bf16=True):
    """Mean squared error over the batch and its gradient (flat vector)."""
    rd = bf16 if round_bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    target = np.asarray(target, dtype=np.float64)
    B = len(target)
    out, c = forward(flat, feats, round_bf16)
    diff = out - target
    loss = float(np.mean(diff * diff))
    g = 2.0 * diff / B
    db3 = np.array([g.sum()])
    dw3 = c["h2"].T @ g
    dh2 = rd(g[:, None] * c["w3"][None, :] * (c["pre2"] > 0.0))
    db2 = dh2.sum(axis=0)
    dW2 = dh2.T @ c["h1"]
    dh1 = dh2 @ c["W2"]
    dpre1 = dh1 * (c["pre1"] > 0.0)
    dW1 = dpre1.T @ c["x"]
    db1 = dpre1.sum(axis=0)
    return loss, pack(dict(W1=dW1, b1=db1, W2=dW2, b2=db2, w3=dw3, b3=db3))


def adam_step(flat, grad, m1, m2, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t counts from 1): returns (new params, m1, m2)."""
    m1 = beta1 * m1 + (1.0 - beta1) * grad
    m2 = beta2 * m2 + (1.0 - beta2) * grad * grad
    mh = m1 / (1.0 - beta1 ** t)
    vh = m2 / (1.0 - beta2 ** t)
    return flat - lr * mh / (np.sqrt(vh) + eps), m1, m2


# ------------------------------------------- proposal-restricted search --
def reachable_triples(pairs, m):
    """Sorted, de-duplicated triples {i, j, k}, k not in {i, j}, over the pairs."""
    s = set()
    for i, j in np.asarray(pairs, dtype=np.int64):
        for k in range(m):
            if k != i and k != j:
                s.add(tuple(sorted((int(i), int(j), k))))
    if not s:
        return np.empty((0, 3), dtype=np.int32)
    return np.array(sorted(s), dtype=np.int32)


def fit_pairs(X, y, pairs, k):
    """Top k of the eligible reachable triples by (SSE, lexicographic order).
    Returns dict(tuples [k, 3] (-1 padded), score (SSE), rmse)."""
    X = np.asarray(X, dtype=np.float64)
    m, n = X.shape
    tri = reachable_triples(pairs, m)
    sse, rho = _score(X, y, tri) if len(tri) else (np.empty((0, 1)), np.empty((0, 1)))
    ok = rho[:, 0] >= RHO_MIN
    tri, s = tri[ok], sse[ok, 0]
    order = np.lexsort((tri[:, 2], tri[:, 1], tri[:, 0], s))[:k]
    out_t = np.full((k, 3), -1, dtype=np.int32)
    out_s = np.full(k, np.inf)
    out_t[:len(order)] = tri[order]
    out_s[:len(order)] = s[order]
    return dict(tuples=out_t, score=out_s, rmse=np.sqrt(out_s / n))
