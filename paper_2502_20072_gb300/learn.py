"""Training recipe of the learned pair scorer.

The learned d = 3 search ranks feature pairs with a small network and fits
only the triples reachable from the best pairs (the paper's search is
exhaustive, Sec. 2.4; the exhaustive search stays the reference).  The network
learns from the exhaustive search's own results: for every pair of a
training task, the log of its best completion min_k SSE(i, j, k) / S_yy,
z-scored within the task (only a pair's rank inside its task matters).

Everything numeric runs in the library's kernels (pair features and labels
from the tensor-core Gram, the network's BF16 forward/backward on the tensor
cores, Adam); this module only strings the calls together and shuffles rows.
"""

from __future__ import annotations

import time

from . import MIXED_BF16X3, Handle, Scorer


def pair_training_set(problems, device=0, seed=0):
    """Features [P, 8] and standardized labels [P] of every pair of every
    problem (one task each), concatenated and shuffled, as CUDA tensors."""
    import torch
    feats, labs = [], []
    with Handle(precision=MIXED_BF16X3, device=device) as h:
        for p in problems:
            f, lb = h.pair_data(p.X, p.y, labels=True, standardize=True)
            feats.append(f)
            labs.append(lb)
    F = torch.cat(feats)
    Y = torch.cat(labs)
    g = torch.Generator(device="cpu").manual_seed(int(seed))
    perm = torch.randperm(len(Y), generator=g).to(F.device)
    return F[perm].contiguous(), Y[perm].contiguous()


def train_scorer(F, Y, steps=3000, batch_rows=8192, lr=2e-3, seed=0, device=0, scorer=None):
    """Adam on (F, Y); returns (scorer, per-step losses, seconds)."""
    import torch
    s = scorer if scorer is not None else Scorer(device=device, seed=seed)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = s.train(F, Y, batch_rows=batch_rows, steps=steps, lr=lr)
    torch.cuda.synchronize()
    return s, losses, time.perf_counter() - t0
