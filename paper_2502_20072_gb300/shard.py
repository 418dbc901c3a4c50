"""One l0 search over several GPUs (one process per GPU).

Every rank searches its own disjoint slice of the tuple space
(``Handle.fit_shard``: every n-th work item), then the ranks all-gather
their FP64 re-fitted candidate pools -- the single exchange step, at most
``MAX_POOL`` candidates of 16 bytes per rank -- and every rank ranks the
union (``Handle.merge_shards``).  The paper likewise spreads descriptors over
devices and gathers the selected models at the end (Sec. 3.2.1).
"""

from __future__ import annotations

import numpy as np

from . import MAX_POOL


def gather_candidates(keys, sse, bound, delta, group=None, device=None):
    """All-gather each rank's candidates.  Returns (keys, sse, bounds,
    deltas) of all ranks as numpy arrays (candidates concatenated in rank
    order).  Uses torch.distributed (NCCL with CUDA tensors when ``device``
    is a CUDA device, gloo with CPU tensors otherwise)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    dev = torch.device(device) if device is not None else torch.device("cpu")
    n = len(keys)
    if n > MAX_POOL:
        raise ValueError("more than MAX_POOL candidates")
    buf = torch.zeros((MAX_POOL + 1, 2), dtype=torch.float64)
    buf[0, 0] = float(n)
    buf[0, 1] = 0.0
    # keys travel bit-exactly through the float64 payload
    buf[1:n + 1, 0] = torch.from_numpy(np.asarray(keys, dtype=np.uint64).view(np.int64).copy()).view(torch.float64)
    buf[1:n + 1, 1] = torch.from_numpy(np.asarray(sse, dtype=np.float64))
    meta = torch.tensor([[bound, delta]], dtype=torch.float64)
    buf, meta = buf.to(dev), meta.to(dev)
    outs = [torch.empty_like(buf) for _ in range(world)]
    metas = [torch.empty_like(meta) for _ in range(world)]
    dist.all_gather(outs, buf, group=group)
    dist.all_gather(metas, meta, group=group)
    ks, ss = [], []
    for o in outs:
        o = o.cpu()
        c = int(o[0, 0].item())
        ks.append(o[1:c + 1, 0].contiguous().view(torch.int64).numpy().view(np.uint64))
        ss.append(o[1:c + 1, 1].numpy())
    mt = torch.cat([m.cpu() for m in metas]).numpy()
    return (np.concatenate(ks) if ks else np.empty(0, np.uint64),
            np.concatenate(ss) if ss else np.empty(0), mt[:, 0].copy(), mt[:, 1].copy())


def fit_sharded(handle, X, y, n_dim, k, group=None):
    """Sharded single-task search on the calling rank's GPU.  Returns
    (tuples [k, n_dim], rmse [k], certified) on every rank."""
    import torch
    import torch.distributed as dist
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    m, n = int(X.shape[0]), int(X.shape[1])
    keys, sse, bound, delta = handle.fit_shard(X, y, n_dim, k, rank, world)
    if world > 1:
        dev = ("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else None
        keys, sse, bounds, deltas = gather_candidates(
            keys, sse, bound, delta, group, device=torch.device(*dev) if dev else None)
    else:
        bounds, deltas = np.array([bound]), np.array([delta])
    return handle.merge_shards(m, n_dim, k, n, keys, sse, bounds, deltas)
