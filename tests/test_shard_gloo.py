"""The sharded search's exchange step on CPU: two gloo ranks each hold the
candidates of their own slice of the tuple space (scored by the oracle), the
all-gather gives both ranks the union, and ranking the union reproduces the
exhaustive top k."""

import itertools
import math
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _lex_rank(t, m):
    """Lexicographic rank of the ascending tuple t among C(m, d) tuples."""
    d = len(t)
    r, prev = 0, -1
    for i, v in enumerate(t):
        for u in range(prev + 1, v):
            r += math.comb(m - 1 - u, d - 1 - i)
        prev = v
    return r


def _worker(rank, world, port, m, d, kpool, out_path):
    import torch.distributed as dist
    import oracle
    from workloads import make_problem
    from paper_2502_20072_gb300.shard import gather_candidates
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = make_problem(n_samples=60, n_sis=m, seed=42, n_planted=3, sigma=0.05)
    tuples = np.array(list(itertools.combinations(range(m), d)), dtype=np.int32)
    ranks = np.array([_lex_rank(t, m) for t in tuples], dtype=np.uint64)
    mine = (ranks % world) == rank
    sse, rho = oracle.score(p.X, p.y, tuples[mine])
    s = np.where(rho[:, 0] >= oracle.RHO_MIN, sse[:, 0], np.inf)
    order = np.lexsort((ranks[mine], s))[:kpool]
    bound = s[order[-1]] if len(order) == kpool else np.inf
    keys, ss, bounds, deltas = gather_candidates(ranks[mine][order], s[order], bound, 0.0)
    np.savez(out_path % rank, keys=keys, sse=ss, bounds=bounds, deltas=deltas)
    dist.destroy_process_group()


def test_two_rank_exchange_reproduces_exhaustive_top_k(tmp_path):
    import oracle
    from workloads import make_problem
    m, d, kpool, k = 13, 3, 24, 10
    world = 2
    out = str(tmp_path / "rank%d.npz")
    torch.multiprocessing.spawn(_worker, args=(world, _free_port(), m, d, kpool, out),
                                nprocs=world, join=True)
    r0, r1 = np.load(out % 0), np.load(out % 1)
    for key in ("keys", "sse", "bounds", "deltas"):
        np.testing.assert_array_equal(r0[key], r1[key])
    assert len(r0["keys"]) == 2 * kpool and len(set(r0["keys"].tolist())) == 2 * kpool
    # rank the union (SSE, lexicographic rank) and compare with the oracle
    order = np.lexsort((r0["keys"], r0["sse"]))[:k]
    p = make_problem(n_samples=60, n_sis=m, seed=42, n_planted=3, sigma=0.05)
    ref = oracle.fit(p.X, p.y, d, k)
    ref_ranks = [_lex_rank(t, m) for t in ref["tuples"][0]]
    np.testing.assert_array_equal(r0["keys"][order], np.array(ref_ranks, dtype=np.uint64))
    np.testing.assert_allclose(r0["sse"][order], ref["score"][0], rtol=1e-14)
    # every rank's bound covers the merged k-th score
    assert np.min(r0["bounds"]) >= r0["sse"][order][-1]
