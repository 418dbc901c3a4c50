"""Shared helpers for the GPU parity tests."""

import numpy as np

import oracle
import paper_2502_20072_gb300 as l0

RMSE_RTOL = 1e-10     # FP64 re-fit vs oracle, relative
TIE_GAP = 1e-9        # adjacent oracle SSEs closer than this are a tie group


def score_fn(X, y, offsets=None, task=0):
    def f(tuples):
        if len(tuples) == 0:
            return []
        sse, _ = oracle.score(X, y, np.array(tuples, dtype=np.int32), offsets=offsets)
        return sse[:, task]
    return f


def check_against_oracle(X, y, d, k, offsets=None, **opts):
    """Run the library and the oracle on the same inputs; assert tuple
    agreement (tie rule) and RMSE agreement.  Returns (tuples, rmse, stats)."""
    ref = oracle.fit(X, y, d, k, offsets=offsets)
    with l0.Handle(**opts) as h:
        got_t, got_r = h.fit(X, y, d, k, offsets=offsets)
        st = h.stats()
    n_out = ref["tuples"].shape[0]
    for o in range(n_out):
        ok, msg = oracle.agreement(ref["tuples"][o], ref["score"][o], got_t[o], rel_gap=TIE_GAP,
                                   score_fn=score_fn(X, y, offsets, o))
        assert ok, "list %d: %s" % (o, msg)
        fin = np.isfinite(ref["rmse"][o])
        np.testing.assert_array_equal(np.isfinite(got_r[o]), fin)
        np.testing.assert_allclose(got_r[o][fin], ref["rmse"][o][fin], rtol=RMSE_RTOL, atol=0)
        assert np.all(got_t[o][~fin] == -1)
    return got_t, got_r, st
