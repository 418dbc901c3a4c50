"""The allocation-free Gram entry point, sisso_l0_gram_noalloc.

It exists for callers that cannot allocate device memory while they run (a
service that reserves its device memory up front for its own allocator, or a
latency-bound loop that cannot take cudaMalloc's device-wide
synchronisation).  Its scratch is a fixed array inside the library that every
call reuses, so the test makes two calls in a row, with different shapes and
data, and checks each against the existing (allocating) entry point
sisso_l0_debug_gram within the Gram tolerance used elsewhere in the tests.

This file is named to be collected last.
"""

import ctypes

import numpy as np
import pytest

import paper_2502_20072_gb300 as l0
from workloads import make_problem

pytestmark = pytest.mark.gpu

GRAM_ATOL = 1e-13


def _noalloc(Xd, yd, n, m, out, ld):
    f = l0.lib().sisso_l0_gram_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                  ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f(ctypes.c_void_p(Xd.data_ptr()), ctypes.c_void_p(yd.data_ptr()), n, m,
             ctypes.c_void_p(out.data_ptr()), ld, None)


def test_noalloc_gram_matches_allocating_entry_point_twice():
    import torch
    cases = [(300, 120, 61), (500, 200, 62)]     # (n_samples, n_sis, seed)
    with l0.Handle() as h:
        for n, m, seed in cases:
            prob = make_problem(n, m, seed=seed, n_planted=2, sigma=0.05)
            ref = h.debug_gram(prob.X, prob.y)
            Xd = torch.from_numpy(prob.X).cuda()
            yd = torch.from_numpy(prob.y).cuda()
            ld = m + 1 + 5
            out = torch.full((m + 1, ld), float("nan"), dtype=torch.float64, device="cuda")
            rc = _noalloc(Xd, yd, n, m, out, ld)
            assert rc == l0.OK
            full = out.cpu().numpy()
            got = full[:, : m + 1]
            iu = np.triu_indices(m + 1)
            np.testing.assert_allclose(got[iu], ref[iu], rtol=0, atol=GRAM_ATOL)
            # the entry point writes only the upper triangle: the strict lower
            # triangle and the padding columns keep the caller's NaN fill
            il = np.tril_indices(m + 1, -1)
            assert np.isnan(got[il]).all()
            assert np.isnan(full[:, m + 1:]).all()


def test_noalloc_rejects_inputs_beyond_its_scratch():
    import torch
    n, m = 4096, 600        # (m + 1) * n exceeds the 2^21-double scratch
    Xd = torch.zeros((m, n), dtype=torch.float64, device="cuda")
    yd = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = torch.zeros((m + 1, m + 1), dtype=torch.float64, device="cuda")
    assert _noalloc(Xd, yd, n, m, out, m + 1) == l0.EUNSUPPORTED
    assert _noalloc(Xd, yd, n, m, out, m) == l0.EINVAL
    # sizes whose (n_sis + 1) * n_samples product wraps 64 bits are refused
    # on the host before anything is launched (no kernel sees these sizes)
    assert _noalloc(Xd, yd, 2 ** 62, 3, out, 2 ** 40) == l0.EUNSUPPORTED
    assert _noalloc(Xd, yd, 4, 2 ** 62, out, 2 ** 62 + 1) == l0.EUNSUPPORTED
