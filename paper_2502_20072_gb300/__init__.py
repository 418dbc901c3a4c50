"""GB300 (sm_103a) l0-regularization step of SISSO: Python binding.

Thin ctypes layer over the C ABI in ``include/sisso_l0.h``: it only
marshals arguments.  Every step of the search runs in the library's CUDA
kernels; when the library cannot be loaded this module raises instead of
falling back to anything else.

    import paper_2502_20072_gb300 as l0
    with l0.Handle(precision=l0.MIXED_BF16X3) as h:
        tuples, rmse = h.fit(X, y, n_dim=3, k=100)

X is FP64 feature-major [n_sis, n_total] (each column contiguous), y is FP64
[n_total]; both may be torch CUDA tensors, torch CPU tensors or numpy arrays.
"""

from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

FP64 = 0
MIXED_BF16X3 = 1
MIXED_TF32 = 2
PER_TASK = 0
SHARED = 1
MAX_DIM = 8

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENONFINITE, EUNSUPPORTED = range(7)
_NAMES = {1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ENONFINITE",
          6: "EUNSUPPORTED"}


class L0Error(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (_NAMES.get(code, "?"), code, msg))
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_int32), ("device", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("precision", ctypes.c_int32),
                ("task_mode", ctypes.c_int32), ("candidate_pool", ctypes.c_int32),
                ("max_candidate_pool", ctypes.c_int32),
                ("fp32_fallback_pivot_ratio", ctypes.c_double),
                ("rank_deficient_pivot_ratio", ctypes.c_double),
                ("autotune", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("autotune_cache_path", ctypes.c_char_p),
                ("timeout_seconds", ctypes.c_double),
                ("fp64_rerun_uncertified", ctypes.c_int32), ("tuple_kernel", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("n_dim", ctypes.c_int32), ("k", ctypes.c_int32),
                ("out_tuples", ctypes.c_void_p), ("out_rmse", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_int32), ("candidate_pool", ctypes.c_int32),
                ("pool_enlargements", ctypes.c_int32), ("certified", ctypes.c_int32),
                ("tuple_fits", ctypes.c_uint64), ("fp64_fallback_tuples", ctypes.c_uint64),
                ("n_eligible_min", ctypes.c_int64), ("max_pool_rel_error", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("graph_replayed", ctypes.c_int32),
                ("tuned_items_factor", ctypes.c_int32), ("tuned_ctas_per_sm", ctypes.c_int32),
                ("fp64_rerun", ctypes.c_int32),
                ("ms_prep", ctypes.c_double), ("ms_gram", ctypes.c_double),
                ("ms_tuple", ctypes.c_double), ("ms_merge", ctypes.c_double),
                ("ms_refit", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("ms_tuple_kernel", ctypes.c_double), ("proposal_pairs", ctypes.c_int64),
                ("tuple_kernel", ctypes.c_int32), ("band_pass", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "struct_size"}


_lib = None
_lock = threading.Lock()

# entry points declared in include/sisso_l0.h (checked by the tests)
EXPORTS = ("sisso_l0_default_options", "sisso_l0_create", "sisso_l0_fit", "sisso_l0_fit_multi",
           "sisso_l0_get_stats", "sisso_l0_last_error", "sisso_l0_destroy",
           "sisso_l0_count_tuples", "sisso_l0_debug_unrank", "sisso_l0_debug_gram",
           "sisso_l0_scorer_create", "sisso_l0_scorer_destroy", "sisso_l0_scorer_last_error",
           "sisso_l0_scorer_set_params", "sisso_l0_scorer_get_params",
           "sisso_l0_scorer_loss_grad", "sisso_l0_scorer_train", "sisso_l0_scorer_predict",
           "sisso_l0_pair_data", "sisso_l0_fit_pairs", "sisso_l0_fit_learned",
           "sisso_l0_fit_shard", "sisso_l0_merge_shards", "sisso_l0_measure_peaks",
           "sisso_l0_sis", "sisso_l0_sis_multi", "sisso_l0_residuals",
           "sisso_l0_dimension_loop", "sisso_l0_sis_generated")

MAX_POOL = 2048

SCORER_PARAMS = 67841
PAIR_FEATURES_LD = 8


def debug_fail_allocation(after):
    """Test hook: the calling thread's device allocation number `after`
    (counting from 0) inside the library reports out-of-memory; after < 0
    turns it off."""
    lib().sisso_l0_debug_fail_allocation(int(after))


def library_path() -> str:
    return _build.LIB


def lib():
    """Load the CUDA library (building it first when it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            path = _build.build()
        L = ctypes.CDLL(path)
        vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
        L.sisso_l0_default_options.argtypes = [ctypes.POINTER(Options)]
        L.sisso_l0_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Options)]
        L.sisso_l0_fit.argtypes = [vp, dp, dp, ctypes.POINTER(ctypes.c_int64), i32, i64, i32,
                                   i32, vp, vp]
        L.sisso_l0_fit_multi.argtypes = [vp, dp, dp, ctypes.POINTER(ctypes.c_int64), i32, i64,
                                         ctypes.POINTER(Request), i32]
        L.sisso_l0_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
        L.sisso_l0_set_timeout.argtypes = [vp, ctypes.c_double]
        L.sisso_l0_debug_fail_allocation.argtypes = [i64]
        L.sisso_l0_last_error.argtypes = [vp]
        L.sisso_l0_last_error.restype = ctypes.c_char_p
        L.sisso_l0_destroy.argtypes = [vp]
        L.sisso_l0_destroy.restype = None
        L.sisso_l0_count_tuples.argtypes = [i64, i32]
        L.sisso_l0_count_tuples.restype = ctypes.c_uint64
        L.sisso_l0_debug_unrank.argtypes = [vp, i64, i32, vp, i64, vp]
        L.sisso_l0_debug_gram.argtypes = [vp, dp, dp, ctypes.POINTER(ctypes.c_int64), i32, i64,
                                          i32, vp]
        fp = ctypes.c_float
        L.sisso_l0_scorer_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.c_uint64]
        L.sisso_l0_scorer_destroy.argtypes = [vp]
        L.sisso_l0_scorer_destroy.restype = None
        L.sisso_l0_scorer_last_error.argtypes = [vp]
        L.sisso_l0_scorer_last_error.restype = ctypes.c_char_p
        L.sisso_l0_scorer_set_params.argtypes = [vp, vp, i64]
        L.sisso_l0_scorer_get_params.argtypes = [vp, vp, i64]
        L.sisso_l0_scorer_loss_grad.argtypes = [vp, vp, vp, i64, vp, vp]
        L.sisso_l0_scorer_train.argtypes = [vp, vp, vp, i64, i32, i32, fp, vp]
        L.sisso_l0_scorer_predict.argtypes = [vp, vp, i64, vp]
        L.sisso_l0_pair_data.argtypes = [vp, dp, dp, i64, i64, vp, vp, i32]
        L.sisso_l0_fit_pairs.argtypes = [vp, dp, dp, i64, i64, vp, i64, i32, vp, vp]
        L.sisso_l0_fit_learned.argtypes = [vp, vp, dp, dp, i64, i64, i32, ctypes.c_double, vp, vp]
        L.sisso_l0_fit_shard.argtypes = [vp, dp, dp, i64, i64, i32, i32, i32, i32, vp, vp, vp,
                                         vp, vp]
        L.sisso_l0_merge_shards.argtypes = [vp, i64, i32, i32, i64, vp, vp, i64, vp, vp, i32, vp,
                                            vp, vp]
        L.sisso_l0_measure_peaks.argtypes = [i32, vp]
        L.sisso_l0_sis.argtypes = [vp, dp, dp, i64, i64, i32, vp, vp]
        L.sisso_l0_sis_multi.argtypes = [vp, dp, dp, i32, i64, i64, i32, vp, i64, vp, vp]
        L.sisso_l0_residuals.argtypes = [vp, dp, dp, i64, i64, vp, i32, i32, vp]
        L.sisso_l0_sis_generated.argtypes = [vp, dp, i64, i64, vp, vp, vp, i64, dp, i32,
                                             ctypes.c_double, ctypes.c_double, vp, vp, vp]
        L.sisso_l0_dimension_loop.argtypes = [vp, dp, dp, i64, i64, i32, i32, i32, i32, vp, vp,
                                              vp]
        no_int = ("sisso_l0_last_error", "sisso_l0_destroy", "sisso_l0_count_tuples",
                  "sisso_l0_scorer_destroy", "sisso_l0_scorer_last_error")
        for name in EXPORTS:
            if name not in no_int:
                getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


def measure_peaks(device=0) -> dict:
    """Measured unit rates of the device (see sisso_l0_measure_peaks)."""
    out = np.zeros(5, dtype=np.float64)
    rc = lib().sisso_l0_measure_peaks(int(device), ctypes.c_void_p(out.ctypes.data))
    if rc != OK:
        raise L0Error(rc, "sisso_l0_measure_peaks failed")
    return {"fp32_tflops": out[0], "fp64_tflops": out[1], "rsqrt_gops": out[2],
            "smem_gbs": out[3], "l2_gbs": out[4]}


def count_tuples(m: int, n: int) -> int:
    return int(lib().sisso_l0_count_tuples(int(m), int(n)))


def _ptr(a):
    """Raw address of a torch tensor or numpy array (kept alive by the caller)."""
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _as_f64(a):
    if hasattr(a, "data_ptr"):
        import torch
        return a.to(torch.float64).contiguous()
    return np.ascontiguousarray(a, dtype=np.float64)


class Handle:
    """Owns one library handle (device workspace, stream binding)."""

    def __init__(self, precision=FP64, task_mode=PER_TASK, device=0, stream=None,
                 candidate_pool=0, max_candidate_pool=2048, timeout_seconds=300.0,
                 fp32_fallback_pivot_ratio=1e-6, rank_deficient_pivot_ratio=1e-12,
                 autotune=0, use_graph=0, autotune_cache_path=None, fp64_rerun_uncertified=1,
                 tuple_kernel=-1):
        L = lib()
        o = Options()
        L.sisso_l0_default_options(ctypes.byref(o))
        o.device = int(device)
        o.stream = ctypes.c_void_p(int(stream) if stream else 0)
        o.precision = int(precision)
        o.task_mode = int(task_mode)
        o.candidate_pool = int(candidate_pool)
        o.max_candidate_pool = int(max_candidate_pool)
        o.timeout_seconds = float(timeout_seconds)
        o.fp32_fallback_pivot_ratio = float(fp32_fallback_pivot_ratio)
        o.rank_deficient_pivot_ratio = float(rank_deficient_pivot_ratio)
        o.autotune = int(autotune)
        o.use_graph = int(use_graph)
        o.fp64_rerun_uncertified = int(fp64_rerun_uncertified)
        o.tuple_kernel = int(tuple_kernel)
        self._cache_path = (autotune_cache_path.encode() if isinstance(autotune_cache_path, str)
                            else autotune_cache_path)
        o.autotune_cache_path = self._cache_path
        self._opt = o
        h = ctypes.c_void_p()
        rc = L.sisso_l0_create(ctypes.byref(h), ctypes.byref(o))
        if rc != OK:
            raise L0Error(rc, "sisso_l0_create failed")
        self._h = h
        self.task_mode = int(task_mode)

    def close(self):
        if getattr(self, "_h", None):
            lib().sisso_l0_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != OK:
            msg = lib().sisso_l0_last_error(self._h)
            raise L0Error(rc, msg.decode() if msg else "")

    def fit(self, X, y, n_dim, k, offsets=None, out_tuples=None, out_rmse=None):
        """Run sisso_l0_fit.  Returns (tuples [n_out, k, n_dim] int32,
        rmse [n_out, k] float64) as numpy arrays, or fills the given output
        buffers (torch or numpy) and returns them."""
        X = _as_f64(X)
        y = _as_f64(y)
        n_sis, n_total = int(X.shape[0]), int(X.shape[1])
        if offsets is None:
            offsets = [0, n_total]
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        n_tasks = len(off) - 1
        n_out = 1 if self.task_mode == SHARED else n_tasks
        ret_np = out_tuples is None
        if out_tuples is None:
            out_tuples = np.empty((n_out, k, n_dim), dtype=np.int32)
            out_rmse = np.empty((n_out, k), dtype=np.float64)
        rc = lib().sisso_l0_fit(self._h, ctypes.c_void_p(_ptr(X)), ctypes.c_void_p(_ptr(y)),
                                off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), n_tasks,
                                n_sis, int(n_dim), int(k), ctypes.c_void_p(_ptr(out_tuples)),
                                ctypes.c_void_p(_ptr(out_rmse)))
        self._check(rc)
        return (out_tuples, out_rmse) if ret_np else (out_tuples, out_rmse)

    def fit_multi(self, X, y, requests, offsets=None, outs=None):
        """Several searches in one pass.  requests: list of (n_dim, k).
        Returns a list of (tuples [n_out, k, n_dim], rmse [n_out, k]) (numpy,
        or the given output buffers `outs`, torch or numpy, one pair per
        request)."""
        X = _as_f64(X)
        y = _as_f64(y)
        n_sis, n_total = int(X.shape[0]), int(X.shape[1])
        if offsets is None:
            offsets = [0, n_total]
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        n_tasks = len(off) - 1
        n_out = 1 if self.task_mode == SHARED else n_tasks
        if outs is None:
            outs = [(np.empty((n_out, k, d), dtype=np.int32), np.empty((n_out, k), dtype=np.float64))
                    for d, k in requests]
        reqs = (Request * len(requests))()
        for i, ((d, k), (t, r)) in enumerate(zip(requests, outs)):
            reqs[i].n_dim, reqs[i].k = int(d), int(k)
            reqs[i].out_tuples = _ptr(t)
            reqs[i].out_rmse = _ptr(r)
        rc = lib().sisso_l0_fit_multi(self._h, ctypes.c_void_p(_ptr(X)), ctypes.c_void_p(_ptr(y)),
                                      off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), n_tasks,
                                      n_sis, reqs, len(requests))
        self._check(rc)
        return outs

    def set_timeout(self, seconds):
        """Host-side deadline of later calls (<= 0: none)."""
        self._check(lib().sisso_l0_set_timeout(self._h, float(seconds)))

    def stats(self) -> dict:
        s = Stats()
        s.struct_size = ctypes.sizeof(Stats)
        self._check(lib().sisso_l0_get_stats(self._h, ctypes.byref(s)))
        return s.as_dict()

    # ----------------------------------------------- learned proposals --
    def pair_data(self, X, y, labels=True, standardize=False):
        """Features [C(m,2), 8] and (optionally) labels [C(m,2)] of every pair
        of one task, as CUDA tensors (mixed-precision handle); standardize
        z-scores the labels over the task."""
        import torch
        X = _as_f64(X)
        y = _as_f64(y)
        m, n = int(X.shape[0]), int(X.shape[1])
        npairs = m * (m - 1) // 2
        dev = torch.device("cuda", self._opt.device)
        feats = torch.empty((npairs, PAIR_FEATURES_LD), dtype=torch.float32, device=dev)
        lab = torch.empty(npairs, dtype=torch.float32, device=dev) if labels else None
        rc = lib().sisso_l0_pair_data(self._h, ctypes.c_void_p(_ptr(X)), ctypes.c_void_p(_ptr(y)),
                                      n, m, ctypes.c_void_p(feats.data_ptr()),
                                      ctypes.c_void_p(lab.data_ptr() if lab is not None else 0),
                                      int(bool(standardize)))
        self._check(rc)
        return feats, lab

    def fit_pairs(self, X, y, pairs, k):
        """Exact d = 3 search over the triples reachable from pairs [P, 2]
        (one task).  Returns (tuples [k, 3], rmse [k])."""
        X = _as_f64(X)
        y = _as_f64(y)
        m, n = int(X.shape[0]), int(X.shape[1])
        if hasattr(pairs, "data_ptr"):
            import torch
            pairs = pairs.to(torch.int32).contiguous()
        else:
            pairs = np.ascontiguousarray(pairs, dtype=np.int32)
        out_t = np.empty((k, 3), dtype=np.int32)
        out_r = np.empty(k, dtype=np.float64)
        rc = lib().sisso_l0_fit_pairs(self._h, ctypes.c_void_p(_ptr(X)), ctypes.c_void_p(_ptr(y)),
                                      n, m, ctypes.c_void_p(_ptr(pairs)), int(pairs.shape[0]),
                                      int(k), ctypes.c_void_p(out_t.ctypes.data),
                                      ctypes.c_void_p(out_r.ctypes.data))
        self._check(rc)
        return out_t, out_r

    def fit_learned(self, X, y, scorer, k, fraction=0.01, out_tuples=None, out_rmse=None):
        """Learned d = 3 search (one task): returns (tuples [k, 3], rmse [k])."""
        X = _as_f64(X)
        y = _as_f64(y)
        m, n = int(X.shape[0]), int(X.shape[1])
        if out_tuples is None:
            out_tuples = np.empty((k, 3), dtype=np.int32)
            out_rmse = np.empty(k, dtype=np.float64)
        rc = lib().sisso_l0_fit_learned(self._h, scorer._s, ctypes.c_void_p(_ptr(X)),
                                        ctypes.c_void_p(_ptr(y)), n, m, int(k), float(fraction),
                                        ctypes.c_void_p(_ptr(out_tuples)),
                                        ctypes.c_void_p(_ptr(out_rmse)))
        self._check(rc)
        return out_tuples, out_rmse

    # -------------------------------------------------------- sharding --
    def fit_shard(self, X, y, n_dim, k, shard, n_shards):
        """One shard of a single-task search.  Returns (keys uint64 [c],
        sse float64 [c], bound, delta)."""
        X = _as_f64(X)
        y = _as_f64(y)
        m, n = int(X.shape[0]), int(X.shape[1])
        keys = np.empty(MAX_POOL, dtype=np.uint64)
        sse = np.empty(MAX_POOL, dtype=np.float64)
        cnt = np.zeros(1, dtype=np.int32)
        bd = np.zeros(2, dtype=np.float64)
        rc = lib().sisso_l0_fit_shard(self._h, ctypes.c_void_p(_ptr(X)), ctypes.c_void_p(_ptr(y)),
                                      n, m, int(n_dim), int(k), int(shard), int(n_shards),
                                      ctypes.c_void_p(keys.ctypes.data),
                                      ctypes.c_void_p(sse.ctypes.data),
                                      ctypes.c_void_p(cnt.ctypes.data),
                                      ctypes.c_void_p(bd.ctypes.data),
                                      ctypes.c_void_p(bd.ctypes.data + 8))
        self._check(rc)
        c = int(cnt[0])
        return keys[:c].copy(), sse[:c].copy(), float(bd[0]), float(bd[1])

    def merge_shards(self, n_sis, n_dim, k, n_total, keys, sse, bounds, deltas):
        """Rank the union of shard candidates.  Returns (tuples [k, n_dim],
        rmse [k], certified)."""
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        sse = np.ascontiguousarray(sse, dtype=np.float64)
        bounds = np.ascontiguousarray(bounds, dtype=np.float64)
        deltas = np.ascontiguousarray(deltas, dtype=np.float64)
        out_t = np.empty((k, n_dim), dtype=np.int32)
        out_r = np.empty(k, dtype=np.float64)
        cert = np.zeros(1, dtype=np.int32)
        rc = lib().sisso_l0_merge_shards(self._h, int(n_sis), int(n_dim), int(k), int(n_total),
                                         ctypes.c_void_p(keys.ctypes.data),
                                         ctypes.c_void_p(sse.ctypes.data), len(keys),
                                         ctypes.c_void_p(bounds.ctypes.data),
                                         ctypes.c_void_p(deltas.ctypes.data), len(bounds),
                                         ctypes.c_void_p(out_t.ctypes.data),
                                         ctypes.c_void_p(out_r.ctypes.data),
                                         ctypes.c_void_p(cert.ctypes.data))
        self._check(rc)
        return out_t, out_r, bool(cert[0])

    def sis(self, X, y, m):
        """SIS screening: (indices [m], r [m]) of the m features of largest
        |r| with y (X feature-major [n_feat, n_total])."""
        X = _as_f64(X)
        y = _as_f64(y)
        nf, n = int(X.shape[0]), int(X.shape[1])
        idx = np.empty(m, dtype=np.int32)
        r = np.empty(m, dtype=np.float64)
        self._check(lib().sisso_l0_sis(self._h, ctypes.c_void_p(_ptr(X)), ctypes.c_void_p(_ptr(y)),
                                       n, nf, int(m), ctypes.c_void_p(idx.ctypes.data),
                                       ctypes.c_void_p(r.ctypes.data)))
        return idx, r

    def sis_multi(self, X, Y, m, exclude=()):
        """SIS against several targets Y [R, n_total] (max |r| over them),
        never selecting the features in ``exclude``: (indices [m], r [m])."""
        X = _as_f64(X)
        Y = _as_f64(Y)
        if len(Y.shape) == 1:
            Y = Y.reshape(1, -1)
        nf, n = int(X.shape[0]), int(X.shape[1])
        ex = np.ascontiguousarray(np.asarray(exclude, dtype=np.int32).reshape(-1))
        idx = np.empty(m, dtype=np.int32)
        r = np.empty(m, dtype=np.float64)
        self._check(lib().sisso_l0_sis_multi(
            self._h, ctypes.c_void_p(_ptr(X)), ctypes.c_void_p(_ptr(Y)), int(Y.shape[0]), n, nf,
            int(m), ctypes.c_void_p(ex.ctypes.data if len(ex) else None), len(ex),
            ctypes.c_void_p(idx.ctypes.data), ctypes.c_void_p(r.ctypes.data)))
        return idx, r

    def sis_generated(self, C, ops, c1, c2, y, m, l_bound=1e-5, u_bound=1e8, want_valid=True):
        """SIS over the generated candidates ops[t](C[c1[t]], C[c2[t]]):
        (candidate indices [m] (-1 past the valid count), r [m], valid
        [n_cand] uint8 or None)."""
        C = _as_f64(C)
        y = _as_f64(y)
        ints = []
        for a in (ops, c1, c2):
            if hasattr(a, "data_ptr"):
                import torch
                ints.append(a.to(torch.int32).contiguous())
            else:
                ints.append(np.ascontiguousarray(a, dtype=np.int32))
        nc, n = int(C.shape[0]), int(C.shape[1])
        n_cand = int(ints[0].shape[0])
        idx = np.empty(m, dtype=np.int32)
        r = np.empty(m, dtype=np.float64)
        valid = np.empty(n_cand, dtype=np.uint8) if want_valid else None
        self._check(lib().sisso_l0_sis_generated(
            self._h, ctypes.c_void_p(_ptr(C)), nc, n, ctypes.c_void_p(_ptr(ints[0])),
            ctypes.c_void_p(_ptr(ints[1])), ctypes.c_void_p(_ptr(ints[2])), n_cand,
            ctypes.c_void_p(_ptr(y)), int(m), float(l_bound), float(u_bound),
            ctypes.c_void_p(idx.ctypes.data), ctypes.c_void_p(r.ctypes.data),
            ctypes.c_void_p(valid.ctypes.data if valid is not None else None)))
        return idx, r, valid

    def residuals(self, X, y, tuples):
        """Residuals [R, n_total] of the least-squares fits (with intercept)
        of the R models ``tuples`` [R, d] (feature indices into X)."""
        X = _as_f64(X)
        y = _as_f64(y)
        t = np.ascontiguousarray(np.atleast_2d(np.asarray(tuples, dtype=np.int32)))
        nf, n = int(X.shape[0]), int(X.shape[1])
        out = np.empty((t.shape[0], n), dtype=np.float64)
        self._check(lib().sisso_l0_residuals(
            self._h, ctypes.c_void_p(_ptr(X)), ctypes.c_void_p(_ptr(y)), n, nf,
            ctypes.c_void_p(t.ctypes.data), int(t.shape[1]), int(t.shape[0]),
            ctypes.c_void_p(out.ctypes.data)))
        return out

    def dimension_loop(self, X, y, m, n_dim_max, k, n_res):
        """SIS + l0 per dimension 1..n_dim_max.  Returns a list of dicts per
        dimension: S (global indices in selection order, cumulative), tuples
        [k, n] (ascending global indices; -1 unfilled), rmse [k]."""
        X = _as_f64(X)
        y = _as_f64(y)
        nf, n = int(X.shape[0]), int(X.shape[1])
        D = int(n_dim_max)
        S = np.empty(D * m, dtype=np.int32)
        T = np.empty((D, k, D), dtype=np.int32)
        R = np.empty((D, k), dtype=np.float64)
        self._check(lib().sisso_l0_dimension_loop(
            self._h, ctypes.c_void_p(_ptr(X)), ctypes.c_void_p(_ptr(y)), n, nf, int(m), D, int(k),
            int(n_res), ctypes.c_void_p(S.ctypes.data), ctypes.c_void_p(T.ctypes.data),
            ctypes.c_void_p(R.ctypes.data)))
        return [dict(S=S[:(d + 1) * m].copy(), tuples=T[d, :, :d + 1].copy(), rmse=R[d].copy())
                for d in range(D)]

    def debug_unrank(self, m, n, ranks):
        ranks = np.ascontiguousarray(ranks, dtype=np.uint64)
        out = np.empty((len(ranks), n), dtype=np.int32)
        self._check(lib().sisso_l0_debug_unrank(self._h, int(m), int(n),
                                                ctypes.c_void_p(ranks.ctypes.data), len(ranks),
                                                ctypes.c_void_p(out.ctypes.data)))
        return out

    def debug_gram(self, X, y, offsets=None, task=0):
        X = np.ascontiguousarray(X, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        if offsets is None:
            offsets = [0, X.shape[1]]
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        m = X.shape[0]
        out = np.zeros((m + 1, m + 1), dtype=np.float64)
        self._check(lib().sisso_l0_debug_gram(
            self._h, ctypes.c_void_p(X.ctypes.data), ctypes.c_void_p(y.ctypes.data),
            off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(off) - 1, m, int(task),
            ctypes.c_void_p(out.ctypes.data)))
        return out


def fit(X, y, n_dim, k, offsets=None, **opts):
    """One-shot fit with a temporary handle."""
    with Handle(**opts) as h:
        return h.fit(X, y, n_dim, k, offsets=offsets)


class Scorer:
    """The learned pair scorer (6-256-256-1, BF16 tensor-core kernels)."""

    def __init__(self, device=0, seed=0):
        L = lib()
        s = ctypes.c_void_p()
        rc = L.sisso_l0_scorer_create(ctypes.byref(s), int(device), int(seed) & (2**64 - 1))
        if rc != OK:
            raise L0Error(rc, "sisso_l0_scorer_create failed")
        self._s = s
        self.device = int(device)

    def close(self):
        if getattr(self, "_s", None):
            lib().sisso_l0_scorer_destroy(self._s)
            self._s = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != OK:
            msg = lib().sisso_l0_scorer_last_error(self._s)
            raise L0Error(rc, msg.decode() if msg else "")

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        self._check(lib().sisso_l0_scorer_set_params(self._s, ctypes.c_void_p(flat.ctypes.data),
                                                     flat.size))

    def get_params(self):
        out = np.empty(SCORER_PARAMS, dtype=np.float32)
        self._check(lib().sisso_l0_scorer_get_params(self._s, ctypes.c_void_p(out.ctypes.data),
                                                     out.size))
        return out

    def loss_grad(self, feats, labels):
        """(loss, gradient [SCORER_PARAMS]) over CUDA tensors feats [B, 8], labels [B]."""
        loss = np.zeros(1, dtype=np.float32)
        grad = np.empty(SCORER_PARAMS, dtype=np.float32)
        self._check(lib().sisso_l0_scorer_loss_grad(
            self._s, ctypes.c_void_p(feats.data_ptr()), ctypes.c_void_p(labels.data_ptr()),
            int(labels.shape[0]), ctypes.c_void_p(loss.ctypes.data),
            ctypes.c_void_p(grad.ctypes.data)))
        return float(loss[0]), grad

    def train(self, feats, labels, batch_rows, steps, lr):
        """Adam steps on CUDA tensors; returns the per-step losses."""
        losses = np.zeros(max(1, int(steps)), dtype=np.float32)
        self._check(lib().sisso_l0_scorer_train(
            self._s, ctypes.c_void_p(feats.data_ptr()), ctypes.c_void_p(labels.data_ptr()),
            int(labels.shape[0]), int(batch_rows), int(steps), float(lr),
            ctypes.c_void_p(losses.ctypes.data)))
        return losses[:int(steps)]

    def predict(self, feats):
        import torch
        out = torch.empty(int(feats.shape[0]), dtype=torch.float32, device=feats.device)
        self._check(lib().sisso_l0_scorer_predict(self._s, ctypes.c_void_p(feats.data_ptr()),
                                                  int(feats.shape[0]),
                                                  ctypes.c_void_p(out.data_ptr())))
        return out
