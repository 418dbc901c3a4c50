"""Benchmark: l0 tuple-fits per second on the d = 3 workload.

Workload (default): one task, n_samples = 1000, n_sis = 1000, d = 3,
k = 100 (C(1000, 3) = 166,167,000 intercept + 3-feature least-squares fits),
synthetic SISSO-shaped columns (see workloads/synth.py).  One step = one full
sisso_l0_fit: centring, Gram, tuple search, merge, FP64 re-fit of the
candidate pool, final ranking.

The headline path is the mixed-precision one (split-BF16 tensor-core Gram,
FP32 tuple search, FP64 re-fit), with CUDA-graph replay and launch tuning;
the plain FP64 GPU path is timed in the same run (``fp64_path``) and must
return the same tuples.  Prints one JSON line (rank 0).  ``--impl reference``
times the CPU FP64 oracle instead (bounded samples of the same workload).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "l0 tuple-fits/sec at d=3 (top-100 agreement with the FP64 oracle)"
UNIT = "tuple-fits/s"
FP64_PEAK_TFLOPS = 1.25          # GB300 FP64 (nominal, FMA pipe)
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def fp32_peak_tflops(sm_mhz):
    return SM_COUNT * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


# DRAM bytes (read + write) of one tuple-kernel launch on the d=3 workload,
# from the ncu captures summarised in profiles/tile_kernel_l0_d3_n1000_m1000.md
# (shape 0, the general kernel) and profiles/tile32_kernel_l0_d3_n1000_m1000.md
# (shapes 1-3).  They describe the kernel built from sources with this hash;
# once the sources change the figure no longer applies and the bench reports
# null.  Keys: (workload, precision, kernel shape).
TRAFFIC_SOURCES = {0: ("l0_common.cuh", "l0_tile.cuh", "l0_tuple.cu", "l0_kernels.cuh")}
for _v in (1, 2, 3):
    TRAFFIC_SOURCES[_v] = ("l0_common.cuh", "l0_tile.cuh", "l0_tile32.cu", "l0_kernels.cuh",
                           "l0_tc.cuh")
TRAFFIC_CAPTURED = {("C2", "mixed", 3): (3051264 + 31744, "61a98c245ab10f0d")}
TUPLE_KERNEL_NAMES = {
    0: "tile_kernel (tuple search, any d)",
    1: "tile32_kernel (d <= 3 FP32 tuple search, 256 threads, one CTA per SM)",
    2: "tile32_kernel (d <= 3 FP32 tuple search, 256 threads, two CTAs per SM)",
    3: "tile32_kernel (d <= 3 FP32 tuple search, 512 threads, one CTA per SM)",
}


def tile_traffic(workload, precision, shape=0):
    import hashlib
    rec = TRAFFIC_CAPTURED.get((workload, precision, int(shape)))
    if rec is None:
        return None
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES[int(shape)]:
        with open(os.path.join(ROOT, "paper_2502_20072_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return rec[0] if h.hexdigest()[:16] == rec[1] else None


# DRAM bytes of one pre-screen launch per feature of n_samples=1000, from the
# ncu capture in profiles/sis_prescreen_n1000.md (500000 features: 4000389632
# read + 10852352 written), scaled by the features of a launch (the kernel
# reads each row once).  Tied to the sources it was taken from, as above.
SIS_TRAFFIC_SOURCES = ("l0_sis.cu", "l0_tc.cuh", "l0_screen.cuh")
SIS_TRAFFIC_CAPTURED = {1000: ((4000389632 + 10852352) / 500000, "46094b2b70d46d7e")}


def sis_traffic(fp64, n_feat, n):
    import hashlib
    rec = SIS_TRAFFIC_CAPTURED.get(n)
    if fp64 or rec is None or rec[1] is None:
        return None
    h = hashlib.sha256()
    for f in SIS_TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_2502_20072_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return rec[0] * n_feat if h.hexdigest()[:16] == rec[1] else None


def same_up_to_ties(t_ref, r_ref, t_got, r_got, rel_gap=1e-9):
    """The same tuples at every rank, where positions whose reference RMSEs lie
    within rel_gap of each other form a tie group whose tuple sets must match
    (the order inside a group is rounding).  Per task; both as tensors."""
    t_ref, r_ref = t_ref.cpu().numpy(), r_ref.cpu().numpy()
    t_got, r_got = t_got.cpu().numpy(), r_got.cpu().numpy()
    for task in range(t_ref.shape[0]):
        rr = r_ref[task]
        i = 0
        while i < len(rr):
            j = i + 1
            while j < len(rr) and (rr[j] == rr[j - 1] or
                                   abs(rr[j] - rr[j - 1]) <= rel_gap * max(abs(rr[j]), 1e-300)):
                j += 1
            a = sorted(map(tuple, t_ref[task][i:j].tolist()))
            b = sorted(map(tuple, t_got[task][i:j].tolist()))
            # a tie group that reaches rank k may continue past it: not compared
            if a != b and not (j == len(rr) and j - i > 1):
                return False
            i = j
    return True


def flops_per_tuple(d):
    # hoisted per-tuple work of the tuple kernel's fast path:
    # (d-2) FMA for h, MUL g2, FMA pp, FMA w, MUL w^2, FMA t  ->  d+1 FMA + 2 MUL
    return 2 * (d + 1) + 2


def flops_per_tuple_hoisted(d):
    # the per-tuple count of the (d-1)-prefix hoisted augmented-Cholesky form:
    # forward solve g = L_P^-1 C_Pk ((d-1)(d-2)/2 FMA + (d-1) MUL), pivot
    # p = C_kk - g.g (d-1 FMA), w = c_k - g.z_P (d-1 FMA), SSE/S_yy = p_P - w^2/p
    # (1 reciprocal + 2 multiplications); FMA = 2 flop -> 8, 15, 24 at d = 2, 3, 4
    return (d - 1) * (d - 2) + 5 * (d - 1) + 3


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, gpu_index):
        self.p = None
        # raw samples (the JSON line carries their summary); CLOCKS_CSV moves them
        self.path = os.environ.get("CLOCKS_CSV") or os.path.join(tempfile.gettempdir(),
                                                                 "clocks_bench.csv")
        self.idx = gpu_index

    def start(self):
        try:
            f = open(self.path, "w")
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(prob, d, budget_s=12.0):
    """The CPU FP64 oracle on a bounded sample: all d-tuples of the first m'
    columns (same samples), m' grown until the run takes a few seconds."""
    import oracle
    m_prime = 40
    while True:
        X = prob.X[:m_prime]
        t0 = time.perf_counter()
        oracle.fit(X, prob.y, d, 100)
        dt = time.perf_counter() - t0
        n = math.comb(m_prime, d)
        if dt > budget_s / 4 or m_prime >= prob.n_sis:
            break
        grow = (budget_s / 2 / max(dt, 1e-3)) ** (1.0 / d)
        m_prime = min(prob.n_sis, max(m_prime + 10, int(m_prime * min(grow, 3.0))))
    return {"value": n / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": "all C(%d,%d)=%d tuples of the first %d columns, n_samples=%d, %.1f s"
                      % (m_prime, d, n, m_prime, prob.n_total, dt)}


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return
    from workloads import make_config
    import oracle
    prob, d, k = make_config(args.workload)
    oracle.build()
    # one step = the oracle on the first m' columns, sized to ~5 s of CPU work
    base = cpu_baseline(prob, d, budget_s=8.0)
    m_prime = int(base["sample"].split("first ")[1].split(" ")[0])
    n = math.comb(m_prime, d)
    for _ in range(args.warmup):
        oracle.fit(prob.X[:m_prime], prob.y, d, k)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.fit(prob.X[:m_prime], prob.y, d, k)
        times.append(time.perf_counter() - t0)
    ms = 1000 * statistics.mean(times)
    value = n / (ms / 1000)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": _workload_desc(args.workload, prob, d, k)},
            "cpu_baseline": {"kind": "oracle", "cores": os.cpu_count(), "value": value,
                             "unit": UNIT, "sample": "all C(%d,%d) tuples of the first %d columns"
                                                     % (m_prime, d, m_prime)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _workload_desc(name, prob, d, k):
    ds = "+".join(str(x) for x in d) if isinstance(d, (tuple, list)) else str(d)
    return "%s: n_tasks=%d n_samples=%d n_sis=%d d=%s k=%d" % (
        name, prob.n_tasks, prob.n_total, prob.n_sis, ds, k)


def run_ours(args):
    import numpy as np
    import torch
    import paper_2502_20072_gb300 as l0
    from workloads import make_config

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    prob, d, k = make_config(args.workload)
    precision = {"fp64": l0.FP64, "mixed": l0.MIXED_BF16X3}[args.precision]
    dims = list(d) if isinstance(d, (tuple, list)) else [d]
    reqs = [(dd, k) for dd in dims]
    n_fits = sum(math.comb(prob.n_sis, dd) for dd in dims) * prob.n_tasks
    fl_all = sum(flops_per_tuple(dd) * math.comb(prob.n_sis, dd) for dd in dims) * prob.n_tasks
    fl_hoisted = sum(flops_per_tuple_hoisted(dd) * math.comb(prob.n_sis, dd)
                     for dd in dims) * prob.n_tasks
    # N > 1: one search split over the ranks (every N-th work item per rank,
    # one all-gather of the re-fitted candidate pools, the merge on every
    # rank): strong scaling.  --replicas runs N independent copies instead.
    sharded = ws > 1 and not args.replicas and prob.n_tasks == 1 and len(dims) == 1
    if sharded:
        from paper_2502_20072_gb300 import shard
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    X = torch.from_numpy(prob.X).cuda()
    y = torch.from_numpy(prob.y).cuda()

    def outputs(dev):
        if dev:
            return [(torch.empty((prob.n_tasks, k, dd), dtype=torch.int32, device="cuda"),
                     torch.empty((prob.n_tasks, k), dtype=torch.float64, device="cuda"))
                    for dd in dims]
        return [(np.empty((prob.n_tasks, k, dd), dtype=np.int32),
                 np.empty((prob.n_tasks, k), dtype=np.float64)) for dd in dims]

    def run(handle, Xa, ya, outs):
        if sharded:
            t_, r_, _ = shard.fit_sharded(handle, Xa, ya, dims[0], k)
            outs[0][0].copy_(torch.as_tensor(t_)[None]) if torch.is_tensor(outs[0][0]) else \
                np.copyto(outs[0][0], np.asarray(t_)[None])
            return
        if len(dims) == 1:
            handle.fit(Xa, ya, dims[0], k, offsets=prob.offsets, out_tuples=outs[0][0],
                       out_rmse=outs[0][1])
        else:
            handle.fit_multi(Xa, ya, reqs, offsets=prob.offsets, outs=outs)

    outs_dev = outputs(True)
    out_t = outs_dev[-1][0]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    opts = dict(device=local, stream=stream.cuda_stream, use_graph=int(not args.no_graph),
                autotune=int(not args.no_autotune))
    h = l0.Handle(precision=precision, **opts)

    def step():
        run(h, X, y, outs_dev)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    tuple_ms, launches = [], 0
    for i in range(args.steps):
        flush.zero_()            # L2 flush (256 MB > 129 MB L2), outside the timed events
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
        st = h.stats()
        tuple_ms.append(st["ms_tuple_kernel"])
        launches += int(st["kernel_launches"])
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = [a.elapsed_time(b) for a, b in ev]
    ms_step = statistics.mean(ms)
    if ws > 1:
        t = torch.tensor([ms_step], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_step = float(t.item())
    value = (1 if sharded else ws) * n_fits / (ms_step / 1000.0)
    st = h.stats()
    # e2e: host buffers through the C ABI (copies inside the timed region)
    Xh = torch.from_numpy(prob.X).pin_memory()
    yh = torch.from_numpy(prob.y).pin_memory()
    outs_h = outputs(False)
    e2e = []
    for i in range(max(2, min(args.steps, 5))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run(h, Xh, yh, outs_h)
        e2e.append(time.perf_counter() - t0)
    e2e_val = n_fits / statistics.median(e2e)
    # the plain FP64 GPU path on the same workload, same timing method
    fp64_line = None
    if precision != l0.FP64 and not args.no_fp64_path and not sharded:
        h64 = l0.Handle(precision=l0.FP64, **opts)
        outs64 = outputs(True)
        for _ in range(3):
            run(h64, X, y, outs64)
        ms64 = []
        for _ in range(max(2, min(args.steps, 5))):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            run(h64, X, y, outs64)
            b.record(stream)
            torch.cuda.synchronize()
            ms64.append(a.elapsed_time(b))
        v64 = n_fits / (statistics.mean(ms64) / 1000.0)
        same = all(bool(torch.equal(a[0], b[0])) for a, b in zip(outs64, outs_dev))
        fp64_line = {"value": v64, "ms_per_step": statistics.mean(ms64),
                     "speedup_of_this_path": value / v64 / ws,
                     "same_top_k_tuples": same,
                     "same_top_k_up_to_ties": same or all(
                         same_up_to_ties(a[0], a[1], b[0], b[1]) for a, b in zip(outs64, outs_dev))}
        h64.close()
    # roofline of the dominant kernel (the tuple kernel), timed by CUDA events
    # around its launch on the library's stream; events inside a replayed
    # graph may not be timeable, so measure extra un-graphed fits then
    stage = {s: st["ms_" + s] for s in ("prep", "gram", "tuple", "merge", "refit")}
    if min(tuple_ms) <= 0.0 and not sharded:
        hk = l0.Handle(precision=precision, device=local, stream=stream.cuda_stream,
                       autotune=int(not args.no_autotune), use_graph=0)
        tuple_ms = []
        acc = {s: [] for s in stage}
        for i in range(max(3, args.warmup) + max(2, min(args.steps, 5))):
            flush.zero_()
            run(hk, X, y, outs_dev)
            if i >= max(3, args.warmup):
                sk = hk.stats()
                tuple_ms.append(sk["ms_tuple_kernel"])
                for s in acc:
                    acc[s].append(sk["ms_" + s])
        hk.close()
        stage = {s: statistics.mean(v) for s, v in acc.items()}
    t_tuple = statistics.mean(tuple_ms) / 1000.0
    per_rank = ws if sharded else 1          # a shard's kernel does 1/N of the tuples
    achieved = fl_hoisted / per_rank / t_tuple / 1e12
    achieved_kernel_count = fl_all / per_rank / t_tuple / 1e12
    pk = l0.measure_peaks(local)
    if precision == l0.FP64 or st["fp64_rerun"]:
        # an uncertified mixed fit is redone in FP64: its last tuple kernel is the FP64 one
        peak, peak_note = pk["fp64_tflops"], "measured FP64 FMA rate (sisso_l0_measure_peaks)"
    else:
        peak, peak_note = pk["fp32_tflops"], "measured FP32 FMA rate (sisso_l0_measure_peaks)"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "strong" if sharded else "weak", "vs_baseline": None,
        "dtype": "f64" if precision == l0.FP64 else "f32",
        "data": "synthetic",
        "config": {"workload": _workload_desc(args.workload, prob, d, k),
                   "precision": args.precision,
                   "parallelism": ("sharded over %d GPUs: every %d-th work item per rank, "
                                   "one all-gather of the re-fitted candidate pools" % (ws, ws)
                                   if sharded else ("replicas" if ws > 1 else "single")),
                   "l2": "flushed between steps (256 MB write, outside the timed events)",
                   "candidate_pool": st["candidate_pool"], "certified": st["certified"],
                   "fp64_redo_tuples": int(st["fp64_fallback_tuples"]),
                   "graph_replayed": int(st["graph_replayed"]),
                   "fp64_rerun": int(st["fp64_rerun"]),
                   "tuned": [int(st["tuned_items_factor"]), int(st["tuned_ctas_per_sm"])],
                   "tuple_kernel_shape": int(st["tuple_kernel"]),
                   "stage_ms": {s: round(v, 4) for s, v in stage.items()},
                   "stage_ms_source": ("un-graphed fits on the same inputs"
                                       if st["graph_replayed"] else "the timed fits")},
        "e2e": {"value": e2e_val, "unit": UNIT,
                "h2d_bytes_per_step": int(prob.X.nbytes + prob.y.nbytes),
                "d2h_bytes_per_step": int(sum(a.nbytes + b.nbytes for a, b in outs_h))},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "traffic": tile_traffic(args.workload, args.precision, st["tuple_kernel"]),
                     "kernel": TUPLE_KERNEL_NAMES.get(int(st["tuple_kernel"]), "tuple kernel"),
                     "peak_source": peak_note,
                     "flops_per_tuple": {str(dd): flops_per_tuple_hoisted(dd) for dd in dims},
                     "flops_per_tuple_source": "hoisted (d-1)-prefix augmented Cholesky count",
                     "achieved_kernel_count": achieved_kernel_count,
                     "frac_kernel_count": achieved_kernel_count / peak,
                     "kernel_flops_per_tuple": {str(dd): flops_per_tuple(dd) for dd in dims}},
        "clocks": clk,
        "measured_peaks": {kk: round(v, 1) for kk, v in pk.items()},
    }
    if fp64_line is not None:
        line["fp64_path"] = fp64_line
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(prob, dims[-1])
    h.close()
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_learned(args):
    """The learned d = 3 search on the 20000-column workload: train the pair
    scorer on the exhaustive labels of 50 seeded 2000-column instances, run the
    exhaustive search once as the reference, then time the learned search."""
    import numpy as np
    import torch
    import paper_2502_20072_gb300 as l0
    from paper_2502_20072_gb300 import learn
    from workloads import make_config, make_problem
    from workloads.synth import C5L_TRAIN, C5L_TRAIN_SEEDS

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    t0 = time.perf_counter()
    train = [make_problem(seed=sd, **C5L_TRAIN) for sd in C5L_TRAIN_SEEDS[:args.train_instances]]
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    F, Y = learn.pair_training_set(train, device=local, seed=0)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    n_rows = int(Y.shape[0])
    del train
    scorer, losses, t_train = learn.train_scorer(F, Y, steps=args.train_steps, batch_rows=8192,
                                                lr=2e-3, seed=0, device=local)
    del F, Y
    torch.cuda.empty_cache()
    prob, d, k = make_config("C5L", n_sis=args.learned_sis)
    m = prob.n_sis
    X = torch.from_numpy(prob.X).cuda()
    y = torch.from_numpy(prob.y).cuda()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    h = l0.Handle(precision=l0.MIXED_BF16X3, device=local, stream=stream.cuda_stream)
    # the reference: exhaustive FP32 search with FP64 re-fit
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    ex_t, ex_r = h.fit(X, y, 3, k)
    e1.record(stream)
    torch.cuda.synchronize()
    ex_ms = e0.elapsed_time(e1)
    ex_fits = int(h.stats()["tuple_fits"])
    out_t = torch.empty((k, 3), dtype=torch.int32, device="cuda")
    out_r = torch.empty(k, dtype=torch.float64, device="cuda")
    for _ in range(max(3, args.warmup)):
        h.fit_learned(X, y, scorer, k, fraction=args.fraction, out_tuples=out_t, out_rmse=out_r)
    clocks = Clocks(local)
    clocks.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(args.steps):
        h.fit_learned(X, y, scorer, k, fraction=args.fraction, out_tuples=out_t, out_rmse=out_r)
    ev[1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev[0].elapsed_time(ev[1]) / args.steps
    st = h.stats()
    ms_scan = st["ms_tuple_kernel"]          # the scan kernel of the last step
    got = set(map(tuple, out_t.cpu().numpy().tolist()))
    ref = set(map(tuple, ex_t[0].tolist()))
    recall = len(got & ref) / len(ref)
    total = math.comb(m, 3)
    line = {
        "metric": "l0 tuple-fits/sec at d=3, learned proposals (search-space tuples per second;"
                  " recall@100 against the exhaustive search)",
        "value": total / (ms / 1000.0), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": _workload_desc("C5L", prob, d, k), "precision": "mixed",
                   "fraction": args.fraction, "inputs": "larger than L2 (X is 320 MB)"},
        "learned": {"recall_at_100": recall, "proposal_pairs": int(st["proposal_pairs"]),
                    "exact_fits_per_step": int(st["tuple_fits"]),
                    "exhaustive_ms": ex_ms, "exhaustive_fits": ex_fits,
                    "exhaustive_tuple_fits_per_s": ex_fits / (ex_ms / 1000.0),
                    "speedup_vs_exhaustive": ex_ms / ms,
                    "train_instances": args.train_instances, "train_rows": n_rows,
                    "train_steps": args.train_steps, "train_s": t_train,
                    "train_loss_first_last": [float(np.mean(losses[:10])),
                                              float(np.mean(losses[-50:]))],
                    "data_s": t_data, "generate_s": t_gen},
        "gpu_launches": None, "roofline": None, "clocks": clk,
    }
    h.close()
    scorer.close()
    if rank == 0:
        print(json.dumps(line))


def run_sis(args):
    """SIS screening (the step before l0): Pearson r of n_feat seeded
    candidate features with y and the top m, device-resident inputs."""
    import torch
    import paper_2502_20072_gb300 as l0
    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    n_feat, n, m = args.sis_features, 1000, 20000
    g = torch.Generator(device="cuda").manual_seed(7)
    X = torch.randn((n_feat, n), generator=g, device="cuda", dtype=torch.float64)
    w = torch.randn((8,), generator=g, device="cuda", dtype=torch.float64)
    y = (X[:8].T @ w) + 0.1 * torch.randn((n,), generator=g, device="cuda", dtype=torch.float64)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    prec = {"fp64": l0.FP64, "mixed": l0.MIXED_BF16X3}[args.precision]
    h = l0.Handle(precision=prec, device=local, stream=stream.cuda_stream)
    idx = torch.empty(m, dtype=torch.int32, device="cuda")
    r = torch.empty(m, dtype=torch.float64, device="cuda")
    lib = l0.lib()
    import ctypes

    def step():
        rc = lib.sisso_l0_sis(h._h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                              n, n_feat, m, ctypes.c_void_p(idx.data_ptr()),
                              ctypes.c_void_p(r.data_ptr()))
        h._check(rc)

    for _ in range(max(3, args.warmup)):
        step()
    clocks = Clocks(local)
    clocks.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(args.steps):
        step()
    ev[1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev[0].elapsed_time(ev[1]) / args.steps
    st = h.stats()
    ms_scan = st["ms_tuple_kernel"]          # the scan kernel of the last step
    pk_hbm = None
    mp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(mp):
        pk_hbm = json.load(open(mp)).get("hbm_gbs")
    gbs = n_feat * n * 8 / (ms * 1e-3) / 1e9
    gbs_scan = n_feat * n * 8 / (ms_scan * 1e-3) / 1e9 if ms_scan > 0 else None
    # end to end through the C entry with host buffers (pinned), copies timed:
    # a 1/8 slice of the features so the host copy stays a few GB
    ne = max(m, n_feat // 8)
    Xh = X[:ne].cpu().pin_memory()
    yh = y.cpu().pin_memory()
    idx_h = torch.empty(m, dtype=torch.int32).pin_memory()
    r_h = torch.empty(m, dtype=torch.float64).pin_memory()

    def step_host():
        rc = lib.sisso_l0_sis(h._h, ctypes.c_void_p(Xh.data_ptr()), ctypes.c_void_p(yh.data_ptr()),
                              n, ne, m, ctypes.c_void_p(idx_h.data_ptr()),
                              ctypes.c_void_p(r_h.data_ptr()))
        h._check(rc)

    step_host()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(3):
        step_host()
    torch.cuda.synchronize()
    ms_e2e = (time.perf_counter() - t0) * 1e3 / 3
    del Xh
    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        sys.path.insert(0, ROOT)
        from oracle import sis as osis
        ns = 4000
        Xs = X[:ns].cpu().numpy()
        ys = y.cpu().numpy()
        t0 = time.perf_counter()
        osis.sis(Xs, ys, 100)
        dt = time.perf_counter() - t0
        cpu = {"value": ns / dt, "unit": "features/s", "cores": 1, "kind": "oracle",
               "sample": "%d of the %d features (n_samples=%d), top 100" % (ns, n_feat, n)}
    line = {"metric": "SIS screening features/sec (Pearson r + top-m)",
            "value": n_feat / (ms * 1e-3), "unit": "features/s", "n_gpus": ws,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == l0.FP64 else "f32 pre-screen + f64",
            "data": "synthetic (seeded normal features on the device)",
            "config": {"workload": "SIS: n_feat=%d n_samples=%d m=%d" % (n_feat, n, m),
                       "inputs": "larger than L2 (%.1f GB)" % (n_feat * n * 8 / 1e9),
                       "fp64_rescored": int(st["fp64_fallback_tuples"])},
            "e2e": {"value": ne / (ms_e2e * 1e-3), "unit": "features/s",
                    "h2d_bytes_per_step": ne * n * 8 + n * 8, "d2h_bytes_per_step": m * 12,
                    "sample": "%d features from pinned host memory" % ne},
            "gpu_launches": int(st["kernel_launches"]) * args.steps,
            "roofline": {"bound": "hbm", "achieved": gbs_scan, "peak": pk_hbm, "unit": "GB/s",
                         "frac": gbs_scan / pk_hbm if (pk_hbm and gbs_scan) else None,
                         "traffic": sis_traffic(prec == l0.FP64, n_feat, n),
                         "kernel": "sis_score_kernel" if prec == l0.FP64 else
                                   "sis_prescreen_bulk_kernel",
                         "kernel_ms": ms_scan, "whole_pass_gbs": gbs,
                         "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy)"},
            "cpu_baseline": cpu,
            "clocks": clk}
    h.close()
    if rank == 0:
        print(json.dumps(line))


def run_loop(args):
    """The dimension loop (SIS -> l0 -> residuals -> multi-residual SIS ...):
    n_feat seeded candidate features resident on the device, one planted
    three-term descriptor among decoys."""
    import torch
    import paper_2502_20072_gb300 as l0
    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    n_feat, n, m, D, k, n_res = args.loop_features, 1000, args.loop_m, 3, 10, 10
    g = torch.Generator(device="cuda").manual_seed(11)
    X = torch.randn((n_feat, n), generator=g, device="cuda", dtype=torch.float64)
    a, b, c = 11, n_feat // 2, (7 * n_feat) // 9
    X[:64] = X[a] + 0.4 * torch.randn((64, n), generator=g, device="cuda", dtype=torch.float64)
    y = 2.0 * X[a] + 0.6 * X[b] - 0.4 * X[c] + 0.02 * torch.randn((n,), generator=g, device="cuda",
                                                                  dtype=torch.float64)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    prec = {"fp64": l0.FP64, "mixed": l0.MIXED_BF16X3}[args.precision]
    h = l0.Handle(precision=prec, device=local, stream=stream.cuda_stream)
    out = None

    def step():
        nonlocal out
        out = h.dimension_loop(X, y, m, D, k, n_res)

    for _ in range(max(3, args.warmup)):
        step()
    clocks = Clocks(local)
    clocks.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(args.steps):
        step()
    ev[1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev[0].elapsed_time(ev[1]) / args.steps
    found = tuple(int(t) for t in out[2]["tuples"][0]) == tuple(sorted((a, b, c)))
    # screening passes over X: one per dimension (all residuals in one pass)
    passes = D
    xbytes = passes * n_feat * n * 8
    tuples = sum(math.comb(m * d, d) for d in range(1, D + 1))
    pk_hbm = None
    mp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(mp):
        pk_hbm = json.load(open(mp)).get("hbm_gbs")
    gbs = xbytes / (ms * 1e-3) / 1e9
    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        sys.path.insert(0, ROOT)
        from oracle import loop as oloop
        ns, ms_s = 20000, 20
        Xs = X[:ns].cpu().numpy()
        ys = y.cpu().numpy()
        t0 = time.perf_counter()
        oloop.dimension_loop(Xs, ys, ms_s, 2, k, n_res)
        dt = time.perf_counter() - t0
        cpu = {"value": dt * 1e3, "unit": "ms per loop", "cores": 16, "kind": "oracle",
               "sample": "%d of the features, m=%d, dimensions 1-2 (not comparable in size: "
                         "context only)" % (ns, ms_s)}
    line = {"metric": "dimension loop (SIS + l0 per dimension, 3 dimensions) ms per loop",
            "value": ms, "unit": "ms", "n_gpus": ws, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == l0.FP64 else "f32 pre-screen + f64; FP32 l0 search + FP64 re-fit",
            "data": "synthetic (seeded normal features on the device, planted 3-term descriptor)",
            "config": {"workload": "LOOP: n_feat=%d n_samples=%d m=%d per dimension D=%d k=%d "
                                   "residuals=%d" % (n_feat, n, m, D, k, n_res),
                       "inputs": "larger than L2 (%.1f GB)" % (n_feat * n * 8 / 1e9),
                       "planted_found": found, "l0_tuples": tuples,
                       "screening_passes": passes},
            "gpu_launches": int(h.stats()["kernel_launches"]) * args.steps,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": pk_hbm, "unit": "GB/s",
                         "frac": gbs / pk_hbm if pk_hbm else None, "traffic": None,
                         "kernel": "whole loop: X bytes of the screening passes / loop time"},
            "cpu_baseline": cpu, "clocks": clk}
    h.close()
    if rank == 0:
        print(json.dumps(line))


def run_generated(args):
    """SIS over generated features (operators on child pairs, value rules,
    Pearson in one pass, nothing stored): every pair of n_child children for
    the five binary operators (both orders for - and /) and the nine unary
    operators on every child."""
    import torch
    import paper_2502_20072_gb300 as l0
    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    nc, n, m = args.gen_children, 200, 5000
    g = torch.Generator(device="cuda").manual_seed(13)
    C = (0.3 + 2.7 * torch.rand((nc, n), generator=g, device="cuda", dtype=torch.float64))
    y = torch.log(C[4]) * C[7] + 0.05 * torch.randn((n,), generator=g, device="cuda",
                                                    dtype=torch.float64)
    i, j = torch.triu_indices(nc, nc, 1, device="cuda")
    parts = []
    for op, both in ((0, False), (1, True), (2, False), (3, True), (4, False)):
        parts.append((torch.full_like(i, op), i, j))
        if both:
            parts.append((torch.full_like(i, op), j, i))
    ar = torch.arange(nc, device="cuda")
    for op in range(5, 14):
        parts.append((torch.full_like(ar, op), ar, torch.zeros_like(ar)))
    ops = torch.cat([p[0] for p in parts]).to(torch.int32)
    c1 = torch.cat([p[1] for p in parts]).to(torch.int32)
    c2 = torch.cat([p[2] for p in parts]).to(torch.int32)
    n_cand = int(ops.shape[0])
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    mixed = args.precision != "fp64"
    lib = l0.lib()
    import ctypes

    def timed(handle, idx, r):
        def step():
            rc = lib.sisso_l0_sis_generated(
                handle._h, ctypes.c_void_p(C.data_ptr()), nc, n, ctypes.c_void_p(ops.data_ptr()),
                ctypes.c_void_p(c1.data_ptr()), ctypes.c_void_p(c2.data_ptr()), n_cand,
                ctypes.c_void_p(y.data_ptr()), m, 1e-5, 1e8, ctypes.c_void_p(idx.data_ptr()),
                ctypes.c_void_p(r.data_ptr()), None)
            handle._check(rc)

        for _ in range(max(3, args.warmup)):
            step()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        for _ in range(args.steps):
            step()
        ev[1].record(stream)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / args.steps

    # the headline path: FP32 pre-screen + FP64 re-score (mixed handle), or
    # the FP64 evaluation of every candidate (--precision fp64)
    h = l0.Handle(precision=l0.MIXED_BF16X3 if mixed else l0.FP64, device=local,
                  stream=stream.cuda_stream)
    idx = torch.empty(m, dtype=torch.int32, device="cuda")
    r = torch.empty(m, dtype=torch.float64, device="cuda")
    clocks = Clocks(local)
    clocks.start()
    ms = timed(h, idx, r)
    clk = clocks.stop()
    st = h.stats()
    ms_k = st["ms_tuple_kernel"]
    fp64_line = None
    if mixed:
        h64 = l0.Handle(precision=l0.FP64, device=local, stream=stream.cuda_stream)
        idx64 = torch.empty(m, dtype=torch.int32, device="cuda")
        r64 = torch.empty(m, dtype=torch.float64, device="cuda")
        ms64 = timed(h64, idx64, r64)
        h64.close()
        same = bool(torch.equal(idx, idx64)) and bool(torch.allclose(r, r64, rtol=1e-12, atol=0))
        fp64_line = {"ms_per_step": ms64, "value": n_cand / (ms64 * 1e-3),
                     "speedup_of_this_path": ms64 / ms, "same_selection": same}
    flop = n_cand * n * 7
    tf = flop / (ms_k * 1e-3) / 1e12 if ms_k > 0 else None
    peaks = {}
    try:
        peaks = l0.measure_peaks(local)
    except Exception:
        pass
    pk = peaks.get("fp32_tflops" if mixed else "fp64_tflops")
    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        sys.path.insert(0, ROOT)
        from oracle import generate as og
        ns = 20000
        Cs = C.cpu().numpy()
        ys = y.cpu().numpy()
        sel = torch.randperm(n_cand, generator=torch.Generator().manual_seed(0))[:ns].numpy()
        o_h, a_h, b_h = ops.cpu().numpy()[sel], c1.cpu().numpy()[sel], c2.cpu().numpy()[sel]
        t0 = time.perf_counter()
        og.sis_generated(Cs, o_h, a_h, b_h, ys, 100)
        dt = time.perf_counter() - t0
        cpu = {"value": ns / dt, "unit": "candidates/s", "cores": 1, "kind": "oracle",
               "sample": "%d random candidates of the %d" % (ns, n_cand)}
    line = {"metric": "generated-feature SIS candidates/sec (operator values + rules + Pearson "
                      "+ top-m)",
            "value": n_cand / (ms * 1e-3), "unit": "candidates/s", "n_gpus": ws,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 pre-screen + f64" if mixed else "f64",
            "data": "synthetic (seeded uniform children on the device)",
            "config": {"workload": "GEN: n_child=%d n_samples=%d candidates=%d m=%d"
                                   % (nc, n, n_cand, m),
                       "inputs": "children %.1f MB (L2-resident), candidate lists %.0f MB"
                                 % (nc * n * 8 / 1e6, n_cand * 12 / 1e6)},
            "gpu_launches": int(st["kernel_launches"]) * args.steps,
            "roofline": {"bound": "alu", "achieved": tf, "peak": pk, "unit": "TFLOP/s",
                         "frac": tf / pk if (tf and pk) else None, "traffic": None,
                         "kernel": "gen_prescreen_kernel (FP32)" if mixed else
                                   "gen_score_kernel (FP64)", "kernel_ms": ms_k,
                         "peak_source": "measured %s FMA rate (sisso_l0_measure_peaks)"
                                        % ("FP32" if mixed else "FP64"),
                         "flop_per_sample": 7},
            "cpu_baseline": cpu, "clocks": clk}
    if fp64_line:
        line["fp64_path"] = fp64_line
    h.close()
    if rank == 0:
        print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--replicas", action="store_true",
                    help="N > 1: N independent copies of the workload instead of one sharded search")
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-fp64-path", action="store_true")
    ap.add_argument("--workload", default="C2")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fraction", type=float, default=0.01)
    ap.add_argument("--train-steps", type=int, default=4000)
    ap.add_argument("--train-instances", type=int, default=50)
    ap.add_argument("--sis-features", type=int, default=4000000)
    ap.add_argument("--loop-features", type=int, default=1000000)
    ap.add_argument("--gen-children", type=int, default=3000)
    ap.add_argument("--loop-m", type=int, default=500)
    ap.add_argument("--learned-sis", type=int, default=20000,
                    help="columns of the learned workload (smaller for profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "C5L":
        run_learned(args)
    elif args.workload == "SIS":
        run_sis(args)
    elif args.workload == "LOOP":
        run_loop(args)
    elif args.workload == "GEN":
        run_generated(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
