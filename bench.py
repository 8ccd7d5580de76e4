"""Benchmark: incremental all-pairs SimRank update stream on one GB300.

Workload (the power-law update stream): directed Chung-Lu graph, n = 20,000,
in/out-degree exponent 2.1, mean degree 10 (m = 200,000), C = 0.6, K = 20,
S in FP32 (1.6 GB, larger than L2; upper tiles kept), xi/eta recurrence
vectors in FP64, affected-area pruning on.  One step applies a batch of 1,000
sequential unit updates (80% insertions with degree-biased endpoints, 20%
deletions of uniform existing edges); each update runs Alg 1 (one cooperative
launch for its recurrence) and its rank-2(K+1) S change is applied by the
tensor-core S pass (3-term FP16 split), 16 pending updates per pass by
default (--defer / --tc / --vec-fp64 select the other forms).  Steps
continue one valid stream, so every step changes the graph.

Prints one JSON line (see the keys below): the device-timed throughput, the
same through the public call with host buffers (e2e), the two kernels of the
path against their roofline, the per-edge S pass alone, the other vector
precision over the same steps, and the max-abs error against the FP64 oracle
(Alg 1 at the same K on sampled columns, and the drift from the converged
fixed point after one step).  ``--impl reference`` times the FP64 CPU oracle
(Alg 1 as printed, dense) on a bounded sample instead.  Under torchrun each
rank runs an independent replica of the workload (the update stream is
sequential and has no data-parallel split).  Other workloads (--workload
batched / multi / column / grad / accelerate) print their own line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import chung_lu_digraph, update_stream, EdgeSet  # noqa: E402

N, M, GAMMA, C, K = 20000, 200000, 2.1, 0.6, 20
UPDATES_PER_STEP = 1000
SEED_GRAPH, SEED_STREAM = 2, 3
METRIC = "edge updates/sec & HBM GB/s: fused rank-2K ΔS vs plain Inc-uSR at 1e-6 error"
UNIT = "edge updates/s"
# DRAM bytes (read + write) per launch from one ncu capture of each kernel on
# the default stream configuration (profiles/ holds the summaries)
TRAFFIC_PREP = 6.137e7
TRAFFIC_S_PASS = 1.828e9
# the per-update S pass (--defer 0 replica, FP16 split): a typical launch
TRAFFIC_S_PASS_EDGE = 1.417e9


def workload_name(args):
    vec = "FP64" if args.vec_fp64 else "FP32"
    return ("power-law update stream: directed Chung-Lu n=20000, exponent 2.1, mean degree 10, "
            f"C=0.6, K=20, FP32 S, {vec} xi/eta vectors, AFF pruning, 1000 sequential unit updates "
            "per step (80% insert / 20% delete), rank-2(K+1) S changes applied by the tensor-core "
            "S pass")


def read_bf16_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f)["bf16_tflops"])
    return 1900.0


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
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
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def make_streams(total_steps, per_step=UPDATES_PER_STEP):
    s, d = chung_lu_digraph(N, M, GAMMA, GAMMA, SEED_GRAPH)
    es = EdgeSet(N, s, d)
    streams = [update_stream(N, s, d, per_step, SEED_STREAM + t, edge_set=es)
               for t in range(total_steps)]
    return s, d, streams


def cpu_baseline_sample(s, d, stream, max_updates=1):
    """The oracle (Alg 1 as printed: dense FP64 Q, S and M_k) on the first
    update(s) of the stream at full n.  Its cost does not depend on the values
    of S, so S = (1 - C) I stands in for the converged old S."""
    from oracle import simrank_oracle as O

    S = (1.0 - C) * np.eye(N)
    t0 = time.perf_counter()
    done = 0
    src, dst = s, d
    for i, j, op in stream[:max_updates].tolist():
        S = O.inc_usr(N, src, dst, S, int(j), [int(i)], int(op), C, K)
        done += 1
    dt = time.perf_counter() - t0
    return done / dt, dt, done


def max_over_ranks(values, dist=None, device="cpu"):
    """Element-wise maximum of per-rank timings over all ranks (an all-reduce
    with MAX; the values unchanged without a process group).  With N
    independent replicas the whole-job rate is the units of all ranks divided
    by the slowest rank's time."""
    import torch

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def run_reference(args, rank):
    if rank != 0:
        return
    s, d, streams = make_streams(1)
    stream = streams[0]
    per = []
    for t in range(args.warmup + args.steps):
        v, dt, n_up = cpu_baseline_sample(s, d, stream[t % len(stream):], 1)
        if t >= args.warmup:
            per.append(dt / n_up)
    value = 1.0 / statistics.mean(per)
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * statistics.mean(per), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args), "n": N, "m": M, "C": C, "K": K,
                   "l2": "S larger than L2 (1.6 GB FP32)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "one unit update per step at full n (Alg 1, dense FP64), "
                                   "S = (1-C) I stand-in (cost is value-independent)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def stream_prep_bytes(n_pad, m, k, pair_bytes, npend_avg, delta=1):
    """Algorithmic bytes of one pre-update launch (k_prep): each of the K
    steps reads the column indices (4 B per nonzero) and reads and writes one
    (xi, eta) pair column (pair_bytes per row each way; the gathered values
    are re-reads of that column and are not counted again); the panels are
    written once (2 (K+1) n FP32 values); the rows of S read (delta + 1 rows
    of FP32) and the pending panels read to correct them (2 n FP32 values per
    pending term)."""
    steps = k * (4 * m + 2 * n_pad * pair_bytes)
    panels = 2 * (k + 1) * n_pad * 4
    rows = (delta + 1) * n_pad * 4
    pending = npend_avg * 2 * n_pad * 4
    return steps + panels + rows + pending


def stream_accuracy(P, s, d, stream0, form, cuda_stream, n_updates, seed=7):
    """max-abs error of the benchmarked form against the FP64 oracle.

    same_k: a fresh handle applies the first ``n_updates`` updates of the
    stream; sampled columns are compared with Alg 1 applied update by update
    at the same K in FP64 (oracle.alg1_stream_columns), whose initial S is the
    converged fixed point (Procedure 1 at K = 80: C^81 / (1 - C) < 1e-17).
    drift: the same form at K = 60 (truncation below 1e-13) applies the whole
    first step; sampled columns are compared with the converged fixed point of
    Eq. 1 on the graph after that step (Procedure 1 at K = 80)."""
    from oracle import simrank_oracle as O

    K_FP, K_CONV = 80, 60
    ups = stream0[:n_updates]
    Q0 = O.transition_matrix(N, s, d, sparse=True)
    rng = np.random.default_rng(seed)
    query = sorted(set(rng.choice(N, 12, replace=False).tolist())
                   | {int(x) for x in ups[-1, :2]} | {int(ups[0, 1])})
    h = P.SimRank(N, s, d, C=C, K=K, s_precision=32, aff=1, stream=cuda_stream, **form)
    h.apply_updates(ups)
    got = h.columns(np.array(query, np.int32))
    h.close()
    t0 = time.perf_counter()
    want = O.alg1_stream_columns(N, s, d, lambda c: O.partial_sim_block(Q0, c, K_FP, C),
                                 ups.tolist(), C, K, query)
    oracle_s = time.perf_counter() - t0
    same_k = float(np.max(np.abs(got - want)))
    # drift over one full step at a K where truncation has vanished
    h = P.SimRank(N, s, d, C=C, K=K_CONV, s_precision=32, aff=1, stream=cuda_stream, **form)
    h.apply_updates(stream0)
    edges = set(zip(s.tolist(), d.tolist()))
    for i, j, op in stream0.tolist():
        if op > 0:
            edges.add((i, j))
        else:
            edges.discard((i, j))
    fs = np.array([a for a, _ in edges], np.int32)
    fd = np.array([b for _, b in edges], np.int32)
    qcols = np.array(sorted(set(rng.choice(N, 12, replace=False).tolist())
                            | {int(x) for x in stream0[-1, :2]}), np.int32)
    got = h.columns(qcols)
    h.close()
    want = O.partial_sim_block(O.transition_matrix(N, fs, fd, sparse=True), qcols, K_FP, C)
    drift = float(np.max(np.abs(got - want)))
    return {"max_abs_same_k": same_k,
            "same_k": f"first {len(ups)} updates of the stream at K={K} vs FP64 Alg 1 per update "
                      f"(oracle, {len(query)} sampled columns, {oracle_s:.1f} s on the host)",
            "max_abs_vs_fixed_point_after_step": drift,
            "drift": f"the same form at K={K_CONV} after the {len(stream0)} updates of one step vs "
                     f"the converged fixed point of Eq. 1 on the final graph ({qcols.size} columns)"}


def run_gpu(args, rank, world):
    import torch

    import paper_1711_00121_gb300 as P

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod

        dist = dist_mod
        dist.init_process_group("nccl")
    stream = torch.cuda.Stream()
    total = args.warmup + args.steps
    per_step = args.updates_per_step
    s, d, streams = make_streams(total, per_step)
    # all-or-nothing per step: pack the per-step update arrays in pinned memory
    packed = []
    for st in streams:
        arr = P.updates_array(st)
        t = torch.from_numpy(arr.view(np.uint8)).pin_memory()
        packed.append((t, arr.size))
    form = dict(defer=args.defer, tc=args.tc, vec_fp64=args.vec_fp64)
    tuned = {}
    if args.tuned:
        from paper_1711_00121_gb300 import tune

        tuned = tune.tuned_knobs("stream", N, K, 32, args.vec_fp64)
        form.update(tuned)
    args.defer, args.tc = form["defer"], form["tc"]

    def handle(profile, **over):
        kw = dict(form)
        kw.update(over)
        h = P.SimRank(N, s, d, C=C, K=K, s_precision=32, aff=1, profile=profile,
                      stream=stream.cuda_stream, **kw)
        h.sync()
        return h

    def apply(h, t):
        h.apply_updates_ptr(packed[t][0].data_ptr(), packed[t][1])

    def timed_steps(h, clocks=False):
        """W untimed steps, then the K timed steps bracketed by events."""
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            for t in range(args.warmup):
                apply(h, t)
            h.sync()
            st0 = h.stats()
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            clk = ClockSampler(local) if clocks else None
            if clk:
                clk.__enter__()
            ev0.record(stream)
            for t in range(args.warmup, total):
                apply(h, t)
            ev1.record(stream)
            torch.cuda.synchronize()
            if clk:
                clk.__exit__(None, None, None)
            if dist:
                dist.barrier()
        return ev0.elapsed_time(ev1), st0, h.stats(), clk

    # ---- value: device-timed steps of the headline form (no per-launch profiling)
    sr = handle(0)
    ms, st0, st1, clk = timed_steps(sr, clocks=True)
    # drift re-anchor (FP64 Jacobi sweeps of Eq. 1 from the current S)
    ra0 = time.perf_counter()
    ra_change = sr.reanchor(2)
    sr.sync()
    reanchor_ms = (time.perf_counter() - ra0) * 1000.0 / 2
    sr.close()
    del sr
    torch.cuda.empty_cache()
    # ---- e2e: the public call with host buffers, a host read-back of two S
    # columns of the last update every step, on a second identical replica
    d2h = 0
    sr2 = handle(0)
    with torch.cuda.stream(stream):
        for t in range(args.warmup):
            apply(sr2, t)
        sr2.sync()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for t in range(args.warmup, total):
            apply(sr2, t)
            last = streams[t][-1]
            cols = sr2.columns(np.array([last[0], last[1]], np.int32), fp64=False)
            d2h = cols.nbytes
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
    sr2.close()
    del sr2
    torch.cuda.empty_cache()
    # ---- per-kernel times: a replica with CUDA events around every launch,
    # over the first timed step (kernel times, phase split, roofline)
    sr3 = handle(1)
    with torch.cuda.stream(stream):
        for t in range(args.warmup):
            apply(sr3, t)
        sr3.sync()
        pst0 = sr3.stats()
        apply(sr3, args.warmup)
        sr3.sync()
        pst1 = sr3.stats()
    sr3.close()
    del sr3
    torch.cuda.empty_cache()
    # ---- the per-edge S pass (each update's rank-2(K+1) change applied alone,
    # an HBM-bound read-modify-write of the affected tiles), profiled replica
    sr5 = handle(1, defer=0)
    pe_n = min(args.per_edge_updates, per_step)
    with torch.cuda.stream(stream):
        sr5.apply_updates(streams[0][:8])
        sr5.sync()
        e0 = sr5.stats()
        sr5.apply_updates(streams[0][8:8 + pe_n])
        sr5.sync()
        e1 = sr5.stats()
    sr5.close()
    del sr5
    torch.cuda.empty_cache()
    # ---- the other vector precision over the same timed steps
    other = None
    if total >= 2:
        o_fp64 = 0 if args.vec_fp64 else 1
        sr4 = handle(0, vec_fp64=o_fp64)
        oms, _, _, oclk = timed_steps(sr4, clocks=True)
        sr4.close()
        del sr4
        torch.cuda.empty_cache()
        other = {"vectors": "f64" if o_fp64 else "f32",
                 "value": args.steps * per_step / (oms / 1000.0), "unit": UNIT,
                 "steps": args.steps, "warmup": args.warmup, "ms_per_step": oms / args.steps,
                 "clocks": oclk.summary()}
    # max over ranks
    ms, e2e_s = max_over_ranks([ms, e2e_s], dist, "cuda")
    updates = args.steps * per_step * world
    value = updates / (ms / 1000.0)
    e2e_val = updates / e2e_s
    peak, peak_kind = read_peaks()
    # tensor peak of the operand type: FP16 = the measured bf16 burst (same
    # nominal rate); TF32 = that x 1.1/2.25 (the nominal TF32/BF16 ratio)
    tc_peak = read_bf16_peak() * (1.0 if args.tc == 2 else 1.1 / 2.25)
    tc_peak_kind = ("measured bf16 burst (FP16 has the same nominal dense rate)" if args.tc == 2
                    else "measured bf16 burst x 1.1/2.25 (nominal TF32/BF16)")
    # profiled step: the two kernels of the path
    pd = {k: pst1[k] - pst0[k] for k in ("s_update_launches", "s_bytes", "s_update_ms",
                                        "tiles_touched", "tiles_total")}
    phase = [b - a for a, b in zip(pst0["phase_ms"], pst1["phase_ms"])]
    launches = pd["s_update_launches"]
    sp_ms = pd["s_update_ms"]
    G = max(1, args.defer)
    terms = G * (K + 1)
    rg = (terms + 63) // 64 * 64 if args.tc == 2 else (terms + 31) // 32 * 32
    n_pad = (N + 127) // 128 * 128
    entries = pd["tiles_touched"] * 128 * 128
    # useful arithmetic of the method: each touched entry of S takes the
    # 2 G (K+1) rank-one terms of the pass, one FMA (2 flops) each
    method_flops = entries * 2 * terms * 2
    if args.tc:
        eb = 2 if args.tc == 2 else 4
        operand_bytes = launches * n_pad * (2 * rg) * eb * 2  # hi and lo operands
        hw_flops = entries * (2 * rg) * 2 * 3  # three split products, padded inner dim
    else:
        operand_bytes = launches * 2 * terms * n_pad * 4
        hw_flops = method_flops
    sp_bytes = pd["s_bytes"] + operand_bytes
    sp_gbs = sp_bytes / (sp_ms / 1000.0) / 1e9 if sp_ms > 0 else 0.0
    sp_tflops = hw_flops / (sp_ms / 1000.0) / 1e12 if sp_ms > 0 else 0.0
    sp_method_tflops = method_flops / (sp_ms / 1000.0) / 1e12 if sp_ms > 0 else 0.0
    # wide operands (at least 1 KB of K per row) take jobs of two tile pairs
    # sharing their row tile, one N = 256 product per split term
    paired = bool(args.tc) and 2 * rg * (2 if args.tc == 2 else 4) >= 1024
    split = "3-term " + ("FP16" if args.tc == 2 else "TF32") + " split"
    if not args.tc:
        sp_name = "k_s_update_ws (CUDA-core S pass)"
    elif paired:
        sp_name = "k_s_update_tc_pair (tcgen05, jobs of two tile pairs, N = 256, " + split + ")"
    else:
        sp_name = "k_s_update_tc (tcgen05, " + split + ", S pass)"
    if args.tc and sp_tflops / tc_peak > sp_gbs / peak:
        s_pass = {"kernel": sp_name, "bound": "tensor", "achieved": sp_tflops, "peak": tc_peak,
                  "unit": "TFLOP/s", "frac": sp_tflops / tc_peak, "peak_kind": tc_peak_kind,
                  "hbm_gbs": sp_gbs}
    else:
        s_pass = {"kernel": sp_name, "bound": "hbm", "achieved": sp_gbs, "peak": peak,
                  "unit": "GB/s", "frac": sp_gbs / peak, "peak_kind": peak_kind,
                  "tflops": sp_tflops}
    s_pass.update({"method_tflops": sp_method_tflops,
                   "method_flops_note": "4(K+1) flops per touched entry per update; the hardware "
                                        "figure counts the 3 split products and the inner "
                                        f"dimension padded from {2 * terms} to {2 * rg}"})
    # DRAM bytes (read + write) per launch from one ncu capture of each kernel
    # on this workload (n = 20,000, K = 20, 24 pending updates, FP16 split,
    # FP64 vectors, flat split); null for any other form
    profiled = ((N, K, args.defer, args.tc, args.vec_fp64) == (20000, 20, 24, 2, 1)
                and form.get("prep_item", 0) == 0)
    s_pass.update({"traffic": TRAFFIC_S_PASS if profiled else None,
                   "bytes_per_launch": sp_bytes / max(launches, 1),
                   "ms_per_launch": sp_ms / max(launches, 1), "launches": launches})
    # k_prep: one launch per update, latency-bound (L2-resident working set)
    prep_ms = phase[0]
    pair_bytes = 16 if args.vec_fp64 else 8
    npend_avg = ((G - 1) / 2.0) * (K + 1) if args.defer > 1 else 0.0
    prep_bytes_1 = stream_prep_bytes(n_pad, M, K, pair_bytes, npend_avg)
    prep_us = 1000.0 * prep_ms / per_step
    prep_gbs = prep_bytes_1 / (prep_us / 1e6) / 1e9 if prep_ms > 0 else 0.0
    prep = {"kernel": "k_prep<" + ("double" if args.vec_fp64 else "float") + ", float> "
                      "(cooperative: patch, rows of S, gamma, K recurrence steps, masks)",
            "bound": "latency", "achieved": prep_gbs, "peak": peak, "unit": "GB/s",
            "frac": prep_gbs / peak, "peak_kind": peak_kind,
            "traffic": TRAFFIC_PREP if profiled else None,
            "bytes_per_launch": prep_bytes_1, "us_per_launch": prep_us,
            "us_per_step": prep_us / (K + 4), "grid_barriers": K + 3,
            "launches": per_step,
            "note": "algorithmic bytes as stream_prep_bytes states; L2-resident working set, so "
                    "the time is set by K + 3 grid barriers and one L2 round trip per step"}
    # the per-edge S pass (each update alone)
    pe_launches = e1["s_update_launches"] - e0["s_update_launches"]
    pe_ms = e1["s_update_ms"] - e0["s_update_ms"]
    pe_terms = K + 1
    pe_rg = (pe_terms + 63) // 64 * 64 if args.tc == 2 else (pe_terms + 31) // 32 * 32
    pe_ops = pe_launches * n_pad * (2 * pe_rg) * (2 if args.tc == 2 else 4) * 2 if args.tc else \
        pe_launches * 2 * pe_terms * n_pad * 4
    pe_bytes = (e1["s_bytes"] - e0["s_bytes"]) + pe_ops
    pe_gbs = pe_bytes / (pe_ms / 1000.0) / 1e9 if pe_ms > 0 else 0.0
    s_pass_per_edge = {"kernel": ("k_s_update_tc (tcgen05, " + split + ")") if args.tc
                       else "k_s_update_ws", "bound": "hbm", "achieved": pe_gbs, "peak": peak,
                       "unit": "GB/s", "frac": pe_gbs / peak, "peak_kind": peak_kind,
                       "launches": pe_launches, "ms_per_launch": pe_ms / max(pe_launches, 1),
                       "bytes_per_launch": pe_bytes / max(pe_launches, 1),
                       "aff_tile_fraction": (e1["tiles_touched"] - e0["tiles_touched"])
                       / max(e1["tiles_total"] - e0["tiles_total"], 1),
                       "traffic": (TRAFFIC_S_PASS_EDGE if (N, K, args.tc) == (20000, 20, 2)
                                   else None),
                       "note": "each update's S change applied alone (--defer 0), S bytes of the "
                               "touched upper tiles read + written, plus the operands once"}
    dominant = s_pass if sp_ms >= prep_ms else prep
    tiles_touched = st1["tiles_touched"] - st0["tiles_touched"]
    tiles_total = st1["tiles_total"] - st0["tiles_total"]
    vec = "f64" if args.vec_fp64 else "f32"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": f"{vec} xi/eta vectors, f32 S, 3x{'f16' if args.tc == 2 else 'tf32'} split S pass",
        "data": "synthetic",
        "config": {"workload": workload_name(args), "n": N, "m": M, "C": C, "K": K,
                   "updates_per_step": per_step, "defer": args.defer, "tc": args.tc,
                   "launch": {k: form[k] for k in ("defer", "tc", "prep_item", "prep_ctas")
                              if k in form},
                   "launch_from_autotuner": bool(tuned),
                   "vectors": vec, "storage": "upper tiles",
                   "l2": "inputs larger than L2 (S is 1.6 GB FP32)",
                   "aff_tile_fraction": tiles_touched / max(tiles_total, 1),
                   "s_bytes_gbs_step": (st1["s_bytes"] - st0["s_bytes"]) / (ms / 1000.0) / 1e9,
                   "phase_us_per_update": {
                       name: 1000.0 * v / per_step
                       for name, v in zip(["prep", "patch_chain_per_step", "deferred_passes",
                                          "s_pass"], phase)},
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": dominant,
        "kernels": {"s_pass": s_pass, "prep": prep, "s_pass_per_edge": s_pass_per_edge},
        "reanchor": {"ms_per_sweep": reanchor_ms, "max_change_last_sweep": ra_change,
                     "note": "FP64 Jacobi sweep of Eq. 1 on the n=20000 S after the timed steps"},
        "other_vectors": other,
        "e2e": {"value": e2e_val, "unit": UNIT,
                "h2d_bytes_per_step": int(packed[0][1] * 16), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(st1["kernel_launches"] - st0["kernel_launches"]),
        "clocks": clk.summary(),
    }
    if rank == 0 and args.accuracy_updates > 0:
        line["accuracy"] = stream_accuracy(P, s, d, streams[0], form, stream.cuda_stream,
                                           args.accuracy_updates)
        line["max_abs"] = line["accuracy"]["max_abs_same_k"]
    if rank == 0 and not args.no_cpu_baseline:
        v, dt, n_up = cpu_baseline_sample(s, d, streams[0], 1)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": os.cpu_count(),
                                "kind": "oracle",
                                "sample": f"{n_up} unit update at full n (Alg 1, dense FP64), "
                                          f"{dt:.1f} s; S = (1-C) I stand-in (cost is value-independent)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# --------------------------------------------------------------------------
# Batched workload: directed Chung-Lu n = 100,000, m = 1.5M, exponent 2.2,
# C = 0.8, K = 25, S in FP32 (40 GB); batches of b edges, 10% of them
# attaching new nodes (source-new / target-new / both-new).  The one-shot
# rank-2r tensor-core form and the per-edge fused form are timed on the same
# batches, and each one's max-abs error against an FP64 batch recomputation
# (Procedure 1 to convergence on the final graph) is reported on sampled
# columns, so the two are compared at measured accuracy.
# --------------------------------------------------------------------------
BN, BM, BGAMMA, BC, BK = 100000, 1500000, 2.2, 0.8, 25
B_SEED = 3


def run_batched(args):
    import torch

    import paper_1711_00121_gb300 as P
    from synth import batch_with_new_nodes

    torch.cuda.set_device(0)
    b = args.batch
    BK = args.batch_k
    total = args.warmup + args.steps
    s, d = chung_lu_digraph(BN, BM, BGAMMA, BGAMMA, B_SEED)
    es = EdgeSet(BN, s, d)
    batches = []
    for t in range(total):
        ups, _ = batch_with_new_nodes(BN, s, d, b, B_SEED + 100 + t, edge_set=es)
        batches.append(ups)
    cap = es.n + 128
    # per-edge timing sample of each batch: updates between nodes that existed
    # before the batch whose edge no other update of the batch touches, so the
    # sample can run first and the rest of the batch after it
    samples, rests = [], []
    n_before = BN
    for t in range(total):
        ups = batches[t]
        keys = [(int(a), int(c)) for a, c, _ in ups.tolist()]
        cnt = {}
        for k_ in keys:
            cnt[k_] = cnt.get(k_, 0) + 1
        new_ids = max(int(ups[:, 0].max()), int(ups[:, 1].max())) + 1
        pick = [q for q, (a, c) in enumerate(keys)
                if a < n_before and c < n_before and cnt[(a, c)] == 1][:args.per_edge_sample]
        chosen = set(pick)
        samples.append(ups[pick])
        rests.append(ups[[q for q in range(len(keys)) if q not in chosen]])
        n_before = max(n_before, new_ids)
    stream = torch.cuda.Stream()
    res = {}
    per_edge_sample = min(b, args.per_edge_sample)
    for form in ("one_shot_tc", "per_edge", "per_edge_tc"):
        kw = dict(C=BC, K=BK, s_precision=32, n_capacity=cap, profile=1, stream=stream.cuda_stream)
        if form == "one_shot_tc":
            # the whole batch as one rank-2r update on the tensor cores (FP16 split)
            kw.update(apply=P.APPLY_ONE_SHOT, tc=2)
        elif form == "per_edge":
            # the plain per-edge form: each edge its own fused S pass on the CUDA cores
            kw.update(apply=P.APPLY_UNIT, defer=0, tc=0)
        else:
            # each edge its own S pass on the tensor cores (FP16 split)
            kw.update(apply=P.APPLY_UNIT, defer=0, tc=2)
        sr = P.SimRank(BN, s, d, **kw)
        with torch.cuda.stream(stream):
            for t in range(args.warmup):
                sr.apply_updates(batches[t])
            sr.sync()
            st0 = sr.stats()
            sampled = form.startswith("per_edge") and per_edge_sample < b
            pairs = []
            n_upd = 0
            with ClockSampler(0) as clk:
                if not sampled:
                    pairs.append((torch.cuda.Event(enable_timing=True),
                                  torch.cuda.Event(enable_timing=True)))
                    pairs[0][0].record(stream)
                for t in range(args.warmup, total):
                    if sampled:
                        # the per-edge cost does not depend on b: time a sample
                        # of each batch, then apply the rest of it untimed
                        pairs.append((torch.cuda.Event(enable_timing=True),
                                      torch.cuda.Event(enable_timing=True)))
                        pairs[-1][0].record(stream)
                        sr.apply_updates(samples[t])
                        pairs[-1][1].record(stream)
                        n_upd += len(samples[t])
                        sr.apply_updates(rests[t])
                    else:
                        sr.apply_updates(batches[t])
                        n_upd += b
                if not sampled:
                    pairs[0][1].record(stream)
                torch.cuda.synchronize()
            ms = sum(a.elapsed_time(z) for a, z in pairs)
            st1 = sr.stats()
        res[form] = {"updates_per_s": n_upd / (ms / 1000.0), "ms": ms, "updates_timed": n_upd,
                     "s_update_ms": st1["s_update_ms"] - st0["s_update_ms"],
                     "s_update_launches": st1["s_update_launches"] - st0["s_update_launches"],
                     "clocks": clk.summary()}
        res[form]["_handle"] = sr
    # accuracy of both forms on sampled columns against FP64 Procedure 1 on the final graph
    from oracle import simrank_oracle as O

    fs = np.array([a for a, _ in es.edges], np.int32)
    fd = np.array([x for _, x in es.edges], np.int32)
    Qf = O.transition_matrix(es.n, fs, fd, sparse=True)
    rng = np.random.default_rng(7)
    cols = np.sort(rng.choice(es.n, size=8, replace=False)).astype(np.int32)
    truth = O.partial_sim_block(Qf, cols, 110, BC)  # 0.8^111 < 1e-10
    for form in res:
        sr = res[form].pop("_handle")
        got = sr.columns(cols)
        res[form]["max_abs_vs_fp64_batch"] = float(np.max(np.abs(got - truth)))
        sr.close()
    # the one-shot form against the two per-edge forms
    one = res["one_shot_tc"]
    line = {"workload": f"batched: Chung-Lu n={BN} m={BM} exponent {BGAMMA}, C={BC}, K={BK}, "
                        f"FP32 S, batches of b={b} with 10% new nodes",
            "batch": b, "steps": args.steps, "warmup": args.warmup, "forms": res,
            "speedup_one_shot_vs_per_edge": one["updates_per_s"] / res["per_edge"]["updates_per_s"],
            "speedup_one_shot_vs_per_edge_tc": one["updates_per_s"] / res["per_edge_tc"]["updates_per_s"]}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# Many-graph workload: 512 directed Chung-Lu graphs (exponent 2.1), n uniform
# in [500, 8000], mean degree 8, C = 0.6, K = 15, S in FP32 (46 GB in all);
# each graph gets its own stream of 1-32 unit updates.  The batched form (one
# prep launch over all graphs and one S pass over all their tiles per round,
# replayed from a CUDA graph) and the per-graph-launch form run the same
# kernels on two handles over statistically identical streams.
# --------------------------------------------------------------------------
MG, MN_LO, MN_HI, MDEG, MC, MK, M_SEED = 512, 500, 8000, 8, 0.6, 15, 4


def run_multi(args):
    import torch

    import paper_1711_00121_gb300 as P
    from synth.graphs import EdgeSet as ES

    torch.cuda.set_device(0)
    G = args.graphs
    rng = np.random.default_rng(M_SEED)
    sizes = rng.integers(MN_LO, MN_HI + 1, size=G)
    counts = rng.integers(1, 33, size=G)
    graphs = []
    for g in range(G):
        n = int(sizes[g])
        s, d = chung_lu_digraph(n, MDEG * n, 2.1, 2.1, M_SEED * 100000 + g)
        graphs.append((n, s, d))
    res = {}
    from paper_1711_00121_gb300 import tune

    tuned_tc = tune.tuned_knobs("multi", MN_HI, MK, 32, 0).get("tc")
    forms = [("batched_cuda_graph", 0, args.multi_tc if tuned_tc is None else tuned_tc)]
    if tuned_tc is not None:
        # the library default (CUDA-core S pass) next to the tuner's choice
        forms.append(("batched_untuned", 0, 0))
    forms.append(("per_graph_launches", 1, forms[0][2]))
    for form, launch, mtc in forms:
        sets = [ES(n, s, d) for n, s, d in graphs]

        def draw(tag):
            return [update_stream(n, None, None, int(counts[g]), M_SEED * 7919 + 1000 * tag + g,
                                  edge_set=sets[g]) for g, (n, _, _) in enumerate(graphs)]

        warm = [draw(t) for t in range(args.warmup)]
        timed = [draw(100 + t) for t in range(args.steps)]
        t0 = time.time()
        mh = P.MultiSimRank(graphs, C=MC, K=MK, s_precision=32, multi_launch=launch,
                            init_tol=1e-9, tc=mtc)
        init_s = time.time() - t0
        packed = []
        for ups in warm + timed:
            arrs = [P.updates_array(u) for u in ups]
            off = np.zeros(G + 1, np.int64)
            off[1:] = np.cumsum([a.size for a in arrs])
            packed.append((np.ascontiguousarray(np.concatenate(arrs)), off))
        for pk, off in packed[:args.warmup]:
            mh.apply_packed(pk, off)
        mh.sync()
        st0 = mh.stats()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(0) as clk:
            ev0.record()
            h0 = time.time()
            for pk, off in packed[args.warmup:]:
                mh.apply_packed(pk, off)
            mh.sync()
            host_s = time.time() - h0
            ev1.record()
            torch.cuda.synchronize()
        st1 = mh.stats()
        n_upd = int(counts.sum()) * args.steps
        res[form] = {"updates_per_s": n_upd / host_s, "s": host_s, "updates_timed": n_upd,
                     "kernel_launches": st1["kernel_launches"] - st0["kernel_launches"],
                     "s_bytes": st1["s_bytes"] - st0["s_bytes"],
                     "hbm_gbs": (st1["s_bytes"] - st0["s_bytes"]) / host_s / 1e9,
                     "init_s": init_s, "tc": mtc, "clocks": clk.summary()}
        if form == "batched_cuda_graph":
            # accuracy: the smallest graph's final S against the FP64 oracle
            from oracle import simrank_oracle as O

            g = int(np.argmin(sizes))
            n, s0, d0 = graphs[g]
            S = O.simrank_fixed_point(O.transition_matrix(n, s0, d0, sparse=True), MC, tol=1e-15)
            allu = np.concatenate([w[g] for w in warm + timed])
            want, _ = O.sequential_unit_updates(n, s0, d0, S, allu.tolist(), MC, MK)
            res[form]["max_abs_vs_oracle_smallest_graph"] = float(np.max(np.abs(mh.dense(g) - want)))
        mh.close()
        del mh
        torch.cuda.empty_cache()
    one = res["batched_cuda_graph"]
    line = {"workload": f"many graphs: {G} directed Chung-Lu graphs (exponent 2.1), n~U[{MN_LO},{MN_HI}], "
                        f"mean degree {MDEG}, C={MC}, K={MK}, FP32 S, 1-32 unit updates per graph per call",
            "sum_S_gb": float(sum(int(((n + 127) // 128 * 128)) ** 2 * 4 for n in sizes) / 1e9),
            "updates_per_call": int(counts.sum()), "steps": args.steps, "warmup": args.warmup,
            "forms": res,
            "speedup_batched_vs_per_graph": one["updates_per_s"] / res["per_graph_launches"]["updates_per_s"],
            "autotuner": {"tc": tuned_tc, "cache": tune.cache_path()},
            "speedup_tuned_vs_untuned": (one["updates_per_s"] / res["batched_untuned"]["updates_per_s"]
                                         if "batched_untuned" in res else None)}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# Column-block workload (§7, Alg 7): directed Chung-Lu n = 2,000,000,
# m = 20,000,000 (exponent 2.1), C = 0.6, K = 15, S never stored densely;
# a stream of 32 unit updates is applied (each: Procedure 1 for its two old
# columns on the current graph, gamma, the recurrence, a panel snapshot),
# then blocks of 1024 columns are queried (Procedure 1 on the initial graph
# plus the change through every stored update).  Metric: columns/s.
# --------------------------------------------------------------------------
CN, CDEG, CC, CK, CB, CU = 2000000, 10, 0.6, 15, 1024, 32


def run_column(args):
    import torch

    import paper_1711_00121_gb300 as P
    from synth import keyed_update_stream

    torch.cuda.set_device(0)
    n = args.column_n
    m = CDEG * n
    s, d = chung_lu_digraph(n, m, 2.1, 2.1, 5)
    ups = keyed_update_stream(n, s, d, CU, 6)
    stream = torch.cuda.Stream()
    t0 = time.time()
    sr = P.SimRank(n, s, d, C=CC, K=CK, s_precision=32, mode=P.MODE_COLUMN,
                   stream=stream.cuda_stream)
    init_s = time.time() - t0
    with torch.cuda.stream(stream):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sr.apply_updates(ups)
        e1.record(stream)
        sr.sync()
        apply_ms = e0.elapsed_time(e1)
        rng = np.random.default_rng(8)
        out = torch.empty((CB, n), dtype=torch.float32, device="cuda")
        warm = np.sort(rng.choice(n, size=64, replace=False)).astype(np.int32)
        sr.columns_device(warm, out[:64])
        sr.sync()
        times = []
        with ClockSampler(0) as clk:
            for t in range(args.steps):
                cols = np.sort(rng.choice(n, size=CB, replace=False)).astype(np.int32)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                sr.columns_device(cols, out)
                b.record(stream)
                sr.sync()
                times.append(a.elapsed_time(b))
    ms = sum(times) / len(times)
    sr.close()
    line = {"workload": f"column block: directed Chung-Lu n={n} m={m} exponent 2.1, C={CC}, K={CK}, "
                        f"{CU} stored unit updates, blocks of {CB} columns, FP32",
            "metric": "columns/s", "value": CB / (ms / 1000.0), "unit": "columns/s",
            "ms_per_block": ms, "steps": args.steps, "init_s": init_s,
            "apply_ms_per_update": apply_ms / CU,
            "s_per_column_per_update": (ms / 1000.0) / CB / CU, "clocks": clk.summary()}
    if args.column_blocks:
        line["sink_blocks"] = column_sink_blocks(P, torch, n, s, d, stream)
    print(json.dumps(line), flush=True)


def column_sink_blocks(P, torch, n, s, d, stream, sinks=8, per=8):
    """Alg 7 with similar-sink blocks (§8) at the column-workload size: the
    same sinks x per insertions (per sources into each of `sinks` nodes of
    large in-degree) stored as unit updates or as one block per sink, then
    one query of CB columns; times by CUDA events."""
    rng = np.random.default_rng(13)
    indeg = np.bincount(d, minlength=n)
    top = np.argsort(-indeg)[:64]
    sink_ids = rng.choice(top, size=sinks, replace=False)
    ups = []
    for j in sink_ids.tolist():
        have = set(s[d == j].tolist())
        srcs = set()
        while len(srcs) < per:
            i = int(rng.integers(0, n))
            if i != j and i not in have:
                srcs.add(i)
        ups.extend((i, j, 1) for i in sorted(srcs))
    ups = np.array(ups, np.int32)
    cols = np.sort(rng.choice(n, size=CB, replace=False)).astype(np.int32)
    out = torch.empty((CB, n), dtype=torch.float32, device="cuda")
    res = {}
    for form, apply in (("unit_updates", P.APPLY_UNIT), ("sink_blocks", P.APPLY_SINK_BLOCKS)):
        sr = P.SimRank(n, s, d, C=CC, K=CK, s_precision=32, mode=P.MODE_COLUMN, apply=apply,
                       stream=stream.cuda_stream)
        with torch.cuda.stream(stream):
            a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            a.record(stream)
            sr.apply_updates(ups)
            b.record(stream)
            sr.columns_device(cols, out)
            c.record(stream)
            sr.sync()
        st = sr.stats()
        res[form] = {"stored_updates": st["rank_one_updates"], "store_ms": a.elapsed_time(b),
                     "query_ms": b.elapsed_time(c), "columns_per_s": CB / (b.elapsed_time(c) / 1000.0)}
        sr.close()
        torch.cuda.empty_cache()
    return {"batch": f"{sinks * per} insertions: {per} sources into each of {sinks} sinks of large "
                     f"in-degree", "query_columns": CB, "forms": res,
            "store_speedup": res["unit_updates"]["store_ms"] / res["sink_blocks"]["store_ms"],
            "query_speedup": res["unit_updates"]["query_ms"] / res["sink_blocks"]["query_ms"]}


# --------------------------------------------------------------------------
# Gradient workload (the adjoint): weighted directed Chung-Lu n = 50,000,
# m = 500,000 (exponent 2.1), weights U(0.1, 1], C = 0.6, K = 20; loss over
# 10,000 random pairs with targets U[0, 0.3]; dL/d(edge weights) by
# simrank_grad (column mode, FP64).  Central differences of the library's own
# loss on a few edges check the gradient at full size.
# --------------------------------------------------------------------------
GN, GM, GC, GK, GP = 50000, 500000, 0.6, 20, 10000


def run_grad(args):
    import torch

    import paper_1711_00121_gb300 as P
    from synth import edge_weights, query_pairs

    torch.cuda.set_device(0)
    s, d = chung_lu_digraph(GN, GM, 2.1, 2.1, 5)
    w = edge_weights(GM, 5)
    a, b, t = query_pairs(GN, GP, 5)
    kw = dict(C=GC, K=GK, s_precision=64, mode=P.MODE_COLUMN)
    sr = P.SimRank(GN, s, d, weight=w, **kw)
    L, g = sr.grad(a, b, t, GM)  # warm-up
    times = []
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            t0 = time.perf_counter()
            L, g = sr.grad(a, b, t, GM)
            times.append(time.perf_counter() - t0)
    sr.close()
    # central differences on a few edges of largest |gradient|
    rng = np.random.default_rng(9)
    idx = np.argsort(-np.abs(g))[: args.fd_edges]
    fd = []
    for e in idx.tolist():
        h = 1e-4 * float(w[e])
        vals = []
        for sign in (1.0, -1.0):
            w2 = w.astype(np.float64).copy()
            w2[e] += sign * h
            sr2 = P.SimRank(GN, s, d, weight=w2.astype(np.float32), **kw)
            # the loss at the float32-rounded weights, and the step actually taken
            Lp, _ = sr2.grad(a, b, t, GM)
            sr2.close()
            vals.append((Lp, float(np.float32(w2[e]))))
        (lp, wp), (lm, wm) = vals
        fd.append({"edge": int(e), "grad": float(g[e]), "fd": (lp - lm) / (wp - wm)})
    rel = max(abs(x["grad"] - x["fd"]) / max(abs(x["grad"]), 1e-300) for x in fd) if fd else None
    sec = sum(times) / len(times)
    line = {"workload": f"gradient: weighted directed Chung-Lu n={GN} m={GM} exponent 2.1, "
                        f"weights U(0.1,1], C={GC}, K={GK}, {GP} pairs, FP64 adjoint",
            "metric": "gradient evaluations/s", "value": 1.0 / sec, "unit": "evals/s",
            "s_per_eval": sec, "steps": args.steps, "loss": L,
            "fd_check": fd, "fd_max_rel_err": rel, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# Incremental SimRank as a batch accelerator (§1, Examples 2 and 1): the S of
# a whole graph reached either by the batch algorithm (Jacobi sweeps of Eq. 1
# on the whole graph) or by an easy S_old plus the left-out edges applied as
# updates.  Example 2: a random rooted tree on n = 20,000 nodes plus 1,000
# further edges; S_old of the tree in closed form (SR_INIT_FOREST).  Example
# 1: 8 directed Chung-Lu blocks of 2,500 nodes (mean degree 10) plus 1,000
# edges between blocks; S_old block by block (SR_INIT_COMPONENTS).  The
# left-out edges go in as sink blocks (Table 2, Alg 6), 16 pending per
# tensor-core S pass, FP32 S, FP64 vectors, K = 40.  Time = wall clock from
# the start of simrank_init to the synchronised end of the updates.
# --------------------------------------------------------------------------
AN, AEXTRA, AC, AK = 20000, 1000, 0.6, 40


def run_accelerate(args):
    import torch

    import paper_1711_00121_gb300 as P
    from oracle import simrank_oracle as O
    from synth import tree_with_extra_edges, block_graph

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    rng = np.random.default_rng(12)
    out = {}
    cases = {}
    ts, td, xs, xd = tree_with_extra_edges(AN, AEXTRA, 10)
    cases["example2_tree"] = (ts, td, xs, xd, P.INIT_FOREST)
    bs, bd, bxs, bxd = block_graph([AN // 8] * 8, 10, AEXTRA, 11)
    cases["example1_blocks"] = (bs, bd, bxs, bxd, P.INIT_COMPONENTS)
    for name, (s0, d0, xs_, xd_, form) in cases.items():
        fs = np.concatenate([s0, xs_]).astype(np.int32)
        fd = np.concatenate([d0, xd_]).astype(np.int32)
        ups = np.stack([xs_, xd_, np.ones(xs_.size, np.int32)], axis=1)
        cols = np.array(sorted(rng.choice(AN, 16, replace=False).tolist()), np.int32)
        truth = O.partial_sim_block(O.transition_matrix(AN, fs, fd, sparse=True), cols, 80, AC)
        res = {}
        for rep in range(2):  # the first round warms up the device and the library
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            hb = P.SimRank(AN, fs, fd, C=AC, K=AK, s_precision=32, stream=stream.cuda_stream)
            hb.sync()
            t_batch = time.perf_counter() - t0
            sweeps = hb.stats()["init_sweeps"]
            e_batch = float(np.max(np.abs(hb.columns(cols) - truth)))
            hb.close()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            hi = P.SimRank(AN, s0, d0, C=AC, K=AK, s_precision=32, init_form=form,
                           apply=P.APPLY_SINK_BLOCKS, defer=16, tc=2, vec_fp64=1,
                           stream=stream.cuda_stream)
            hi.sync()
            t_init = time.perf_counter() - t0
            hi.apply_updates(ups)
            hi.sync()
            t_inc = time.perf_counter() - t0
            st = hi.stats()
            e_inc = float(np.max(np.abs(hi.columns(cols) - truth)))
            hi.close()
            res = {"batch_s": t_batch, "batch_sweeps": sweeps, "batch_max_abs": e_batch,
                   "incremental_s": t_inc, "incremental_init_s": t_init,
                   "incremental_rank_one_updates": st["rank_one_updates"],
                   "incremental_max_abs": e_inc, "speedup": t_batch / t_inc}
            torch.cuda.empty_cache()
        out[name] = res
    line = {"workload": f"batch accelerator (Examples 2 and 1): n={AN}; a random rooted tree plus "
                        f"{AEXTRA} edges, and 8 Chung-Lu blocks of {AN // 8} nodes (mean degree 10) "
                        f"plus {AEXTRA} cross-block edges; C={AC}, FP32 S",
            "metric": "seconds to the S of the whole graph", "unit": "s", "higher_is_better": False,
            "forms": {"batch": "Jacobi sweeps of Eq. 1 on the whole graph (FP64 work, to 1e-13)",
                      "incremental": f"S_old (closed form / per-block sweeps) + the left-out edges as "
                                     f"sink blocks, K={AK}, 16 pending per tensor-core S pass"},
            "max_abs_vs": "FP64 Procedure 1 at K=80 on the whole graph, 16 sampled columns",
            "cases": out}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# Autotuner run: times the launch knobs on the stream workload's graph (both
# vector precisions) and the S-pass form on 64 of the many-graph workload's
# graphs, and writes the cache (SIMRANK_TUNE_CACHE, else the package's
# tuned.json) that the other workloads read with --tuned.
# --------------------------------------------------------------------------
def run_tune(args):
    import torch

    from paper_1711_00121_gb300 import tune

    torch.cuda.set_device(0)
    s, d = chung_lu_digraph(N, M, GAMMA, GAMMA, SEED_GRAPH)
    out = {"cache": tune.cache_path(), "gpu": tune.gpu_name(), "stream": {}}
    for v in (1, 0):
        r = tune.tune_stream(N, s, d, C=C, K=K, s_precision=32, vec_fp64=v, updates=192, warmup=64)
        out["stream"][f"vec_fp64={v}"] = {"knobs": r["knobs"], "us_per_update": r["us_per_update"],
                                          "candidates": len(r["measured"])}
    rng = np.random.default_rng(M_SEED)
    sizes = rng.integers(MN_LO, MN_HI + 1, size=args.graphs)[:128]
    graphs = [(int(n), *chung_lu_digraph(int(n), MDEG * int(n), 2.1, 2.1, M_SEED * 100000 + g))
              for g, n in enumerate(sizes)]
    graphs = [(n, s_, d_) for n, s_, d_ in graphs]
    r = tune.tune_multi(graphs, C=MC, K=MK, s_precision=32, updates=8)
    # the many-graph key is the workload's largest n
    entries = tune.load()
    kk = tune.key("multi", tune.gpu_name(), max(int(g[0]) for g in graphs), MK, 32, 0)
    entries[tune.key("multi", tune.gpu_name(), MN_HI, MK, 32, 0)] = entries[kk]
    tune.save(entries)
    out["multi"] = {"knobs": r["knobs"], "measured": r["measured"]}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--updates-per-step", type=int, default=UPDATES_PER_STEP,
                    help="batch size of one step (the benchmarked workload uses 1000)")
    ap.add_argument("--defer", type=int, default=16,
                    help="stream workload: rank-one updates kept pending per S pass (0 = apply each)")
    ap.add_argument("--tc", type=int, default=2,
                    help="S passes on the tensor cores: 1 = 3xTF32 split, 2 = 3xFP16 split")
    ap.add_argument("--vec-fp64", type=int, default=1,
                    help="xi/eta recurrence vectors in FP64 (default; 0 = FP32)")
    ap.add_argument("--tuned", type=int, default=1,
                    help="use the launch knobs the autotuner cached for this GPU (--workload tune)")
    ap.add_argument("--per-edge-updates", type=int, default=64,
                    help="stream workload: updates of the per-edge S-pass replica")
    ap.add_argument("--accuracy-updates", type=int, default=32,
                    help="stream workload: updates checked against the same-K FP64 oracle (0 = skip)")
    ap.add_argument("--workload", default="stream",
                    choices=["stream", "batched", "multi", "column", "grad", "accelerate", "tune"],
                    help="stream: the benchmarked update stream; batched: one-shot vs per-edge; "
                         "multi: many graphs batched vs per-graph launches; column: column-block "
                         "mode queries")
    ap.add_argument("--column-n", type=int, default=CN, help="column workload: node count")
    ap.add_argument("--column-blocks", type=int, default=1,
                    help="column workload: also store a sink-concentrated batch as blocks vs units")
    ap.add_argument("--fd-edges", type=int, default=3, help="grad workload: edges checked by FD")
    ap.add_argument("--graphs", type=int, default=MG, help="multi workload: number of graphs")
    ap.add_argument("--multi-tc", type=int, default=1,
                    help="multi workload: S passes on the tensor cores (TF32 split)")
    ap.add_argument("--batch", type=int, default=64, help="batched workload: edges per batch")
    ap.add_argument("--batch-k", type=int, default=BK,
                    help="batched workload: K (25 as configured)")
    ap.add_argument("--per-edge-sample", type=int, default=256,
                    help="batched workload: per-edge updates timed per batch")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.workload == "batched":
        run_batched(args)
        return
    if args.workload == "multi":
        run_multi(args)
        return
    if args.workload == "column":
        run_column(args)
        return
    if args.workload == "grad":
        run_grad(args)
        return
    if args.workload == "accelerate":
        run_accelerate(args)
        return
    if args.workload == "tune":
        run_tune(args)
        return
    if args.impl == "reference":
        run_reference(args, rank)
    else:
        run_gpu(args, rank, world)


if __name__ == "__main__":
    main()
