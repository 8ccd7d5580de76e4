"""Autotuner for the launch shape of the update path (not in the paper).

Some knobs of the library change how an update is launched but not what it
computes (beyond rounding):

- ``defer``: how many updates' S changes one S pass applies together (the
  pass then is one rank-2G(K+1) product);
- ``tc``: the tensor-core split of that pass (1 = 3xTF32, 2 = 3xFP16);
- ``prep_item``: nonzeros per work item of the pre-update kernel's gathers
  (0: an even split of all nonzeros over the CTAs);
- ``prep_ctas``: the CTA cap of that kernel (0 = every co-resident CTA);
- for many graphs (``MultiSimRank``): ``tc`` (tensor-core or CUDA-core pass).

Their best values depend on the GPU, the graph size, K and the precisions,
so :func:`tune_stream` and :func:`tune_multi` time candidates on the caller's
own graphs (a scratch replica, CUDA events on its stream) and keep the
fastest in a JSON cache keyed by (GPU name, n rounded up to a power of two,
K, s_precision, vec_fp64).  ``SimRank(..., tuned=True)`` and
``MultiSimRank(..., tuned=True)`` read that cache.  The search is coordinate
descent: one knob at a time over its candidates, the others held at the
best values so far.

The stream replica's timing updates are insertions of edges absent from the
graph followed by their deletions, so its graph ends as it started.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

from ._binding import SimRank, MultiSimRank, default_config

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")


def cache_path() -> str:
    """The JSON cache: $SIMRANK_TUNE_CACHE if set, else tuned.json in the package."""
    return os.environ.get("SIMRANK_TUNE_CACHE", DEFAULT_CACHE)


def n_bucket(n: int) -> int:
    """n rounded up to a power of two (at least 128)."""
    return 1 << max(7, math.ceil(math.log2(max(int(n), 1))))


def key(kind: str, gpu: str, n: int, K: int, s_precision: int, vec_fp64: int) -> str:
    return f"{kind}|{gpu}|n{n_bucket(n)}|K{int(K)}|s{int(s_precision)}|v{int(vec_fp64)}"


def load(path: str | None = None) -> dict:
    path = path or cache_path()
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def save(entries: dict, path: str | None = None) -> None:
    path = path or cache_path()
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(entries, f, indent=1, sort_keys=True)
        f.write("\n")
    os.replace(tmp, path)


def lookup(kind: str, gpu: str, n: int, K: int, s_precision: int, vec_fp64: int,
           path: str | None = None) -> dict | None:
    """The cached knobs for this shape, or None."""
    e = load(path).get(key(kind, gpu, n, K, s_precision, vec_fp64))
    return dict(e["knobs"]) if e else None


def coordinate_search(space: dict, measure, start: dict | None = None):
    """Minimises measure(knobs) one knob at a time, in the order of `space`
    (knob -> candidate values), the other knobs at the best values so far.
    Returns (best knobs, best time, every (knobs, time) measured)."""
    best = dict(start) if start else {k: v[0] for k, v in space.items()}
    seen = {}

    def timed(kn):
        t = tuple(sorted(kn.items()))
        if t not in seen:
            seen[t] = float(measure(dict(kn)))
        return seen[t]

    best_t = timed(best)
    for knob, values in space.items():
        for v in values:
            cand = dict(best)
            cand[knob] = v
            t = timed(cand)
            if t < best_t:
                best, best_t = cand, t
    return best, best_t, [(dict(k), t) for k, t in seen.items()]


def gpu_name() -> str:
    import torch

    return torch.cuda.get_device_name(torch.cuda.current_device())


def timing_updates(n: int, src, dst, count: int, seed: int = 0) -> np.ndarray:
    """count / 2 insertions of absent edges into nodes that have in-neighbours
    (sinks drawn in proportion to in-degree + 1), then their deletions."""
    rng = np.random.default_rng(seed)
    src = np.asarray(src)
    dst = np.asarray(dst)
    have = set(zip(src.tolist(), dst.tolist()))
    w = np.bincount(dst, minlength=n).astype(np.float64) + 1.0
    cdf = np.cumsum(w) / w.sum()
    half = count // 2
    ins = []
    while len(ins) < half:
        j = int(min(np.searchsorted(cdf, rng.random(), side="right"), n - 1))
        i = int(rng.integers(0, n))
        if i != j and (i, j) not in have:
            have.add((i, j))
            ins.append((i, j, 1))
    return np.array(ins + [(i, j, -1) for i, j, _ in ins], np.int32)


def stream_space(K: int, num_sms: int) -> dict:
    defer = [g for g in (16, 8, 24, 32) if g * (K + 1) <= 4096]
    return {"defer": defer, "tc": [2, 1], "prep_item": [0, 1024, 512, 2048], "prep_ctas": [0, num_sms]}


def tune_stream(n, src, dst, C: float = 0.6, K: int = 15, s_precision: int = 32, vec_fp64: int = 1,
                updates: int = 96, warmup: int = 32, seed: int = 0, path: str | None = None,
                write: bool = True) -> dict:
    """Times the stream knobs on a replica of the caller's graph and caches the
    fastest.  Returns {"knobs", "us_per_update", "measured"}."""
    import torch

    stream = torch.cuda.Stream()
    ups = timing_updates(n, src, dst, updates, seed)
    warm = timing_updates(n, src, dst, warmup, seed + 1)
    num_sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    space = stream_space(K, num_sms)
    h = SimRank(n, src, dst, C=C, K=K, s_precision=s_precision, vec_fp64=vec_fp64,
                stream=stream.cuda_stream)

    def measure(kn):
        h.set_launch(**kn)
        with torch.cuda.stream(stream):
            h.apply_updates(warm)
            h.sync()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            h.apply_updates(ups)
            b.record(stream)
            h.sync()
        return 1000.0 * a.elapsed_time(b) / len(ups)

    best, t, seen = coordinate_search(space, measure)
    h.close()
    out = {"knobs": best, "us_per_update": t, "measured": seen}
    if write:
        entries = load(path)
        entries[key("stream", gpu_name(), n, K, s_precision, vec_fp64)] = out
        save(entries, path)
    return out


def tune_multi(graphs, C: float = 0.6, K: int = 15, s_precision: int = 32, updates: int = 4,
               seed: int = 0, path: str | None = None, write: bool = True, reps: int = 3) -> dict:
    """Times the many-graph S pass forms (tc = 1 tensor cores, tc = 0 CUDA
    cores) on the caller's graphs, each with `updates` insert/delete pairs
    per call, and caches the faster (each form's time: the best of `reps`
    timed calls after one untimed call).  The key's n is the largest graph's."""
    import torch

    per = [timing_updates(g[0], g[1], g[2], 2 * updates, seed + q) for q, g in enumerate(graphs)]
    res = {}
    for tc in (1, 0):
        h = MultiSimRank(graphs, C=C, K=K, s_precision=s_precision, tc=tc, init_tol=1e-9)
        h.apply_updates(per)
        h.sync()
        best = None
        for _ in range(max(1, reps)):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            h.apply_updates(per)
            b.record()
            h.sync()
            torch.cuda.synchronize()
            t = 1000.0 * a.elapsed_time(b) / sum(len(p) for p in per)
            best = t if best is None else min(best, t)
        res[tc] = best
        h.close()
    tc = min(res, key=res.get)
    out = {"knobs": {"tc": tc}, "us_per_update": res[tc],
           "measured": [({"tc": k}, v) for k, v in res.items()]}
    if write:
        nmax = max(int(g[0]) for g in graphs)
        entries = load(path)
        entries[key("multi", gpu_name(), nmax, K, s_precision, 0)] = out
        save(entries, path)
    return out


def tuned_knobs(kind: str, n: int, K: int, s_precision: int, vec_fp64: int,
                path: str | None = None) -> dict:
    """The cached knobs for the current GPU (empty when nothing is cached)."""
    try:
        gpu = gpu_name()
    except Exception:
        return {}
    return lookup(kind, gpu, n, K, s_precision, vec_fp64, path) or {}


__all__ = ["tune_stream", "tune_multi", "tuned_knobs", "coordinate_search", "lookup", "key",
           "n_bucket", "cache_path", "timing_updates", "stream_space", "default_config"]
