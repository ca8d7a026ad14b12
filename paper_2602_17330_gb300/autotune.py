"""Autotuner for the library's launch-shape knobs.

Each knob changes only how work is mapped onto the GB300 (never a result):
* TUNE_ALIGN_SHAPE -- batched Smith-Waterman launch shape (256 threads x 2
  blocks per SM with 128 registers, 128 x 3 with 168 registers, or one block
  of 384 threads per SM with split score tables);
* TUNE_BAND_PART_LOG2 -- log2 of the target keys per hash partition of the
  banding stage (each partition is grouped by one CTA in shared memory);
* TUNE_FUSE_LANES -- lanes per pair of the fusion forward (4 or 8).

``autotune`` times every candidate on the caller's own workload with CUDA
events on the context's stream, keeps the fastest, and caches the choice per
device and workload shape in a JSON file next to this module.
"""
from __future__ import annotations

import json
import os
import statistics

from . import subquad

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tuning.json")

CANDIDATES = {
    subquad.TUNE_ALIGN_SHAPE: (0, 1, 2),
    subquad.TUNE_BAND_PART_LOG2: (10, 11),
    subquad.TUNE_FUSE_LANES: (4, 8),
}


def _time(ctx, fn, reps: int) -> float:
    torch = ctx.torch
    s = ctx.stream
    fn()  # warm
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        fn()
        e1.record(s)
        times.append((e0, e1))
    s.synchronize()
    return statistics.median(a.elapsed_time(b) for a, b in times)


def _key(ctx, shape: str) -> str:
    return f"{ctx.torch.cuda.get_device_name(ctx.device)}|{shape}"


def load_cached(ctx, shape: str) -> dict | None:
    if not os.path.exists(CACHE):
        return None
    try:
        with open(CACHE) as fh:
            entry = json.load(fh).get(_key(ctx, shape))
    except (OSError, ValueError):
        return None
    if entry:
        for k, v in entry["choice"].items():
            ctx.set_tuning(int(k), int(v))
    return entry


def autotune(ctx, packed, pairs, sig=None, n: int = 0, bands: int = 0, rows: int = 0, bucket_cap: int = 0,
             gap_open: int = 10, gap_extend: int = 1, reps: int = 5, shape: str = "", use_cache: bool = True,
             fuse=None) -> dict:
    """Pick the fastest setting of every knob on this workload (the fusion
    knob when ``fuse`` = (sw, self_scores, emb, params, hidden) is given); returns
    {"choice": {knob: value}, "timings_ms": {knob: {value: ms}}}."""
    if use_cache and shape:
        cached = load_cached(ctx, shape)
        if cached:
            return cached
    out_sw = ctx.torch.empty((int(pairs.shape[0]),), dtype=ctx.torch.int32, device=ctx.device)
    timings, choice = {}, {}
    knob = subquad.TUNE_ALIGN_SHAPE
    timings[knob] = {}
    for v in CANDIDATES[knob]:
        ctx.set_tuning(knob, v)
        timings[knob][v] = _time(ctx, lambda: ctx.align_score(packed, pairs, gap_open, gap_extend, out=out_sw,
                                                              binned=True), reps)
    choice[knob] = min(timings[knob], key=timings[knob].get)
    ctx.set_tuning(knob, choice[knob])
    if sig is not None and n > 1:
        knob = subquad.TUNE_BAND_PART_LOG2
        timings[knob] = {}
        buf = ctx.torch.empty((max(int(pairs.shape[0]), 1), 2), dtype=ctx.torch.int32, device=ctx.device)
        for v in CANDIDATES[knob]:
            ctx.set_tuning(knob, v)
            timings[knob][v] = _time(ctx, lambda: ctx.band_candidates(sig, n, bands, rows, bucket_cap, out=buf),
                                     max(2, reps // 2))
        choice[knob] = min(timings[knob], key=timings[knob].get)
        ctx.set_tuning(knob, choice[knob])
    if fuse is not None:
        sw, self_sc, emb, params, hidden = fuse
        knob = subquad.TUNE_FUSE_LANES
        timings[knob] = {}
        out_f = ctx.torch.empty((int(pairs.shape[0]),), dtype=ctx.torch.float32, device=ctx.device)
        for v in CANDIDATES[knob]:
            ctx.set_tuning(knob, v)
            timings[knob][v] = _time(ctx, lambda: ctx.fuse_forward(pairs, sw, self_sc, packed, emb, params, hidden,
                                                                   out=out_f), reps)
        choice[knob] = min(timings[knob], key=timings[knob].get)
        ctx.set_tuning(knob, choice[knob])
    result = {"choice": {str(k): v for k, v in choice.items()},
              "timings_ms": {str(k): {str(v): t for v, t in d.items()} for k, d in timings.items()}}
    if shape:
        try:
            data = {}
            if os.path.exists(CACHE):
                with open(CACHE) as fh:
                    data = json.load(fh)
            data[_key(ctx, shape)] = result
            tmp = CACHE + f".tmp{os.getpid()}"
            with open(tmp, "w") as fh:
                json.dump(data, fh, indent=1)
            os.replace(tmp, CACHE)
        except OSError:
            pass
    return result
