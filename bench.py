#!/usr/bin/env python3
"""Benchmark of the affinity stage on one donor of 1,000,000 synthetic CDR3-like
sequences: candidate pairs scored per second through the whole hot path
(pack -> MinHash sign -> LSH band/candidates/dedup -> self-scores -> Smith-
Waterman -> gated fusion), plus SW GCUPS, per-stage times, the dominant stage's
roofline, the oracle as a CPU baseline and an end-to-end number with host
buffers.  The timed step is the device-count pipeline captured once as a CUDA
graph and replayed (--no-graph: launched kernel by kernel); the eager steps,
with events between stages, are always run first for the stage breakdown.

python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun each rank processes its own donor repertoire (seeded by rank):
weak scaling, no data-path collective; rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "candidate pairs scored/s and SW GCUPS on 1 GB300 (% of int/DPX peak), batched vs plain"
UNIT = "pairs/s"
# Smith-Waterman algorithmic int32 operations per DP cell: H-diagonal + score,
# max3-with-0, H - open, E add-max, F add-max, running best max.
SW_OPS_PER_CELL = 6
# Edit-distance algorithmic int32 operations per DP cell: diagonal + substitution,
# left + insertion and its min, up + deletion and its min.
ED_OPS_PER_CELL = 5
# The integer roof: 128 integer lane operations per SM per clock (the issue
# width of an sm_103a SM) x SM count x max SM clock, the last two read from the
# device at run time.  profiles/int_issue_peak.json holds the measured rates
# (`python -m paper_2602_17330_gb300.peak --json ...` on a GB300: 2-input add
# and min/max issue at ~125-127 lane-ops/SM/clk; 3-input add, multiply-add and
# every DPX operation at 64).
INT_PEAK_FILE = os.path.join(ROOT, "profiles", "int_issue_peak.json")
INT_LANE_OPS_NOMINAL = 128.0  # 4 sub-partitions x 32 lanes of integer issue per clock
L2_FLUSH_BYTES = 512 << 20


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=1_000_000, help="sequences per donor (default: the 1M donor)")
    p.add_argument("--seed", type=int, default=0, help="data seed (rank r uses seed + r): repertoire and embeddings")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-autotune", action="store_true", help="keep the library's default launch shapes")
    p.add_argument("--no-graph", action="store_true", help="time the eager steps instead of CUDA-graph replays")
    p.add_argument("--stream-n", type=int, default=10_000_000,
                   help="sequences of the streamed Zipf workload (0: skip the streamed measurement)")
    p.add_argument("--stream-batches", type=int, default=0,
                   help="candidate batches timed in the streamed run (0: the whole candidate set)")
    p.add_argument("--stream-capacity", type=int, default=8_000_000, help="pairs per streamed batch")
    p.add_argument("--no-train", action="store_true", help="skip the gate-training measurement")
    p.add_argument("--no-topk", action="store_true", help="skip the cross-donor top-k measurement")
    p.add_argument("--no-graph-step", action="store_true",
                   help="skip the graph construction / RMT threshold / JS distance measurement")
    p.add_argument("--configs", action="store_true",
                   help="also run the long checks at their stated sizes: the 64-donor batch (about 4e7 sequences, "
                        "recall@50 on 10,000 queries against brute force) and 100 gate-training steps beside the "
                        "oracle's FP64 trajectory")
    p.add_argument("--cpu-sample-n", type=int, default=500_000, help="oracle sample for the cpu_baseline key")
    p.add_argument("--ref-sample-n", type=int, default=200_000, help="oracle sample per step of --impl reference")
    return p.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def int_lane_ops_per_sm_clk():
    """(rate, source): the nominal integer issue rate of an sm_103a SM (128
    lanes), with the fastest measured rate from the committed probe beside it."""
    if os.path.exists(INT_PEAK_FILE):
        with open(INT_PEAK_FILE) as fh:
            d = json.load(fh)
        meas = max(v for k, v in d["ops"].items() if k in ("iadd (2-input)", "imax", "__vmaxs2"))
        return INT_LANE_OPS_NOMINAL, (f"128 lane-ops/SM/clk (measured fastest integer issue {meas:.1f}: "
                                      f"{d['command']}, {d['date']})")
    return INT_LANE_OPS_NOMINAL, "128 lane-ops/SM/clk (4 x 32 integer lanes)"


def device_sm_clock(device_index: int):
    """(SM count, max SM clock in MHz) of the device, read at run time."""
    import torch

    sms = torch.cuda.get_device_properties(device_index).multi_processor_count
    mhz = None
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits", "-i",
                              str(device_index)], capture_output=True, text=True, timeout=20).stdout.strip()
        mhz = float(out.splitlines()[0])
    except (OSError, ValueError, IndexError, subprocess.TimeoutExpired):
        path = os.path.join(ROOT, "MEASURED_PEAKS.json")
        if os.path.exists(path):
            with open(path) as fh:
                mhz = float(json.load(fh).get("sm_max_mhz", 0.0)) or None
    return sms, mhz


def alu_peak_gops(sms: int, mhz: float):
    rate, src = int_lane_ops_per_sm_clk()
    return rate * sms * mhz * 1e6 / 1e9, f"{src} x {sms} SMs x {mhz:.0f} MHz"


def traffic_for(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel's
    source has not changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        table = json.load(fh)
    entry = table.get(kernel)
    if not entry:
        return None
    src = os.path.join(ROOT, entry["source"])
    if not os.path.exists(src):
        return None
    with open(src, "rb") as fh:
        digest = hashlib.sha256(fh.read()).hexdigest()
    return entry["dram_bytes_per_launch"] if digest == entry.get("source_sha256") else None


def whole_job(total_ms: float, units: float, world: int, device) -> tuple[float, float]:
    """(time of the slowest rank, units of all ranks): whole-job throughput is
    units / time.  One process per GPU; device is this rank's (CPU for gloo)."""
    if world <= 1:
        return total_ms, units
    import torch

    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    torch.distributed.all_reduce(u, op=torch.distributed.ReduceOp.SUM)
    return float(t[0]), float(u[0])


class ClockSampler:
    """nvidia-smi clock/throttle samples (every 20 ms) kept for the timed
    region only: the sampler is started and waited for before the region
    (nvidia-smi takes longer to come up than a short region lasts), every row
    carries nvidia-smi's timestamp, and stop() keeps the rows between
    mark_start() and mark_end() (20 ms of slack on either side)."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
    SLACK_S = 0.02

    def __init__(self, gpu_index: int, wait_s: float = 3.0):
        self.proc = None
        self.t0 = self.t1 = None
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(gpu_index), "-lms", "20"], stdout=self.file,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        deadline = time.time() + wait_s
        while time.time() < deadline and os.path.getsize(self.file.name) == 0 and self.proc.poll() is None:
            time.sleep(0.01)

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    @staticmethod
    def _stamp(text: str):
        import datetime

        try:
            return datetime.datetime.strptime(text.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    @classmethod
    def summarise(cls, lines, t0, t1):
        """Clock summary of the CSV rows stamped within [t0, t1] (plus slack)."""
        rows = [r.split(",") for r in lines if r.strip()]
        stamped = t0 is not None and t1 is not None and any(cls._stamp(r[0]) is not None for r in rows)
        if stamped:
            rows = [r for r in rows if (ts := cls._stamp(r[0])) is not None
                    and t0 - cls.SLACK_S <= ts <= t1 + cls.SLACK_S]
        if not rows:
            return None
        sm = [float(r[2]) for r in rows if len(r) > 2 and r[2].strip().replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if len(r) > 3 and r[3].strip().replace(".", "").isdigit()]
        reasons = sorted({cls.REASONS[k] for r in rows for k in range(4)
                          if len(r) > 6 + k and "Active" in r[6 + k] and "Not" not in r[6 + k]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "timed_region_only": stamped}

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        lines = self.file.read().strip().splitlines()
        os.unlink(self.file.name)
        return self.summarise(lines, self.t0, self.t1)


# ---------------------------------------------------------------------------
# CPU baseline / reference arm: the oracle on a bounded sample
# ---------------------------------------------------------------------------

def oracle_step(n_sample: int, seed: int = 0, threads: int = 1, with_stages: bool = False):
    """One pass of the oracle over a donor repertoire of n_sample sequences
    (same generator, families of 25, same hashing).  threads > 1 runs the
    signatures, bands, alignments and fusion over that many host threads
    (the oracle's threaded runners).  Returns
    (pairs, seconds), plus the seconds of each stage and the DP cell count
    with with_stages."""
    import oracle
    from paper_2602_17330_gb300 import pipeline, synth

    cfg = pipeline.DONOR_1M
    rep = synth.donor_repertoire(n_sample, seed=seed)
    a, b = synth.hash_coefficients(cfg.hashes, seed=0)
    emb = synth.unit_embeddings(rep.n, cfg.d, seed=seed)
    params = synth.gate_parameters(cfg.hidden, seed=0)
    idx = np.arange(rep.n, dtype=np.uint32)
    marks = [time.perf_counter()]
    if threads > 1:
        sig = oracle.sign_mt(rep.codes, rep.lens, cfg.k, a, b, threads)
        marks.append(time.perf_counter())
        pairs = oracle.candidates_mt(sig, cfg.bands, cfg.rows, cfg.bucket_cap, threads)
        marks.append(time.perf_counter())
        self_sc = oracle.sw_pairs_mt(rep.codes, rep.lens, np.stack([idx, idx], 1), threads, cfg.gap_open,
                                     cfg.gap_extend)
        marks.append(time.perf_counter())
        sw = oracle.sw_pairs_mt(rep.codes, rep.lens, pairs, threads, cfg.gap_open, cfg.gap_extend)
        marks.append(time.perf_counter())
        oracle.fuse_forward_mt(pairs, sw, self_sc, rep.lens, emb, params, cfg.hidden, threads)
    else:
        sig = oracle.sign(rep.codes, rep.lens, cfg.k, a, b)
        marks.append(time.perf_counter())
        pairs = oracle.candidates(sig, cfg.bands, cfg.rows, cfg.bucket_cap)
        marks.append(time.perf_counter())
        self_sc = oracle.self_scores(rep.codes, rep.lens, cfg.gap_open, cfg.gap_extend)
        marks.append(time.perf_counter())
        sw = oracle.sw_pairs(rep.codes, rep.lens, pairs, cfg.gap_open, cfg.gap_extend)
        marks.append(time.perf_counter())
        oracle.fuse_forward(pairs, sw, self_sc, rep.lens, emb, params, cfg.hidden)
    marks.append(time.perf_counter())
    stages = {k: marks[t + 1] - marks[t] for t, k in enumerate(["sign", "band", "self", "align", "fuse"])}
    stages["cells"] = int(pipeline.cells_of(rep.lens, pairs))
    if not with_stages:
        return pairs.shape[0], marks[-1] - marks[0]
    return pairs.shape[0], marks[-1] - marks[0], stages


def host_cpu() -> str:
    """CPU model of the host, for the baseline's record."""
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform

    return platform.processor() or platform.machine()


def workload_of(n: int):
    from paper_2602_17330_gb300 import pipeline

    base = pipeline.DONOR_1M
    return base if n == base.n else pipeline.Workload(f"donor_{n}", n, bucket_cap=base.bucket_cap)


def workload_desc(cfg) -> str:
    return (f"{cfg.name}: {cfg.n:,} CDR3-like sequences per GPU, families of 25, 50 rare subgroups; 3-mers, "
            f"{cfg.hashes} hashes in {cfg.bands}x{cfg.rows} bands, bucket cap {cfg.bucket_cap}; "
            f"BLOSUM62 o{cfg.gap_open} e{cfg.gap_extend}; d={cfg.d}, gate 3-{cfg.hidden}-1")


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    n = args.ref_sample_n
    for _ in range(args.warmup):
        oracle_step(n, seed=args.seed)
    tot_pairs, tot_s = 0, 0.0
    for _ in range(args.steps):
        p, s = oracle_step(n, seed=args.seed)
        tot_pairs += p
        tot_s += s
    value = tot_pairs / tot_s
    cfg = workload_of(args.n)
    sample = (f"oracle, single thread, full pipeline per step on a bounded sample of the workload: a {n:,}-sequence "
              f"donor from the same generator ({tot_pairs // max(args.steps, 1):,} pairs per step)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32/f64",
        "data": "synthetic", "config": {"workload": workload_desc(cfg), "n": cfg.n, "sample_n": n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_ours(args, rank: int, world: int, local_rank: int):
    import numpy as np
    import torch

    from paper_2602_17330_gb300 import _build, pipeline, subquad, synth

    if rank == 0 or not os.path.exists(subquad.LIB_PATH):
        _build.build()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    cfg = workload_of(args.n)

    rep = synth.donor_repertoire(cfg.n, seed=args.seed + rank)
    a, b = synth.hash_coefficients(cfg.hashes, seed=0)
    emb = synth.unit_embeddings(rep.n, cfg.d, seed=args.seed + rank)
    params = synth.gate_parameters(cfg.hidden, seed=0)

    stream = torch.cuda.Stream(device=dev)
    ctx = subquad.Context(local_rank, stream=stream)
    pipe = pipeline.Pipeline(ctx, cfg)  # synchronous form: e2e and the plain/batched comparison
    # the timed step: every count stays on the device, no host synchronisation
    step_pipe = pipeline.BatchedPipeline(ctx, cfg, cfg.n, capacity=8 * cfg.n)
    with torch.cuda.stream(stream):
        x = pipe.upload(rep, a, b, emb, params)
        flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
        for _ in range(max(args.warmup, 1)):
            step_pipe.step(x)
            out = pipe.forward(x)
    stream.synchronize()
    ctx.check()
    from paper_2602_17330_gb300 import autotune

    tuning = {"choice": "defaults"}
    with torch.cuda.stream(stream):
        if not args.no_autotune:
            tuning = autotune.autotune(ctx, out["packed"], out["pairs"], sig=out["sig"], n=cfg.n, bands=cfg.bands,
                                       rows=cfg.rows, bucket_cap=cfg.bucket_cap, gap_open=cfg.gap_open,
                                       gap_extend=cfg.gap_extend, reps=3, use_cache=False,
                                       fuse=(out["sw"], out["self"], x["emb"], x["params"], cfg.hidden))
        out = pipe.forward(x)
        step_pipe.step(x)
    stream.synchronize()
    ctx.check()
    pairs_np = out["pairs"].cpu().numpy().view(np.uint32)
    m = int(pairs_np.shape[0])
    if int(step_pipe.num_pairs.item()) != m:
        raise RuntimeError("the device-count step and the synchronous step disagree on |C|")
    cells = pipeline.cells_of(rep.lens, pairs_np)

    stage_names = ["pack", "sign", "band", "self", "align", "fuse"]
    steps = []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    launches0 = ctx.launch_count()
    ctx.profile(True)
    ctx.profile_reset()
    sampler = ClockSampler(local_rank) if rank == 0 else None
    if sampler:
        sampler.mark_start()
    wall0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            flush.zero_()  # evict L2 between steps (outside the events)
            ev = {"start": torch.cuda.Event(enable_timing=True)}
            ev["start"].record(stream)

            def mark(name, ev=ev):
                e = torch.cuda.Event(enable_timing=True)
                e.record(stream)
                ev[name] = e

            step_pipe.step(x, marks=mark)
            steps.append(ev)
    torch.cuda.synchronize(dev)
    launches = ctx.launch_count() - launches0
    kernel_prof = ctx.profile_read()
    ctx.profile(False)
    ctx.check()

    step_ms = [e["start"].elapsed_time(e["fuse"]) for e in steps]
    stage_ms = {}
    prev = "start"
    for s in stage_names:
        stage_ms[s] = statistics.mean(e[prev].elapsed_time(e[s]) for e in steps)
        prev = s

    # The timed steps proper: the same step captured once as a CUDA graph
    # (profiler off) and replayed K times, L2 flushed between replays outside
    # the events -- the way the batched pipeline runs in production.  The
    # eager steps above (one host launch per kernel, per-stage events) give
    # the stage breakdown and are reported beside it.
    graph_ms = None
    if not args.no_graph:
        step_pipe.capture(x)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        times = []
        with torch.cuda.stream(stream):
            for _ in range(args.steps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                step_pipe.replay()
                e1.record(stream)
                times.append((e0, e1))
        torch.cuda.synchronize(dev)
        ctx.check()
        if int(step_pipe.num_pairs.item()) != m:
            raise RuntimeError("graph replay produced a different |C|")
        graph_ms = [e0.elapsed_time(e1) for e0, e1 in times]
    wall = time.perf_counter() - wall0
    if sampler:
        sampler.mark_end()
    clocks = sampler.stop() if sampler else None

    # whole job: units over all ranks / max time over ranks
    e_max_ms, e_units = whole_job(sum(step_ms), float(m) * args.steps, world, dev)
    eager = {"value": e_units / (e_max_ms / 1e3), "unit": UNIT, "ms_per_step": e_max_ms / args.steps,
             "note": "the same step launched kernel by kernel from the host, per-stage events between stages"}
    if graph_ms is not None:
        max_ms, total_units = whole_job(sum(graph_ms), float(m) * args.steps, world, dev)
        timed_mode = "cuda graph replay"
    else:
        max_ms, total_units = e_max_ms, e_units
        timed_mode = "eager"
    value = total_units / (max_ms / 1e3)

    # batched (length-binned) vs plain alignment on the same pairs
    sw_ms = {}
    with torch.cuda.stream(stream):
        for binned in (False, True):
            times = []
            for _ in range(max(3, min(args.steps, 10))):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.align_score(out["packed"], out["pairs"], cfg.gap_open, cfg.gap_extend, out=pipe.sw_buf[:m],
                                binned=binned)
                e1.record(stream)
                times.append((e0, e1))
            stream.synchronize()
            sw_ms["binned" if binned else "plain"] = statistics.mean(a.elapsed_time(b) for a, b in times)
        # edit distance (the paper's own DP) on the same pairs, same scheduler
        ctx.set_edit_costs()
        ed_out = torch.empty((m,), dtype=torch.int32, device=dev)
        times = []
        for _ in range(max(3, min(args.steps, 10))):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.edit_distance(out["packed"], out["pairs"], out=ed_out)
            e1.record(stream)
            times.append((e0, e1))
        stream.synchronize()
        sw_ms["edit"] = statistics.mean(a.elapsed_time(b) for a, b in times)
        # three-channel fusion (alignment, embedding cosine, MinHash Jaccard) on the same pairs
        params3 = torch.from_numpy(synth.gate_parameters_mc(cfg.hidden, 3, seed=0)).to(dev)
        f3 = torch.empty((m,), dtype=torch.float32, device=dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sig_seq = ctx.sig_sequence_major(out["sig"])
        e1.record(stream)
        stream.synchronize()
        sw_ms["sig_transpose"] = e0.elapsed_time(e1)
        times = []
        for _ in range(max(3, min(args.steps, 10))):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.fuse_forward_mc(out["pairs"], out["sw"], out["self"], out["packed"], x["emb"], sig_seq, params3,
                                cfg.hidden, 3, out=f3)
            e1.record(stream)
            times.append((e0, e1))
        stream.synchronize()
        sw_ms["fuse_mc"] = statistics.mean(a.elapsed_time(b) for a, b in times)

    stream_res = train_res = topk_res = graph_res = configs = None
    if rank == 0 and world == 1:
        if not args.no_train:
            train_res = run_train(args, ctx, stream, rep, step_pipe, m)
        if not args.no_topk:
            topk_res = run_topk(args, ctx, stream)
        if not args.no_graph_step:
            graph_res = graph_step(ctx, stream, step_pipe.pairs[:m], step_pipe.fused[:m], cfg.n)
        if args.stream_n > 0:
            stream_res = run_stream(args, ctx, stream, dev, flush)
        if args.configs:
            configs = {}
            for name, fn in (("config1_tiny", lambda: run_config1(args, ctx, stream)),
                             ("seeds_1_4", lambda: run_seed_variance(args, ctx, stream, flush)),
                             ("config4_trajectory", lambda: run_config4_trajectory(args, ctx, stream, rep, step_pipe, m)),
                             ("recall_vs_band_shape", lambda: run_recall_sweep(args, ctx, stream)),
                             ("config5_full", lambda: run_config5(args, ctx, stream, flush))):
                try:
                    configs[name] = fn()
                except Exception as exc:  # a long side measurement: record its failure, keep the line
                    configs[name] = {"error": f"{type(exc).__name__}: {exc}"}
                    ctx.check() if not isinstance(exc, RuntimeError) else None

    # roofline of the dominant kernel, from the library's live per-kernel event
    # timings over the timed region (same stream as the launches)
    hbm_peak, peak_kind = measured_peaks()
    alu_peak, alu_src = alu_peak_gops(*device_sm_clock(local_rank))
    align_s = stage_ms["align"] / 1e3
    gcups = cells / align_s / 1e9
    L = rep.lens.astype(np.int64)
    hash_evals = float(np.maximum(L - cfg.k + 1, 0).sum()) * cfg.hashes
    self_cells = float((L * L).sum())
    # algorithmic work per step of each tagged kernel: (bound, amount, unit, what)
    algo = {
        "sign": ("alu", 6.0 * hash_evals, "ops", "6 integer ops per hash evaluation"),
        "band_partition": ("hbm", 4.0 * cfg.hashes * cfg.n + 8.0 * cfg.bands * cfg.n, "bytes",
                           "signatures read once, (fingerprint, id) records written once"),
        "band_group": ("hbm", 8.0 * cfg.bands * cfg.n, "bytes", "records read once"),
        "band_emit": ("hbm", 8.0 * m, "bytes", "unique pairs written once"),
        "band_pairsort": ("hbm", 16.0 * m, "bytes", "pairs read and written once"),
        "align": ("alu", SW_OPS_PER_CELL * cells, "ops", f"{SW_OPS_PER_CELL} int32 ops per DP cell"),
        "align_bin": ("hbm", 12.0 * m, "bytes", "pair list read, order written"),
        "self": ("hbm", (cfg.pack_stride + 4.0) * cfg.n, "bytes",
                 "record read, score written once (diagonal sum: the matrix is diagonally dominant)"),
        "fuse": ("hbm", 16.0 * m + cfg.n * (4.0 * cfg.d + 4 + cfg.pack_stride), "bytes",
                 "16 B per pair + each embedding row, self-score and record once"),
    }
    kernel_names = {"sign": "sign_kernel", "band_partition": "part_hist_kernel + scan + part_scatter_kernel",
                    "band_group": "part_group_kernel",
                    "band_emit": "chunk pair-count scan + band_emit_kernel", "band_pairsort": "row counting + per-row sorts (registers, warp, CTA radix)",
                    "align": "align_binned_kernel" if cfg.binned else "align_plain_kernel",
                    "align_bin": "bin_count/offsets/scatter", "self": "self_diag_kernel",
                    "fuse": "fuse_forward_kernel"}
    stage_roof = {}
    for name, (bound, amount, unit, what) in algo.items():
        ms, launches_k = kernel_prof.get(name, (0.0, 0))
        if launches_k == 0 or ms <= 0:
            continue
        per_launch_ms = ms / launches_k
        per_launch_amount = amount * args.steps / launches_k
        achieved = per_launch_amount / (per_launch_ms / 1e3) / 1e9
        peak = alu_peak if bound == "alu" else hbm_peak
        stage_roof[name] = {"kernel": kernel_names[name], "bound": bound, "ms_per_step": ms / args.steps,
                            "launches_per_step": launches_k / args.steps, "achieved": achieved, "peak": peak,
                            "unit": "Gop/s" if bound == "alu" else "GB/s", "frac": achieved / peak,
                            "algorithmic": what}
    dom = max(stage_roof, key=lambda k: stage_roof[k]["ms_per_step"])
    d = stage_roof[dom]
    roof = {"kernel": d["kernel"], "bound": d["bound"], "achieved": d["achieved"], "peak": d["peak"],
            "unit": d["unit"], "frac": d["frac"], "traffic": traffic_for(dom),
            "peak_source": (alu_src if d["bound"] == "alu"
                            else f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"),
            "algorithmic": d["algorithmic"]}

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, pipe, rep, a, b, emb, params, stream, dev, world)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        n_s = args.cpu_sample_n
        p_s, sec, st1 = oracle_step(n_s, seed=args.seed, with_stages=True)
        threads = oracle.host_threads()
        p_n, sec_n, stn = oracle_step(n_s, seed=args.seed, threads=threads, with_stages=True)

        def stage_rates(st, pairs):
            # pairs / s of each stage over the sample, alignment also in GCUPS
            out = {k: pairs / st[k] for k in ("sign", "band", "align", "fuse") if st[k] > 0}
            out["align_gcups"] = st["cells"] / st["align"] / 1e9 if st["align"] > 0 else None
            out["seconds"] = {k: st[k] for k in ("sign", "band", "self", "align", "fuse")}
            return out
        cpu = {"value": p_s / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"single-threaded oracle, full pipeline on a {n_s:,}-sequence donor from the same "
                         f"generator ({p_s:,} pairs, {sec:.1f} s)",
               "host_cpu": host_cpu(), "stages": stage_rates(st1, p_s),
               "n_core": {"value": p_n / sec_n, "unit": UNIT, "cores": threads, "kind": "oracle",
                          "stages": stage_rates(stn, p_n),
                          "sample": f"the same oracle routines over {threads} host threads (signatures, alignments "
                                    f"and fusion split by index range, bands split by band) on the same "
                                    f"donor ({p_n:,} pairs, {sec_n:.1f} s)"}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32/f32", "data": "synthetic",
            "config": {"workload": workload_desc(cfg),
                       "n": cfg.n, "seed": args.seed, "pairs_per_step": m, "cells_per_step": cells,
                       "l2": "flushed between steps",
                       "sw_kernel": ("length-binned" if cfg.binned else "plain") + " (one pair per thread)"},
            "sw_gcups": gcups, "sw_frac_of_int_peak": gcups * SW_OPS_PER_CELL / alu_peak,
            "sw_gcups_plain": cells / (sw_ms["plain"] / 1e3) / 1e9,
            "sw_gcups_binned": cells / (sw_ms["binned"] / 1e3) / 1e9,
            "fuse_mc": {"ms": sw_ms["fuse_mc"], "pairs_per_s": m / (sw_ms["fuse_mc"] / 1e3),
                        "sig_sequence_major_ms": sw_ms["sig_transpose"],
                        "hbm_frac": (16.0 * m + cfg.n * (4.0 * cfg.d + 4 + cfg.pack_stride + 4.0 * cfg.hashes))
                        / (sw_ms["fuse_mc"] / 1e3) / 1e9 / hbm_peak,
                        "note": "three-channel gated fusion (Eq. wm at M = 3, the MinHash Jaccard channel from the "
                                "signatures); algorithmic bytes 16 per pair + each sequence's embedding row, "
                                "self-score, record and signature once"},
            "edit": {"gcups": cells / (sw_ms["edit"] / 1e3) / 1e9, "ms": sw_ms["edit"],
                     "frac_of_int_peak": cells * ED_OPS_PER_CELL / (sw_ms["edit"] / 1e3) / 1e9 / alu_peak,
                     "note": f"edit distance of every candidate pair (length binning + edit_binned_kernel), "
                             f"{ED_OPS_PER_CELL} int32 ops per DP cell, default biochemical costs"},
            "stages_ms": stage_ms, "kernel_rooflines": stage_roof, "wall_s": wall, "autotune": tuning["choice"],
            "timed_mode": timed_mode, "eager": eager, "train": train_res, "topk": topk_res, "stream": stream_res,
            "graph": graph_res, "configs": configs,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
        }
        print(json.dumps(line), flush=True)


def run_train(args, ctx, stream, rep, step_pipe, m):
    """Gate training on the 1M donor's candidate list: the first 4,000,000
    pairs, family-correlated embeddings (d = 128, trained), gate 3-32-1;
    one step = fused forward + weighted BCE + adjoint (parameters and
    embeddings) + Adam, full batch, all on the device; 100 timed steps."""
    import torch

    from paper_2602_17330_gb300 import synth
    from paper_2602_17330_gb300.train import GateTrainer

    d, hidden, mt = 128, 32, min(4_000_000, m)
    steps = 100
    with torch.cuda.stream(stream):
        pairs = step_pipe.pairs[:mt]
        sw = step_pipe.sw[:mt]
        emb = torch.from_numpy(synth.family_embeddings(rep.family, d, seed=1)).to(ctx.device)
        params = torch.from_numpy(synth.gate_parameters(hidden, seed=1)).to(ctx.device)
        label, group = ctx.pair_labels(pairs, torch.from_numpy(rep.family), torch.from_numpy(rep.subgroup))
        weight = ctx.pair_weights(group, int(rep.subgroup.max()) + 1)
        for warm in range(2):  # warm-up trainer (scratch, tables), then the timed one from the same start
            tr = GateTrainer(ctx, pairs, sw, step_pipe.self_sc, step_pipe.packed, emb, params, hidden, label, weight)
            losses = torch.empty((steps,), dtype=torch.float32, device=ctx.device)
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k in range(steps if warm else 3):
                losses[k:k + 1].copy_(tr.step())
            e1.record(stream)
            stream.synchronize()
    ctx.check()
    ms = e0.elapsed_time(e1) / steps
    lv = losses.cpu().numpy()
    return {"workload": f"first {mt:,} candidate pairs of the 1M donor, d={d} (trained), gate 3-{hidden}-1, "
                        "weighted BCE, Adam lr 1e-3, full batch",
            "steps": steps, "ms_per_step": ms, "pairs_per_s": mt / (ms / 1e3),
            "loss_step_1": float(lv[0]), "loss_step_10": float(lv[9]), "loss_step_100": float(lv[99])}


def run_topk(args, ctx, stream):
    """Cross-donor top-50 retrieval on pooled donors (16 donors of 50k-200k
    sequences, 500 public families at 0.01-1% per donor): banding over the
    pooled sequences, batched alignment, top-50 of other-donor candidates for
    100,000 queries; recall@50 (ties counted) against the exhaustive top-50
    for 1,000 public-family queries."""
    import numpy as np
    import torch

    from paper_2602_17330_gb300 import pipeline, synth

    rep = synth.pooled_repertoire(16, 50_000, 200_000, seed=5)
    cfg = pipeline.Workload("pooled", rep.n)
    a, b = synth.hash_coefficients(cfg.hashes, seed=5)
    bp = pipeline.BatchedPipeline(ctx, cfg, rep.n, capacity=8 * rep.n)
    with torch.cuda.stream(stream):
        x = {"codes": torch.from_numpy(rep.codes).to(ctx.device), "lens": torch.from_numpy(rep.lens).to(ctx.device),
             "a": torch.from_numpy(a.view(np.int32)).to(ctx.device), "b": torch.from_numpy(b.view(np.int32)).to(ctx.device),
             "emb": torch.from_numpy(synth.unit_embeddings(rep.n, cfg.d, seed=5)).to(ctx.device),
             "params": torch.from_numpy(synth.gate_parameters(cfg.hidden, seed=5)).to(ctx.device)}
        bp.step(x)  # banding over the pooled donors (no donor confinement: cross-donor pairs are the point)
        x["donor"] = torch.from_numpy(rep.donor).to(ctx.device)
        stream.synchronize()
        ctx.check()
        mq = int(bp.num_pairs.item())
        pairs, scores = bp.pairs[:mq], bp.sw[:mq]
        queries = torch.from_numpy(synth.sample_queries(rep.n, 100_000, seed=5).view(np.int32)).to(ctx.device)
        index = ctx.pair_index(pairs, rep.n)
        ctx.topk_candidates(pairs, scores, rep.n, x["donor"], queries, 50, index=index)  # warm
        e0, e1, e2, e3 = (torch.cuda.Event(enable_timing=True) for _ in range(4))
        e0.record(stream)
        index = ctx.pair_index(pairs, rep.n)
        e1.record(stream)
        ids, sc = ctx.topk_candidates(pairs, scores, rep.n, x["donor"], queries, 50, index=index)
        e2.record(stream)
        # recall on 1,000 queries drawn from the public families (the sequences
        # that have relatives in other donors)
        public = np.flatnonzero((rep.family >= 0) & (rep.family < 500))
        rq = np.sort(np.random.default_rng(5).choice(public, size=min(1000, public.size), replace=False))
        sub = torch.from_numpy(rq.astype(np.int32)).to(ctx.device)
        ids_p, sc_p = ctx.topk_candidates(pairs, scores, rep.n, x["donor"], sub, 50, index=index)
        e2b = torch.cuda.Event(enable_timing=True)
        e2b.record(stream)
        _, sc_b = ctx.topk_bruteforce(bp.packed, x["donor"], sub, 50)
        e3.record(stream)
        stream.synchronize()
    ctx.check()
    g = graph_step(ctx, stream, pairs, bp.fused[:mq], rep.n, donor=x["donor"], num_donors=16)
    got = sc_p.cpu().numpy()
    best = sc_b.cpu().numpy()
    thr = best[:, 49]  # 50th-best exhaustive score (-1: fewer than 50 other-donor sequences)
    hit = ((got >= thr[:, None]) & (got >= 0)).sum(1)
    recall = float(np.minimum(hit, 50).mean() / 50.0)
    with_cand = float((sc[:, 0] >= 0).float().mean().item())
    return {"workload": f"{rep.n:,} sequences pooled from 16 donors (50k-200k each), 500 public families; "
                        f"{mq:,} candidate pairs over the pooled donors; 100,000 queries, k = 50",
            "pair_index_ms": e0.elapsed_time(e1), "topk_ms": e1.elapsed_time(e2),
            "queries_per_s": 100_000 / (e1.elapsed_time(e2) / 1e3),
            "bruteforce_1000_queries_ms": e2b.elapsed_time(e3),
            "queries_with_cross_donor_candidates": with_cand,
            "recall_at_50_public_queries": recall, "graph_and_js": g,
            "recall_note": "tie-aware recall@50 of the candidate route against the exhaustive top-50 (other donors), "
                           "on 1,000 queries drawn from public-family members"}


def run_stream(args, ctx, stream, dev, flush):
    """The streamed form on the 10M-sequence Zipf workload (lengths 6-30, 32
    bands of 4, no cap): pack, sign, self-scores and the band index once,
    then every candidate batch (by default the whole candidate set C), each
    emitted in order, aligned and fused.  Reports |C|, its DP cells, the index
    time, the total time, pairs per second and GCUPS of the alignment
    kernels (their launches timed by the library's event profiler)."""
    import numpy as np
    import torch

    from paper_2602_17330_gb300 import pipeline, synth

    base = pipeline.ZIPF_10M
    cfg = base if args.stream_n == base.n else pipeline.Workload(f"zipf_{args.stream_n}", args.stream_n, bands=32,
                                                                  rows=4, pack_stride=32)
    rep = synth.zipf_repertoire(cfg.n, seed=0)
    a, b = synth.hash_coefficients(cfg.hashes, seed=0)
    emb = synth.unit_embeddings(rep.n, cfg.d, seed=0)
    params = synth.gate_parameters(cfg.hidden, seed=0)
    sp = pipeline.StreamedPipeline(ctx, cfg, cfg.n, args.stream_capacity)
    max_batches = args.stream_batches if args.stream_batches > 0 else None
    with torch.cuda.stream(stream):
        x = pipeline.Pipeline(ctx, cfg).upload(rep, a, b, emb, params)
        lens_t = x["lens"].to(torch.int64)
        del emb
        sp.prepare(x)  # warm-up: reserves scratch
        for _ in sp.batches(x, max_batches=2):
            pass
        stream.synchronize()
        flush.zero_()
        cells = torch.zeros((), dtype=torch.int64, device=dev)
        ctx.profile(True)
        ctx.profile_reset()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        total_raw = sp.prepare(x)
        e1.record(stream)
        pairs, nb = 0, 0
        for p_, _, _ in sp.batches(x, max_batches=max_batches):
            pairs += int(p_.shape[0])
            nb += 1
            pl = p_.to(torch.int64)
            cells += (lens_t[pl[:, 0]] * lens_t[pl[:, 1]]).sum()
        e2.record(stream)
        stream.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)
    ctx.check()
    sp.close()
    prep_ms, batch_ms = e0.elapsed_time(e1), e1.elapsed_time(e2)
    cells = int(cells.item())
    align_ms = prof["align"][0] + prof["align_bin"][0]
    return {"workload": f"{cfg.name}: {cfg.n:,} sequences, lengths 6-30, Zipf(1.2) families up to 50,000, "
                        f"{cfg.hashes} hashes in {cfg.bands}x{cfg.rows} bands, no cap",
            "whole_candidate_set": max_batches is None, "candidate_pairs": pairs, "cells": cells,
            "raw_pairs_total": total_raw, "batches": nb, "batch_capacity": args.stream_capacity,
            "index_ms": prep_ms, "batches_ms": batch_ms, "total_ms": prep_ms + batch_ms,
            "value": pairs / (batch_ms / 1e3), "unit": UNIT,
            "sw_gcups": cells / (align_ms / 1e3) / 1e9 if align_ms > 0 else None,
            "note": "pack, sign, self-scores and the band index once; then candidate batches emitted in order, "
                    "aligned (length-binned) and fused; each batch synchronises once for its count; cells summed "
                    "on the device per batch; GCUPS over the profiled binning + alignment launches"}


GRAPH_TAUS = [round(0.40 + 0.02 * k, 2) for k in range(26)]  # 0.40, 0.42, ..., 0.90


def graph_step(ctx, stream, pairs, fused, n, donor=None, num_donors=0):
    """Graph construction of Algorithm 1 on the fused candidate graph: the
    RMT threshold scan (level statistics of the block-diagonal thresholded
    matrix), the pruned graph G, its connected components as clusters and,
    given donors, their cluster-mass Jensen-Shannon distances."""
    import numpy as np
    import torch

    with torch.cuda.stream(stream):
        stream.synchronize()
        t0 = time.perf_counter()
        e0 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = ctx.rmt_threshold(pairs, fused, n, GRAPH_TAUS, 64)
        t1 = time.perf_counter()
        e1, e2, e3 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e1.record(stream)
        gp, gw = ctx.graph_prune(pairs, fused, res["tau_star"])
        labels, sizes = ctx.graph_components(gp, gw, n, res["tau_star"], want_sizes=True)
        e2.record(stream)
        js = None
        if donor is not None:
            js = ctx.cluster_js(labels, donor, num_donors)
        e3.record(stream)
        stream.synchronize()
    ctx.check()
    sz = sizes.cpu().numpy()
    lab = labels.cpu().numpy()
    roots = np.flatnonzero(lab == np.arange(n))
    clusters = int((sz[roots] >= 2).sum())
    k = GRAPH_TAUS.index(res["tau_star"])
    out = {"tau_star": res["tau_star"], "thresholds_scanned": int(sum(1 for c in res["max_comp"] if c >= 0)),
           "r_at_tau_star": res["r_mean"][k], "levels_at_tau_star": res["num_levels"][k],
           "max_component_at_tau_star": res["max_comp"][k], "edges_in": int(pairs.shape[0]),
           "edges_kept": int(gp.shape[0]), "clusters_ge2": clusters,
           "scan_ms": 1e3 * (t1 - t0), "scan_gpu_ms": e0.elapsed_time(e1), "prune_components_ms": e1.elapsed_time(e2),
           "first_evaluable_tau": next((t for t, c in zip(GRAPH_TAUS, res["max_comp"]) if 0 <= c <= 64), None)}
    if js is not None:
        D = js.cpu().numpy()
        off = D[~np.eye(num_donors, dtype=bool)]
        out.update(js_ms=e2.elapsed_time(e3), js_mean=float(np.nanmean(off)), js_min=float(np.nanmin(off)),
                   js_max=float(np.nanmax(off)))
    return out


def kmer_jaccard_of(rep, pairs, k: int = 3):
    """Exact k-mer Jaccard index of each (i, j) in pairs (host; small lists)."""
    import numpy as np

    cache = {}

    def kset(r):
        if r not in cache:
            c = rep.codes[r]
            cache[r] = {tuple(c[p:p + k]) for p in range(int(rep.lens[r]) - k + 1)}
        return cache[r]

    return np.array([len(kset(int(i)) & kset(int(j))) / max(1, len(kset(int(i)) | kset(int(j)))) for i, j in pairs])


def banding_explains(rep, queries, ids, bands: int, rows: int, sample: int = 200):
    """The exhaustive top-k partners of `sample` queries: their exact 3-mer
    Jaccard index J and the banding's catch probability 1 - (1 - J^rows)^bands
    (over the hash draw); its mean is the recall the band shape can give."""
    import numpy as np

    q = queries[:sample]
    pr = [(int(a), int(b)) for a, row in zip(q, ids[:sample]) for b in row if b != 0xFFFFFFFF]
    J = kmer_jaccard_of(rep, pr)
    P = 1.0 - (1.0 - J ** rows) ** bands
    return {"pairs": len(pr), "jaccard_mean": float(J.mean()), "jaccard_p90": float(np.percentile(J, 90)),
            "catch_probability_mean": float(P.mean())}


def run_recall_sweep(args, ctx, stream):
    """Recall@50 of cross-donor retrieval against the band shape, on a pool of
    4 donors (50k-200k sequences each, 500 public families) with the same 64
    hash functions grouped as 16 bands of 4 rows, 32 of 2 or 64 of 1 (no cap;
    a shape whose candidate set exceeds 1.5e9 pairs is only counted), on 1,000
    public-family queries and 1,000 random queries, beside the banding's catch
    probability of the exhaustive top-50 partners."""
    import numpy as np
    import torch

    from paper_2602_17330_gb300 import pipeline, synth

    rep = synth.pooled_repertoire(4, 50_000, 200_000, seed=5)
    a, b = synth.hash_coefficients(64, seed=5)
    public = np.flatnonzero((rep.family >= 0) & (rep.family < 500))
    rng = np.random.default_rng(5)
    q_pub = np.sort(rng.choice(public, size=min(1000, public.size), replace=False)).astype(np.uint32)
    q_rnd = np.sort(rng.choice(rep.n, size=1000, replace=False)).astype(np.uint32)
    out = {"workload": f"{rep.n:,} sequences pooled from 4 donors, 500 public families"}
    with torch.cuda.stream(stream):
        donor = torch.from_numpy(rep.donor).to(ctx.device)
        codes, lens = torch.from_numpy(rep.codes).to(ctx.device), torch.from_numpy(rep.lens).to(ctx.device)
        packed = ctx.pack(codes, lens, 16)
        best = {}
        for name, q in (("public", q_pub), ("random", q_rnd)):
            ids_b, sc_b = ctx.topk_bruteforce(packed, donor, torch.from_numpy(q.view(np.int32)).to(ctx.device), 50)
            best[name] = (ids_b.cpu().numpy().view(np.uint32), sc_b.cpu().numpy())
        for bands, rows in ((16, 4), (32, 2), (64, 1)):
            sig = ctx.sign(packed, rep.n, 3, torch.from_numpy(a.view(np.int32)).to(ctx.device),
                           torch.from_numpy(b.view(np.int32)).to(ctx.device), bands, rows)
            count = sum(int(bt.shape[0]) for bt in ctx.band_stream(sig, rep.n, bands, rows, 0, capacity=1 << 26))
            res = {"candidate_pairs": count}
            if count < 1_500_000_000:
                pairs = ctx.band_candidates(sig, rep.n, bands, rows, 0, capacity=count + 1)
                scores = ctx.align_score(packed, pairs, binned=True)
                index = ctx.pair_index(pairs, rep.n)
                for name, q in (("public", q_pub), ("random", q_rnd)):
                    _, sc = ctx.topk_candidates(pairs, scores, rep.n, donor,
                                                torch.from_numpy(q.view(np.int32)).to(ctx.device), 50, index=index)
                    got = sc.cpu().numpy()
                    thr = best[name][1][:, 49]
                    hit = ((got >= thr[:, None]) & (got >= 0)).sum(1)
                    res[f"recall_at_50_{name}"] = float(np.minimum(hit, 50).mean() / 50.0)
                    res[f"explained_{name}"] = banding_explains(rep, q, best[name][0], bands, rows)
                del pairs, scores, index
            out[f"{bands}x{rows}"] = res
        stream.synchronize()
    ctx.check()
    return out


def run_config5(args, ctx, stream, flush):
    """The many-repertoire batch at its stated size: 64 donors of log-uniform
    sizes in 5e4..2e6, 500 public families; one batched pass (pack, sign,
    banding over the pooled donors, length-binned alignment, fusion), then the
    top-50 other-donor matches of 100,000 queries, recall@50 (ties counted)
    against the exhaustive GPU top-50 on a 10,000-query subsample of them, and
    the donors' cluster-mass JS distances."""
    import numpy as np
    import torch

    from paper_2602_17330_gb300 import pipeline, synth

    t_gen = time.perf_counter()
    rep = synth.pooled_repertoire(64, 50_000, 2_000_000, seed=5)
    t_gen = time.perf_counter() - t_gen
    cfg = pipeline.Workload("pooled_64", rep.n, bucket_cap=2048)
    a, b = synth.hash_coefficients(cfg.hashes, seed=5)
    with torch.cuda.stream(stream):
        x = {"codes": torch.from_numpy(rep.codes).to(ctx.device), "lens": torch.from_numpy(rep.lens).to(ctx.device),
             "a": torch.from_numpy(a.view(np.int32)).to(ctx.device),
             "b": torch.from_numpy(b.view(np.int32)).to(ctx.device),
             "emb": torch.from_numpy(synth.unit_embeddings(rep.n, cfg.d, seed=5)).to(ctx.device),
             "params": torch.from_numpy(synth.gate_parameters(cfg.hidden, seed=5)).to(ctx.device)}
        # |C| first, streamed (nothing kept but counts), to size the batched pass
        packed = ctx.pack(x["codes"], x["lens"], cfg.pack_stride)
        sig = ctx.sign(packed, rep.n, cfg.k, x["a"], x["b"], cfg.bands, cfg.rows)
        donor_t = torch.from_numpy(rep.donor).to(ctx.device)
        count, cross = 0, 0
        for bt in ctx.band_stream(sig, rep.n, cfg.bands, cfg.rows, cfg.bucket_cap, capacity=1 << 26):
            count += int(bt.shape[0])
            bl = bt.to(torch.int64)
            cross += int((donor_t[bl[:, 0]] != donor_t[bl[:, 1]]).sum())
        del packed, sig, bl
        stream.synchronize()
    # device memory of the batched pass: pairs, scores and fused (16 B), banding
    # scratch (~8 B) and the pair index (8 B) per pair; records, signatures and
    # band index per sequence
    need = 32 * count + 600 * rep.n
    if count >= (1 << 31) or need > 200e9:
        return {"workload": f"{rep.n:,} sequences pooled from 64 donors", "candidate_pairs": count,
                "cross_donor_pairs": cross, "generate_s": t_gen,
                "skipped": f"the batched pass would need about {need / 1e9:.0f} GB of device memory"}
    bp = pipeline.BatchedPipeline(ctx, cfg, rep.n, capacity=count + 1)
    with torch.cuda.stream(stream):
        bp.step(x)  # warm-up (scratch)
        stream.synchronize()
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bp.step(x)
        e1.record(stream)
        stream.synchronize()
        ctx.check()
        mq = int(bp.num_pairs.item())
        pairs, scores = bp.pairs[:mq], bp.sw[:mq]
        donor = torch.from_numpy(rep.donor).to(ctx.device)
        q_np = synth.sample_queries(rep.n, 100_000, seed=5)
        queries = torch.from_numpy(q_np.view(np.int32)).to(ctx.device)
        e2, e3, e4, e5 = (torch.cuda.Event(enable_timing=True) for _ in range(4))
        e2.record(stream)
        index = ctx.pair_index(pairs, rep.n)
        ids, sc = ctx.topk_candidates(pairs, scores, rep.n, donor, queries, 50, index=index)
        e3.record(stream)
        sub_idx = np.sort(np.random.default_rng(5).choice(q_np.size, 10_000, replace=False))
        sub = torch.from_numpy(q_np[sub_idx].view(np.int32)).to(ctx.device)
        e4.record(stream)
        ids_b, sc_b = ctx.topk_bruteforce(bp.packed, donor, sub, 50)
        e5.record(stream)
        stream.synchronize()
    ctx.check()
    got = sc.cpu().numpy()[sub_idx]
    best = sc_b.cpu().numpy()
    thr = best[:, 49]
    hit = ((got >= thr[:, None]) & (got >= 0)).sum(1)
    recall = float(np.minimum(hit, 50).mean() / 50.0)
    public = (rep.family[q_np[sub_idx]] >= 0) & (rep.family[q_np[sub_idx]] < 500)
    rec_pub = float(np.minimum(hit[public], 50).mean() / 50.0) if public.any() else None
    cells = pipeline.cells_of(rep.lens, pairs.cpu().numpy().view(np.uint32))
    explained = banding_explains(rep, q_np[sub_idx], ids_b.cpu().numpy().view(np.uint32), cfg.bands, cfg.rows)
    g = graph_step(ctx, stream, pairs, bp.fused[:mq], rep.n, donor=donor, num_donors=64)
    return {"workload": f"{rep.n:,} sequences pooled from 64 donors (log-uniform 5e4-2e6), 500 public families "
                        "(total public fraction log-uniform 1e-4..1e-2 per donor); 64 hashes in 16x4 bands, cap 2048",
            "generate_s": t_gen, "candidate_pairs": mq, "cross_donor_pairs": cross, "cells": cells,
            "pass_ms": e0.elapsed_time(e1),
            "pairs_per_s": mq / (e0.elapsed_time(e1) / 1e3),
            "topk_100k_queries_ms": e2.elapsed_time(e3), "bruteforce_10k_queries_ms": e4.elapsed_time(e5),
            "recall_at_50": recall, "recall_at_50_public_queries": rec_pub, "public_queries_in_sample": int(public.sum()),
            "queries_with_cross_donor_candidates": float((got[:, 0] >= 0).mean()), "graph": g,
            "recall_explained": explained,
            "recall_note": "tie-aware recall@50 of the candidate route against the exhaustive top-50 among other "
                           "donors' sequences, on a seeded 10,000-query subsample of the 100,000 queries"}


def run_seed_variance(args, ctx, stream, flush):
    """Configs 1 and 2 again with seeds 1-4 (other repertoires, embeddings
    and gate parameters from the same generators; the hash functions stay
    those of seed 0): for the 1M donor |C|, DP cells and the graph-replayed
    step time (10 replays, L2 flushed between them); for the tiny
    repertoire |C| and its equality with the oracle's candidate set."""
    import numpy as np
    import torch

    import oracle
    from paper_2602_17330_gb300 import pipeline, synth

    out = {}
    a, b = synth.hash_coefficients(64, seed=0)
    for seed in (1, 2, 3, 4):
        res = {}
        tiny = synth.tiny_repertoire(seed=seed)
        cfg1 = pipeline.TINY
        bp1 = pipeline.BatchedPipeline(ctx, cfg1, tiny.n, capacity=tiny.n * (tiny.n - 1) // 2)
        with torch.cuda.stream(stream):
            x1 = pipeline.Pipeline(ctx, cfg1).upload(tiny, a, b, synth.unit_embeddings(tiny.n, cfg1.d, seed=seed),
                                                   synth.gate_parameters(cfg1.hidden, seed=seed))
            bp1.step(x1)
        got = bp1.result()["pairs"]
        want = oracle.candidates(oracle.sign(tiny.codes, tiny.lens, cfg1.k, a, b), cfg1.bands, cfg1.rows, 0)
        res["tiny_pairs"] = int(want.shape[0])
        res["tiny_pairs_equal_oracle"] = got.shape == want.shape and bool((got == want).all())
        cfg = pipeline.DONOR_1M
        rep = synth.donor_repertoire(cfg.n, seed=seed)
        bp = pipeline.BatchedPipeline(ctx, cfg, cfg.n, capacity=8 * cfg.n)
        with torch.cuda.stream(stream):
            x = pipeline.Pipeline(ctx, cfg).upload(rep, a, b, synth.unit_embeddings(rep.n, cfg.d, seed=seed),
                                                  synth.gate_parameters(cfg.hidden, seed=seed))
        bp.capture(x)
        ts = []
        with torch.cuda.stream(stream):
            for _ in range(10):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                bp.replay()
                e1.record(stream)
                ts.append((e0, e1))
        stream.synchronize()
        ctx.check()
        m = int(bp.num_pairs.item())
        ms = float(np.median([e0.elapsed_time(e1) for e0, e1 in ts]))
        res.update(donor_pairs=m, donor_cells=int(pipeline.cells_of(rep.lens, bp.pairs[:m].cpu().numpy().view(np.uint32))),
                   donor_ms_per_step=ms, donor_pairs_per_s=m / (ms / 1e3))
        out[str(seed)] = res
        del bp, x
    vals = [r["donor_pairs_per_s"] for r in out.values()]
    out["donor_pairs_per_s_mean"] = float(np.mean(vals))
    out["donor_pairs_per_s_rel_spread"] = float((max(vals) - min(vals)) / np.mean(vals))
    return out


def run_config1(args, ctx, stream):
    """Config 1 at its stated size: the 1,000-sequence tiny repertoire through
    the device-count pipeline, captured once as a CUDA graph and replayed (200
    replays timed by events on the context stream), its pairs checked against
    the oracle's, beside the oracle's own pass over the same repertoire on one
    host core and on all of them."""
    import numpy as np
    import torch

    import oracle
    from paper_2602_17330_gb300 import pipeline, synth

    cfg = pipeline.TINY
    rep = synth.tiny_repertoire(seed=0)
    a, b = synth.hash_coefficients(cfg.hashes, seed=0)
    emb = synth.unit_embeddings(rep.n, cfg.d, seed=0)
    params = synth.gate_parameters(cfg.hidden, seed=0)
    pipe = pipeline.Pipeline(ctx, cfg)
    bp = pipeline.BatchedPipeline(ctx, cfg, rep.n, capacity=rep.n * (rep.n - 1) // 2)
    with torch.cuda.stream(stream):
        x = pipe.upload(rep, a, b, emb, params)
    bp.capture(x)
    reps = 200
    with torch.cuda.stream(stream):
        for _ in range(10):
            bp.replay()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            bp.replay()
        e1.record(stream)
        stream.synchronize()
    gpu_ms = e0.elapsed_time(e1) / reps
    got = bp.result()
    sig_o = oracle.sign(rep.codes, rep.lens, cfg.k, a, b)
    want = oracle.candidates(sig_o, cfg.bands, cfg.rows, cfg.bucket_cap)
    same = got["pairs"].shape == want.shape and bool((got["pairs"] == want).all())
    cells = int(pipeline.cells_of(rep.lens, want))
    p1, s1 = oracle_tiny_step(rep, cfg, a, b, emb, params, 1)
    threads = oracle.host_threads()
    pn, sn = oracle_tiny_step(rep, cfg, a, b, emb, params, threads)
    return {"workload": f"tiny_1k: {rep.n:,} sequences, 100 families; 64 hashes in 16x4 bands, no cap; d=64, gate 3-16-1",
            "candidate_pairs": int(want.shape[0]), "cells": cells, "pairs_equal_oracle": same,
            "gpu_ms_per_step": gpu_ms, "gpu_pairs_per_s": want.shape[0] / (gpu_ms / 1e3),
            "oracle_1core_ms": 1e3 * s1, "oracle_1core_pairs_per_s": p1 / s1,
            "oracle_ncore_ms": 1e3 * sn, "oracle_ncore_pairs_per_s": pn / sn, "oracle_threads": threads,
            "note": "one step = pack, sign, band, self-scores, align, fuse; at this size the GPU step is bound by "
                    "its ~30 dependent launches, not by any kernel"}


def oracle_tiny_step(rep, cfg, a, b, emb, params, threads):
    """The oracle's pass over one repertoire (signatures, candidates,
    self-scores, alignments, fusion) on `threads` host threads.  Returns
    (pairs, seconds)."""
    import numpy as np

    import oracle

    idx = np.arange(rep.n, dtype=np.uint32)
    t0 = time.perf_counter()
    if threads > 1:
        sig = oracle.sign_mt(rep.codes, rep.lens, cfg.k, a, b, threads)
        pairs = oracle.candidates_mt(sig, cfg.bands, cfg.rows, cfg.bucket_cap, threads)
        self_sc = oracle.sw_pairs_mt(rep.codes, rep.lens, np.stack([idx, idx], 1), threads, cfg.gap_open,
                                     cfg.gap_extend)
        sw = oracle.sw_pairs_mt(rep.codes, rep.lens, pairs, threads, cfg.gap_open, cfg.gap_extend)
        oracle.fuse_forward_mt(pairs, sw, self_sc, rep.lens, emb, params, cfg.hidden, threads)
    else:
        sig = oracle.sign(rep.codes, rep.lens, cfg.k, a, b)
        pairs = oracle.candidates(sig, cfg.bands, cfg.rows, cfg.bucket_cap)
        self_sc = oracle.self_scores(rep.codes, rep.lens, cfg.gap_open, cfg.gap_extend)
        sw = oracle.sw_pairs(rep.codes, rep.lens, pairs, cfg.gap_open, cfg.gap_extend)
        oracle.fuse_forward(pairs, sw, self_sc, rep.lens, emb, params, cfg.hidden)
    return pairs.shape[0], time.perf_counter() - t0


def run_config4_trajectory(args, ctx, stream, rep, step_pipe, m):
    """100 full-batch Adam steps of the gate (3-32-1) on the first 4,000,000
    candidate pairs with d = 128 family-correlated embeddings held fixed, on
    the GPU and, beside it, in the FP64 oracle (its threaded forward and
    parameter adjoint, its Adam) from the same start; the loss at steps 1, 10
    and 100 on both, the drift, and the largest parameter difference."""
    import numpy as np
    import torch

    import oracle
    from paper_2602_17330_gb300 import synth
    from paper_2602_17330_gb300.train import GateTrainer

    d, hidden, mt, steps = 128, 32, min(4_000_000, m), 100
    threads = oracle.host_threads()
    # the trajectory's inputs (pair list, alignment scores) from the oracle side
    a, b = synth.hash_coefficients(64, seed=0)
    sig = oracle.sign_mt(rep.codes, rep.lens, 3, a, b, threads)
    pairs_np = oracle.candidates(sig, 16, 4, 2048)[:mt]
    del sig
    sw_np = oracle.sw_pairs_mt(rep.codes, rep.lens, pairs_np, threads)
    idx = np.arange(rep.n, dtype=np.uint32)
    self_np = oracle.sw_pairs_mt(rep.codes, rep.lens, np.stack([idx, idx], 1), threads)
    emb = synth.family_embeddings(rep.family, d, seed=1)
    params0 = synth.gate_parameters(hidden, seed=1)
    with torch.cuda.stream(stream):
        pairs = torch.from_numpy(pairs_np.view(np.int32)).to(ctx.device)
        label, group = ctx.pair_labels(pairs, torch.from_numpy(rep.family), torch.from_numpy(rep.subgroup))
        ng = int(rep.subgroup.max()) + 1
        weight = ctx.pair_weights(group, ng)
        tr = GateTrainer(ctx, pairs, torch.from_numpy(sw_np).to(ctx.device), torch.from_numpy(self_np).to(ctx.device),
                         step_pipe.packed,
                         torch.from_numpy(emb).to(ctx.device), torch.from_numpy(params0).to(ctx.device), hidden,
                         label, weight, train_emb=False)
        losses = torch.empty((steps,), dtype=torch.float32, device=ctx.device)
        for k in range(steps):
            losses[k:k + 1].copy_(tr.step())
        stream.synchronize()
    ctx.check()
    gpu_loss = losses.cpu().numpy().astype(np.float64)
    gpu_params = tr.params.cpu().numpy().astype(np.float64)
    y, g = oracle.pair_labels(pairs_np, rep.family, rep.subgroup)
    w = oracle.pair_weights(g, ng)
    p = params0.astype(np.float64)
    m1, m2 = np.zeros_like(p), np.zeros_like(p)
    ora_loss = []
    t0 = time.perf_counter()
    for t in range(1, steps + 1):
        fused = oracle.fuse_forward_mt(pairs_np, sw_np, self_np, rep.lens, emb, p.astype(np.float32), hidden, threads)
        loss, dL = oracle.bce_loss(fused, y, w)
        ora_loss.append(loss)
        grad = oracle.fuse_backward_params_mt(pairs_np, sw_np, self_np, rep.lens, emb, p.astype(np.float32), hidden,
                                              dL, threads)
        oracle.adam_step(p, grad, m1, m2, t)
    ora_s = time.perf_counter() - t0
    ora_loss = np.array(ora_loss)
    rel = np.abs(gpu_loss - ora_loss) / np.abs(ora_loss)
    return {"workload": f"first {mt:,} candidate pairs of the 1M donor, d={d} (fixed), gate 3-{hidden}-1 trained, "
                        "weighted BCE, Adam lr 1e-3, 100 full-batch steps",
            "gpu_loss": {"1": gpu_loss[0], "10": gpu_loss[9], "100": gpu_loss[99]},
            "oracle_loss": {"1": ora_loss[0], "10": ora_loss[9], "100": ora_loss[99]},
            "loss_rel_drift": {"1": rel[0], "10": rel[9], "100": rel[99], "max": float(rel.max())},
            "max_param_abs_diff_after_100": float(np.abs(gpu_params - p).max()),
            "oracle_s": ora_s, "oracle_threads": threads,
            "note": "the oracle's parameters are rounded to float32 for each forward, like the GPU's"}


def run_e2e(args, pipe, rep, a, b, emb, params, stream, dev, world):
    """The same step end to end through the public API from pinned host
    buffers: every step copies its inputs host->device and its results
    (pairs, scores, fused values) device->host.  The device-count pipeline
    (no host synchronisation inside a step; a CUDA graph replay unless
    --no-graph) runs the compute; copies run on
    their own streams and overlap the neighbouring steps' compute (two input
    sets and two pipelines alternate).  The host reads step k-1's pair count
    only after step k is queued, so the compute stream never waits for the
    host.  The timed region spans all K steps, from the first input copy to
    the last result copy."""
    import numpy as np
    import torch

    from paper_2602_17330_gb300.pipeline import BatchedPipeline

    ctx, cfg = pipe.ctx, pipe.cfg
    host = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in
            dict(codes=rep.codes, lens=rep.lens, a=a.view(np.int32), b=b.view(np.int32),
                 emb=np.ascontiguousarray(emb, dtype=np.float32), params=params).items()}
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    comp, cin, cout = stream, torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    cap = 8 * rep.n
    pipes = [BatchedPipeline(ctx, cfg, rep.n, capacity=cap) for _ in range(2)]
    dev_in = [{k: torch.empty_like(v, device=dev) for k, v in host.items()} for _ in range(2)]
    use_graph = not args.no_graph
    if use_graph:  # each pipeline's step captured once on its own input buffers
        for s in range(2):
            with torch.cuda.stream(cin):
                for key in host:
                    dev_in[s][key].copy_(host[key], non_blocking=True)
            cin.synchronize()
            pipes[s].capture(dev_in[s])
    res = [[torch.empty((cap, 2), dtype=torch.int32, pin_memory=True),
            torch.empty((cap,), dtype=torch.int32, pin_memory=True),
            torch.empty((cap,), dtype=torch.float32, pin_memory=True)] for _ in range(2)]
    counts = [torch.zeros((1,), dtype=torch.int64, pin_memory=True) for _ in range(2)]
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    d2h = [0, 0]

    def h2d_step(k):
        s = k % 2
        if k >= 2:
            cin.wait_event(ev_done[s])  # step k-2 no longer reads this input set
        with torch.cuda.stream(cin):
            for key in host:
                dev_in[s][key].copy_(host[key], non_blocking=True)
        ev_in[s].record(cin)

    def compute_step(k):
        s = k % 2
        comp.wait_event(ev_in[s])
        if k >= 2:
            comp.wait_event(ev_out[s])  # step k-2's results have left this pipeline's buffers
        with torch.cuda.stream(comp):
            if use_graph:
                pipes[s].replay()
            else:
                pipes[s].step(dev_in[s])
            counts[s].copy_(pipes[s].num_pairs, non_blocking=True)
        ev_done[s].record(comp)

    def d2h_step(k):
        s = k % 2
        ev_done[s].synchronize()  # step k's count is on the host (step k+1 is already queued)
        m = int(counts[s][0])
        if m > cap:
            raise RuntimeError("pair capacity exceeded")
        p = pipes[s]
        cout.wait_event(ev_done[s])
        with torch.cuda.stream(cout):
            r = res[s]
            r[0][:m].copy_(p.pairs[:m], non_blocking=True)
            r[1][:m].copy_(p.sw[:m], non_blocking=True)
            r[2][:m].copy_(p.fused[:m], non_blocking=True)
        ev_out[s].record(cout)
        d2h[s] = m * (8 + 4 + 4)
        return m

    def run(steps):
        h2d_step(0)
        units = 0
        for k in range(steps):
            if k + 1 < steps:
                h2d_step(k + 1)
            compute_step(k)
            if k >= 1:
                units += d2h_step(k - 1)
        units += d2h_step(steps - 1)
        return units

    run(max(args.warmup, 2))
    torch.cuda.synchronize(dev)
    ctx.check()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(cin)
    units = float(run(args.steps))
    cout.wait_event(ev_out[(args.steps - 1) % 2])
    e1.record(cout)
    torch.cuda.synchronize(dev)
    ctx.check()
    total, units = whole_job(e0.elapsed_time(e1), units, world, dev)
    return {"value": units / (total / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(max(d2h)), "ms_per_step": total / args.steps,
            "overlap": "input copies, device-count compute and result copies of neighbouring steps on separate "
                       "streams; the host reads a step's pair count after the next step is queued"}


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch

        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch

            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
