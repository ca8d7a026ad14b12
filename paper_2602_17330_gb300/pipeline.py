"""The affinity stage end to end on one GPU: pack -> sign -> band/candidates ->
self-scores -> align -> fuse, through the C ABI (``subquad.Context``).

A ``Workload`` names the method's parameters; a ``Pipeline`` keeps device
buffers between steps so a step does no allocation once warmed up.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    n: int
    k: int = 3
    bands: int = 16
    rows: int = 4
    bucket_cap: int = 0
    gap_open: int = 10
    gap_extend: int = 1
    d: int = 64
    hidden: int = 16
    pack_stride: int = 16
    binned: bool = True  # length-binned alignment (False: pairs in input order)

    @property
    def hashes(self) -> int:
        return self.bands * self.rows


# 1,000 sequences / 100 families, 3-mers, 64 hashes in 16 bands of 4, no cap,
# BLOSUM62 open 10 extend 1, d = 64, gate 3-16-1
TINY = Workload("tiny_1k", 1000)
# one donor of 1,000,000 sequences, 20,000 families of 25, 50 rare subgroups,
# the same hashing with buckets capped at 2,048
DONOR_1M = Workload("donor_1m", 1_000_000, bucket_cap=2048)
# 10,000,000 sequences of lengths 6-30 with Zipf(1.2) family sizes up to
# 50,000 (ragged buckets, no cap), 128 hashes in 32 bands of 4: a candidate set
# of ~1e10 pairs, processed as a stream of batches
ZIPF_10M = Workload("zipf_10m", 10_000_000, bands=32, rows=4, pack_stride=32)


class Pipeline:
    def __init__(self, ctx, cfg: Workload):
        self.ctx = ctx
        self.cfg = cfg
        self.torch = ctx.torch
        self.pairs_buf = None
        self.sw_buf = None
        self.fused_buf = None

    def upload(self, rep, a, b, emb, params):
        """Host numpy inputs -> device tensors (not part of a step)."""
        torch, dev = self.torch, self.ctx.device
        return dict(codes=torch.from_numpy(rep.codes).to(dev), lens=torch.from_numpy(rep.lens).to(dev),
                    a=torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to(dev),
                    b=torch.from_numpy(np.ascontiguousarray(b).view(np.int32)).to(dev),
                    emb=torch.from_numpy(np.ascontiguousarray(emb, dtype=np.float32)).to(dev),
                    params=torch.from_numpy(np.ascontiguousarray(params, dtype=np.float32)).to(dev))

    def _ensure(self, m: int):
        torch, dev = self.torch, self.ctx.device
        if self.sw_buf is None or self.sw_buf.shape[0] < m:
            self.sw_buf = torch.empty((m,), dtype=torch.int32, device=dev)
            self.fused_buf = torch.empty((m,), dtype=torch.float32, device=dev)

    def forward(self, x, marks=None):
        """One pass of the whole hot path on device-resident inputs.

        ``marks``, when given, is a callable invoked with a stage name after each
        stage is queued (the benchmark records CUDA events there)."""
        cfg, ctx = self.cfg, self.ctx
        mark = marks or (lambda name: None)
        n = int(x["lens"].shape[0])
        packed = ctx.pack(x["codes"], x["lens"], cfg.pack_stride)
        mark("pack")
        sig = ctx.sign(packed, n, cfg.k, x["a"], x["b"], cfg.bands, cfg.rows)
        mark("sign")
        if self.pairs_buf is None:
            self.pairs_buf = self.torch.empty((max(1 << 16, 8 * n), 2), dtype=self.torch.int32, device=ctx.device)
        pairs = ctx.band_candidates(sig, n, cfg.bands, cfg.rows, cfg.bucket_cap, out=self.pairs_buf)
        if pairs.data_ptr() != self.pairs_buf.data_ptr():
            self.pairs_buf = pairs  # grown after a capacity retry
        mark("band")
        m = int(pairs.shape[0])
        self._ensure(m)
        self_sc = ctx.self_scores(packed, cfg.gap_open, cfg.gap_extend, binned=cfg.binned)
        mark("self")
        sw = ctx.align_score(packed, pairs, cfg.gap_open, cfg.gap_extend, out=self.sw_buf[:m], binned=cfg.binned)
        mark("align")
        fused = ctx.fuse_forward(pairs, sw, self_sc, packed, x["emb"], x["params"], cfg.hidden,
                                 out=self.fused_buf[:m])
        mark("fuse")
        return dict(packed=packed, sig=sig, pairs=pairs, self=self_sc, sw=sw, fused=fused)

    def forward_numpy(self, rep, a, b, emb, params):
        out = self.forward(self.upload(rep, a, b, emb, params))
        cfg = self.cfg
        other = self.ctx.align_score(out["packed"], out["pairs"], cfg.gap_open, cfg.gap_extend, binned=not cfg.binned)
        self.ctx.check()
        res = dict(sig=out["sig"].cpu().numpy().view(np.uint32), pairs=out["pairs"].cpu().numpy().view(np.uint32),
                   self=out["self"].cpu().numpy(), sw=out["sw"].cpu().numpy(), fused=out["fused"].cpu().numpy())
        res["sw_binned" if not cfg.binned else "sw_plain"] = other.cpu().numpy()
        return res


def cells_of(lens: np.ndarray, pairs: np.ndarray) -> int:
    """Dynamic-programming cells of a pair list: sum of L_i * L_j."""
    if pairs.shape[0] == 0:
        return 0
    return int((lens[pairs[:, 0]].astype(np.int64) * lens[pairs[:, 1]].astype(np.int64)).sum())


class BatchedPipeline:
    """Many repertoires in one pass with no host synchronisation: pack ->
    sign -> donor-confined banding -> length-binned self-scores and alignment
    -> fusion, every count kept on the device, so the whole pass can be
    captured once as a CUDA graph and replayed.  The pair buffer has a fixed
    capacity; an overflow is reported by ``ctx.check()``."""

    def __init__(self, ctx, cfg: Workload, n: int, capacity: int):
        torch = ctx.torch
        self.ctx, self.cfg, self.n, self.capacity = ctx, cfg, n, capacity
        dev = ctx.device
        self.packed = torch.empty((n, cfg.pack_stride), dtype=torch.uint8, device=dev)
        self.sig = torch.empty((cfg.bands, n, cfg.rows), dtype=torch.int32, device=dev)
        self.pairs = torch.empty((capacity, 2), dtype=torch.int32, device=dev)
        self.num_pairs = torch.zeros((1,), dtype=torch.int64, device=dev)
        self.self_sc = torch.empty((n,), dtype=torch.int32, device=dev)
        self.sw = torch.empty((capacity,), dtype=torch.int32, device=dev)
        self.fused = torch.empty((capacity,), dtype=torch.float32, device=dev)
        self.graph = None

    def step(self, x, marks=None):
        """Queue one pass on the context's stream (no host synchronisation).
        ``marks``, when given, is called with each stage name after the stage
        is queued."""
        from . import subquad

        ctx, cfg, n = self.ctx, self.cfg, self.n
        mark = marks or (lambda name: None)
        lib, P = subquad.lib(), subquad._ptr
        subquad._check(lib.subquad_pack(ctx.handle, P(x["codes"]), int(x["codes"].shape[1]), P(x["lens"]), n,
                                        cfg.pack_stride, P(self.packed)), "subquad_pack")
        mark("pack")
        subquad._check(lib.subquad_sign(ctx.handle, P(self.packed), cfg.pack_stride, n, cfg.k, cfg.bands, cfg.rows,
                                        P(x["a"]), P(x["b"]), P(self.sig)), "subquad_sign")
        mark("sign")
        ctx.band_candidates_async(self.sig, n, cfg.bands, cfg.rows, cfg.bucket_cap, self.pairs, self.num_pairs,
                                  donor=x.get("donor"))
        mark("band")
        ctx.self_scores(self.packed, cfg.gap_open, cfg.gap_extend, out=self.self_sc, binned=True)
        mark("self")
        ctx.align_score_binned_async(self.packed, self.pairs, self.num_pairs, self.sw, cfg.gap_open, cfg.gap_extend)
        mark("align")
        ctx.fuse_forward_async(self.pairs, self.num_pairs, self.sw, self.self_sc, self.packed, x["emb"], x["params"],
                               cfg.hidden, self.fused)
        mark("fuse")

    def capture(self, x):
        """Run one pass eagerly (reserves scratch, builds tables), then capture
        the pass as a CUDA graph on the context's stream."""
        torch = self.ctx.torch
        with torch.cuda.stream(self.ctx.stream):
            self.step(x)
        self.ctx.stream.synchronize()
        self.ctx.check()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.ctx.stream):
            self.step(x)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def result(self):
        """(pairs, sw, fused, self) of the last pass as numpy, trimmed to |C|."""
        self.ctx.stream.synchronize()
        self.ctx.check()
        m = int(self.num_pairs.item())
        return dict(pairs=self.pairs[:m].cpu().numpy().view(np.uint32), sw=self.sw[:m].cpu().numpy(),
                    fused=self.fused[:m].cpu().numpy(), self=self.self_sc.cpu().numpy(), m=m)


class StreamedPipeline:
    """Candidate sets larger than one buffer: pack, sign and self-scores once,
    the band index once, then the candidates in batches of at most
    ``batch_capacity`` pairs, each aligned (length-binned) and fused.  Each
    batch is handed to the caller as device tensors (pairs, sw, fused) valid
    until the next batch; together the batches hold every candidate pair
    exactly once."""

    def __init__(self, ctx, cfg: Workload, n: int, batch_capacity: int):
        torch = ctx.torch
        self.ctx, self.cfg, self.n, self.capacity = ctx, cfg, n, batch_capacity
        dev = ctx.device
        self.packed = torch.empty((n, cfg.pack_stride), dtype=torch.uint8, device=dev)
        self.sig = torch.empty((cfg.bands, n, cfg.rows), dtype=torch.int32, device=dev)
        self.self_sc = torch.empty((n,), dtype=torch.int32, device=dev)
        self.pairs = torch.empty((batch_capacity, 2), dtype=torch.int32, device=dev)
        self.sw = torch.empty((batch_capacity,), dtype=torch.int32, device=dev)
        self.fused = torch.empty((batch_capacity,), dtype=torch.float32, device=dev)
        self.stream = None
        self.total_raw = 0

    def prepare(self, x, marks=None):
        """Pack, sign, self-scores and the band index (synchronises once).
        Returns the number of raw pairs (an upper bound of |C|)."""
        import ctypes

        from . import subquad

        ctx, cfg, n = self.ctx, self.cfg, self.n
        mark = marks or (lambda name: None)
        lib, P = subquad.lib(), subquad._ptr
        self.close()
        subquad._check(lib.subquad_pack(ctx.handle, P(x["codes"]), int(x["codes"].shape[1]), P(x["lens"]), n,
                                        cfg.pack_stride, P(self.packed)), "subquad_pack")
        subquad._check(lib.subquad_sign(ctx.handle, P(self.packed), cfg.pack_stride, n, cfg.k, cfg.bands, cfg.rows,
                                        P(x["a"]), P(x["b"]), P(self.sig)), "subquad_sign")
        mark("sign")
        ctx.self_scores(self.packed, cfg.gap_open, cfg.gap_extend, out=self.self_sc, binned=True)
        handle, total = ctypes.c_void_p(), ctypes.c_uint64(0)
        subquad._check(lib.subquad_band_stream_create(ctx.handle, P(self.sig), n, cfg.bands, cfg.rows,
                                                      cfg.bucket_cap, P(x.get("donor")), ctypes.byref(handle),
                                                      ctypes.byref(total)), "subquad_band_stream_create")
        self.stream, self.total_raw = handle, int(total.value)
        mark("index")
        return self.total_raw

    def batches(self, x, max_batches=None):
        """Yields (pairs, sw, fused) for each non-empty batch."""
        import ctypes

        from . import subquad

        ctx, cfg = self.ctx, self.cfg
        lib = subquad.lib()
        done, k = ctypes.c_int(0), 0
        while not done.value and (max_batches is None or k < max_batches):
            count = ctypes.c_int64(0)
            subquad._check(lib.subquad_band_stream_next(ctx.handle, self.stream, subquad._ptr(self.pairs),
                                                        self.capacity, ctypes.byref(count), ctypes.byref(done)),
                           "subquad_band_stream_next")
            k += 1
            m = int(count.value)
            if m == 0:
                continue
            pairs = self.pairs[:m]
            sw = ctx.align_score(self.packed, pairs, cfg.gap_open, cfg.gap_extend, out=self.sw[:m], binned=True)
            fused = ctx.fuse_forward(pairs, sw, self.self_sc, self.packed, x["emb"], x["params"], cfg.hidden,
                                     out=self.fused[:m])
            yield pairs, sw, fused

    def close(self):
        if self.stream is not None:
            from . import subquad

            subquad.lib().subquad_band_stream_destroy(self.stream)
            self.stream = None
