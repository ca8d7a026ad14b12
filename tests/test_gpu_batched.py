"""GPU parity of the batched, graph-capturable pipeline: many donors in one
pass with every count on the device must give exactly what separate
per-donor passes give (pairs with global ids, alignment scores, fused scores),
eagerly and replayed from a captured CUDA graph."""
import numpy as np
import pytest

from paper_2602_17330_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


@pytest.fixture(scope="module")
def ctx(torch):
    from paper_2602_17330_gb300 import _build, subquad

    _build.build()
    stream = torch.cuda.Stream()
    c = subquad.Context(0, stream=stream)
    yield c
    c.close()


def per_donor_reference(ctx, torch, rep, cfg, a, b, emb, params):
    """The plain pipeline run donor by donor, ids shifted to global."""
    from paper_2602_17330_gb300 import pipeline

    out_pairs, out_sw, out_fused = [], [], []
    starts = np.concatenate([[0], np.cumsum(np.bincount(rep.donor))])
    for d in range(len(starts) - 1):
        lo, hi = int(starts[d]), int(starts[d + 1])
        sub = synth.Repertoire(rep.codes[lo:hi], rep.lens[lo:hi], rep.family[lo:hi], rep.subgroup[lo:hi], rep.freq)
        with torch.cuda.stream(ctx.stream):
            res = pipeline.Pipeline(ctx, cfg).forward_numpy(sub, a, b, emb[lo:hi], params)
        out_pairs.append(res["pairs"].astype(np.int64) + lo)
        out_sw.append(res["sw"])
        out_fused.append(res["fused"])
    pairs = np.concatenate(out_pairs)
    order = np.lexsort((pairs[:, 1], pairs[:, 0]))
    return pairs[order].astype(np.uint32), np.concatenate(out_sw)[order], np.concatenate(out_fused)[order]


@pytest.mark.parametrize("cap", [0, 3])
def test_batched_equals_per_donor(ctx, torch, cap):
    from paper_2602_17330_gb300 import pipeline

    rep = synth.pooled_repertoire(6, 400, 6000, n_public=30, public_lo=0.05, public_hi=0.3, seed=8)
    cfg = pipeline.Workload("pooled", rep.n, bucket_cap=cap)
    a, b = synth.hash_coefficients(cfg.hashes, seed=8)
    emb = synth.unit_embeddings(rep.n, cfg.d, seed=8)
    params = synth.gate_parameters(cfg.hidden, seed=8)
    want_pairs, want_sw, want_fused = per_donor_reference(ctx, torch, rep, cfg, a, b, emb, params)
    bp = pipeline.BatchedPipeline(ctx, cfg, rep.n, capacity=max(4 * want_pairs.shape[0], 1024))
    x = pipeline.Pipeline(ctx, cfg).upload(rep, a, b, emb, params)
    x["donor"] = torch.from_numpy(rep.donor).to(ctx.device)
    with torch.cuda.stream(ctx.stream):
        bp.step(x)
    got = bp.result()
    assert got["m"] == want_pairs.shape[0]
    assert (got["pairs"] == want_pairs).all()
    assert (got["sw"] == want_sw).all()
    assert np.array_equal(got["fused"], want_fused)  # same kernels, same inputs: bitwise


def test_graph_replay_equals_eager(ctx, torch, oracle_mod):
    from paper_2602_17330_gb300 import pipeline

    rep = synth.pooled_repertoire(4, 1000, 8000, n_public=30, public_lo=0.05, public_hi=0.3, seed=9)
    cfg = pipeline.Workload("pooled", rep.n, bucket_cap=2048)
    a, b = synth.hash_coefficients(cfg.hashes, seed=9)
    emb = synth.unit_embeddings(rep.n, cfg.d, seed=9)
    params = synth.gate_parameters(cfg.hidden, seed=9)
    x = pipeline.Pipeline(ctx, cfg).upload(rep, a, b, emb, params)
    x["donor"] = torch.from_numpy(rep.donor).to(ctx.device)
    bp = pipeline.BatchedPipeline(ctx, cfg, rep.n, capacity=1 << 20)
    bp.capture(x)
    eager = bp.result()
    for _ in range(2):
        bp.num_pairs.zero_()
        bp.replay()
        got = bp.result()
        assert got["m"] == eager["m"] and (got["pairs"] == eager["pairs"]).all()
        assert (got["sw"] == eager["sw"]).all() and np.array_equal(got["fused"], eager["fused"])
    # and the pairs are exactly the oracle's donor-confined candidate set
    sig = oracle_mod.sign(rep.codes, rep.lens, cfg.k, a, b)
    starts = np.concatenate([[0], np.cumsum(np.bincount(rep.donor))])
    want = []
    for d in range(len(starts) - 1):
        lo, hi = int(starts[d]), int(starts[d + 1])
        want.append(oracle_mod.candidates(sig[lo:hi], cfg.bands, cfg.rows, cfg.bucket_cap).astype(np.int64) + lo)
    want = np.concatenate(want)
    want = want[np.lexsort((want[:, 1], want[:, 0]))].astype(np.uint32)
    assert (got["pairs"] == want).all()
    assert (got["sw"] == oracle_mod.sw_pairs(rep.codes, rep.lens, want)).all()


def test_capacity_overflow_is_reported(ctx, torch):
    from paper_2602_17330_gb300 import pipeline, subquad

    rep = synth.pooled_repertoire(2, 2000, 3000, n_public=10, public_lo=0.05, public_hi=0.2, seed=10)
    cfg = pipeline.Workload("pooled", rep.n)
    a, b = synth.hash_coefficients(cfg.hashes, seed=10)
    x = pipeline.Pipeline(ctx, cfg).upload(rep, a, b, synth.unit_embeddings(rep.n, cfg.d), synth.gate_parameters(16))
    bp = pipeline.BatchedPipeline(ctx, cfg, rep.n, capacity=4)
    with torch.cuda.stream(ctx.stream):
        bp.step(x)
    ctx.stream.synchronize()
    with pytest.raises(subquad.SubquadError) as ei:
        ctx.check()
    assert ei.value.status == subquad.SUBQUAD_ERR_CAPACITY
    assert int(bp.num_pairs.item()) > 4
