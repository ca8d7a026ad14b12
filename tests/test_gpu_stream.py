"""GPU parity for the streamed candidate form: the batches partition the
candidate set (every pair exactly once), each batch is sorted, and together
they equal the oracle's candidate list."""
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
    c = subquad.Context(0)
    yield c
    c.close()


def to_np(t):
    return t.detach().cpu().numpy()


def collect(ctx, sig, n, bands, rows, cap, capacity, donor=None):
    batches = [to_np(bt).view(np.uint32).copy() for bt in
               ctx.band_stream(sig, n, bands, rows, cap, donor=donor, capacity=capacity)]
    for bt in batches:
        key = bt[:, 0].astype(np.uint64) << np.uint64(32) | bt[:, 1].astype(np.uint64)
        assert (np.diff(key.astype(np.int64)) > 0).all(), "a batch is not sorted"
    allp = np.concatenate(batches) if batches else np.zeros((0, 2), np.uint32)
    key = allp[:, 0].astype(np.uint64) << np.uint64(32) | allp[:, 1].astype(np.uint64)
    order = np.argsort(key, kind="stable")
    return allp[order], len(batches)


@pytest.mark.parametrize("cap,capacity", [(0, 32), (4, 1000), (2048, 100_000), (0, 1 << 22)])
def test_stream_equals_oracle(ctx, torch, oracle_mod, cap, capacity):
    rep = synth.donor_repertoire(20_000, seed=6)
    a, b = synth.hash_coefficients(64, seed=6)
    packed = ctx.pack(torch.from_numpy(rep.codes), torch.from_numpy(rep.lens), 16)
    sig = ctx.sign(packed, rep.n, 3, torch.from_numpy(a.view(np.int32)), torch.from_numpy(b.view(np.int32)), 16, 4)
    got, nb = collect(ctx, sig, rep.n, 16, 4, cap, capacity)
    want = oracle_mod.candidates(oracle_mod.sign(rep.codes, rep.lens, 3, a, b), 16, 4, cap)
    assert got.shape == want.shape and (got == want).all()
    if capacity == 32:
        assert nb > 100  # many small batches


def test_stream_equals_batched_with_donors(ctx, torch):
    rep = synth.pooled_repertoire(6, 300, 2000, n_public=30, public_lo=0.05, public_hi=0.3, seed=12)
    a, b = synth.hash_coefficients(64, seed=12)
    packed = ctx.pack(torch.from_numpy(rep.codes), torch.from_numpy(rep.lens), 16)
    sig = ctx.sign(packed, rep.n, 3, torch.from_numpy(a.view(np.int32)), torch.from_numpy(b.view(np.int32)), 16, 4)
    donor = torch.from_numpy(rep.donor).to(ctx.device)
    out = torch.empty((1 << 20, 2), dtype=torch.int32, device=ctx.device)
    cnt = torch.zeros((1,), dtype=torch.int64, device=ctx.device)
    ctx.band_candidates_async(sig, rep.n, 16, 4, 0, out, cnt, donor=donor)
    ctx.check()
    want = to_np(out[:int(cnt.item())]).view(np.uint32)
    got, _ = collect(ctx, sig, rep.n, 16, 4, 0, 5000, donor=donor)
    assert got.shape == want.shape and (got == want).all()


def test_stream_argument_checks(ctx, torch):
    from paper_2602_17330_gb300 import subquad
    import ctypes

    sig = torch.zeros((2, 100, 2), dtype=torch.int32, device=ctx.device)
    h = ctypes.c_void_p()
    total = ctypes.c_uint64(0)
    lib = subquad.lib()
    assert lib.subquad_band_stream_create(ctx.handle, ctypes.c_void_p(sig.data_ptr()), 100, 2, 2, 0, None,
                                          ctypes.byref(h), ctypes.byref(total)) == subquad.SUBQUAD_OK
    try:
        assert total.value == 2 * 100 * 99 // 2  # one bucket per band: raw pairs counted in both bands
        buf = torch.empty((64, 2), dtype=torch.int32, device=ctx.device)
        cnt, done = ctypes.c_int64(0), ctypes.c_int(0)
        st = lib.subquad_band_stream_next(ctx.handle, h, ctypes.c_void_p(buf.data_ptr()), 31, ctypes.byref(cnt),
                                          ctypes.byref(done))
        assert st == subquad.SUBQUAD_ERR_ARG
        seen = 0
        while not done.value:
            assert lib.subquad_band_stream_next(ctx.handle, h, ctypes.c_void_p(buf.data_ptr()), 64,
                                                ctypes.byref(cnt), ctypes.byref(done)) == subquad.SUBQUAD_OK
            seen += cnt.value
        assert seen == 100 * 99 // 2  # the second band's copies are owned by the first
    finally:
        lib.subquad_band_stream_destroy(h)
    lib.subquad_band_stream_destroy(None)


def test_streamed_pipeline_matches_one_pass(ctx, torch, oracle_mod):
    """Zipf families (ragged buckets, no cap), lengths 6-30, 32 bands of 4:
    the streamed pipeline's batches, put together, carry the same pairs,
    scores and fused values as one unbatched pass."""
    from paper_2602_17330_gb300 import pipeline

    cfg = pipeline.Workload("zipf_small", 30_000, bands=32, rows=4, pack_stride=32)
    rep = synth.zipf_repertoire(cfg.n, seed=3, hi=400)
    a, b = synth.hash_coefficients(cfg.hashes, seed=3)
    emb = synth.unit_embeddings(rep.n, cfg.d, seed=3)
    params = synth.gate_parameters(cfg.hidden, seed=3)
    one = pipeline.Pipeline(ctx, cfg)
    x = one.upload(rep, a, b, emb, params)
    ref = one.forward(x)
    want_pairs = to_np(ref["pairs"]).view(np.uint32)
    want_sw, want_f = to_np(ref["sw"]), to_np(ref["fused"])
    sp = pipeline.StreamedPipeline(ctx, cfg, rep.n, batch_capacity=40_000)
    total = sp.prepare(x)
    assert total >= want_pairs.shape[0]
    got_p, got_s, got_f, nb = [], [], [], 0
    for pairs, sw, fused in sp.batches(x):
        got_p.append(to_np(pairs).view(np.uint32).copy())
        got_s.append(to_np(sw).copy())
        got_f.append(to_np(fused).copy())
        nb += 1
    sp.close()
    ctx.check()
    assert nb > 3
    gp, gs, gf = np.concatenate(got_p), np.concatenate(got_s), np.concatenate(got_f)
    key = gp[:, 0].astype(np.uint64) << np.uint64(32) | gp[:, 1].astype(np.uint64)
    order = np.argsort(key)
    assert (gp[order] == want_pairs).all()
    assert (gs[order] == want_sw).all()
    assert np.allclose(gf[order], want_f, rtol=1e-6, atol=1e-7)
    # the candidate set itself against the oracle
    want = oracle_mod.candidates(oracle_mod.sign(rep.codes, rep.lens, 3, a, b), 32, 4, 0)
    assert want.shape == want_pairs.shape and (want == want_pairs).all()
