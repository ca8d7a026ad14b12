"""GPU parity of the edit-distance kernel (the GPU appendix's recurrence, a
second alignment mode on the length-binned scheduler) against the oracle:
bit-exact integer distances."""
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


def run(ctx, torch, rep, pairs, stride):
    packed = ctx.pack(torch.from_numpy(rep.codes), torch.from_numpy(rep.lens), stride)
    p = torch.from_numpy(np.ascontiguousarray(pairs, dtype=np.uint32).view(np.int32)).to(ctx.device)
    out = to_np(ctx.edit_distance(packed, p))
    ctx.check()
    return out


def test_edit_all_pairs_tiny_bitexact(ctx, torch, oracle_mod):
    rep = synth.tiny_repertoire()
    iu, ju = np.triu_indices(rep.n, 1)
    pairs = np.stack([iu, ju], 1).astype(np.uint32)
    ctx.set_edit_costs()
    got = run(ctx, torch, rep, pairs, 16)
    assert (got == oracle_mod.edit_pairs(rep.codes, rep.lens, pairs)).all()


@pytest.mark.parametrize("shape", [0, 1, 2])
@pytest.mark.parametrize("m", [1, 31, 33, 64, 65, 1000, 4097])
@pytest.mark.parametrize("stride", [16, 32])
def test_edit_ragged_counts_and_lengths(ctx, torch, oracle_mod, m, stride, shape):
    """Random pairs of lengths 1..max (a thread's two pairs differ in both
    lengths, so the transparent padding is exercised), both record sizes."""
    rng = np.random.default_rng(m + stride)
    n = 3000
    max_len = 24 if stride == 16 else 30
    lens = rng.integers(1, max_len + 1, n).astype(np.uint8)
    codes = np.full((n, 32), synth.PAD, np.uint8)
    for r in range(n):
        codes[r, : lens[r]] = rng.integers(0, 20, lens[r])
    rep = synth.Repertoire(codes, lens, np.full(n, -1, np.int32), np.zeros(n, np.int32), np.ones(20) / 20)
    pairs = rng.integers(0, n, (m, 2)).astype(np.uint32)
    from paper_2602_17330_gb300 import subquad

    ctx.set_edit_costs()
    old = ctx.get_tuning(subquad.TUNE_ALIGN_SHAPE)
    try:
        ctx.set_tuning(subquad.TUNE_ALIGN_SHAPE, shape)
        got = run(ctx, torch, rep, pairs, stride)
    finally:
        ctx.set_tuning(subquad.TUNE_ALIGN_SHAPE, old)
    assert (got == oracle_mod.edit_pairs(codes, lens, pairs)).all()


@pytest.mark.parametrize("indel,kind", [(1, "unit"), (0, "default"), (7, "random"), (255, "random"), (3, "heavy")])
def test_edit_costs(ctx, torch, oracle_mod, indel, kind):
    rng = np.random.default_rng(indel)
    if kind == "unit":
        sub = (np.ones((20, 20)) - np.eye(20)).astype(np.uint8)
    elif kind == "default":
        sub = oracle_mod.default_edit_costs()
    elif kind == "heavy":
        sub = np.full((20, 20), 255, np.uint8)
        np.fill_diagonal(sub, 0)
    else:
        sub = rng.integers(0, 256, (20, 20)).astype(np.uint8)
        sub = np.minimum(sub, sub.T)
        np.fill_diagonal(sub, 0)
    rep = synth.zipf_repertoire(4000, seed=indel, hi=100)
    pairs = rng.integers(0, rep.n, (5000, 2)).astype(np.uint32)
    ctx.set_edit_costs(indel, sub.reshape(-1).tolist())
    try:
        got = run(ctx, torch, rep, pairs, 32)
    finally:
        ctx.set_edit_costs()
    assert (got == oracle_mod.edit_pairs(rep.codes, rep.lens, pairs, indel, sub)).all()


def test_edit_rejects_asymmetric_costs(ctx):
    from paper_2602_17330_gb300 import subquad

    sub = (np.ones((20, 20)) - np.eye(20)).astype(np.uint8)
    sub[0, 1] = 3
    with pytest.raises(subquad.SubquadError):
        ctx.set_edit_costs(1, sub.reshape(-1).tolist())
    diag = np.zeros((20, 20), np.uint8)
    diag[2, 2] = 1
    with pytest.raises(subquad.SubquadError):
        ctx.set_edit_costs(1, diag.reshape(-1).tolist())
    with pytest.raises(subquad.SubquadError):
        ctx.set_edit_costs(256)


def test_edit_async_matches_sync_and_full_size_sample(ctx, torch, oracle_mod):
    """The 1M-sequence donor's candidate pairs (the benchmark workload): the
    device-count form equals the synchronous one, and a seeded sample of
    20,000 pairs equals the oracle."""
    rep = synth.donor_repertoire(1_000_000, seed=0)
    a, b = synth.hash_coefficients(64, seed=0)
    packed = ctx.pack(torch.from_numpy(rep.codes), torch.from_numpy(rep.lens), 16)
    sig = ctx.sign(packed, rep.n, 3, torch.from_numpy(a.view(np.int32)), torch.from_numpy(b.view(np.int32)), 16, 4)
    pairs = ctx.band_candidates(sig, rep.n, 16, 4, 2048)
    ctx.set_edit_costs()
    d1 = ctx.edit_distance(packed, pairs)
    d_m = torch.tensor([pairs.shape[0]], dtype=torch.int64, device=ctx.device)
    big = torch.zeros((pairs.shape[0] + 1000, 2), dtype=torch.int32, device=ctx.device)
    big[: pairs.shape[0]] = pairs
    d2 = torch.full((pairs.shape[0] + 1000,), -7, dtype=torch.int32, device=ctx.device)
    ctx.edit_distance_async(packed, big, d_m, d2)
    ctx.check()
    assert torch.equal(d1, d2[: pairs.shape[0]]) and bool((d2[pairs.shape[0]:] == -7).all())
    P = to_np(pairs).view(np.uint32)
    idx = np.random.default_rng(0).choice(P.shape[0], 20_000, replace=False)
    assert (to_np(d1)[idx] == oracle_mod.edit_pairs(rep.codes, rep.lens, P[idx])).all()
