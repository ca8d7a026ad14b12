"""GPU parity: the CUDA path through the C ABI against the oracle, element by
element, on seeded inputs.  Signatures, candidate sets and alignment scores
must be bit-exact; fused scores must satisfy |x - y| <= 1e-5 * max(|y|, 1e-3)
against the FP64 oracle."""
import numpy as np
import pytest

from paper_2602_17330_gb300 import synth

pytestmark = pytest.mark.gpu

FUSED_RTOL = 1e-5
FUSED_FLOOR = 1e-3


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


def gpu_sig(ctx, torch, rep, k, a, b, bands, rows, stride):
    packed = ctx.pack(torch.from_numpy(rep.codes), torch.from_numpy(rep.lens), stride)
    sig = ctx.sign(packed, rep.n, k, torch.from_numpy(a.view(np.int32)), torch.from_numpy(b.view(np.int32)),
                   bands, rows)
    return packed, sig


def oracle_sig_layout(sig_oracle, bands, rows):
    n = sig_oracle.shape[0]
    return sig_oracle.reshape(n, bands, rows).transpose(1, 0, 2)


def assert_fused_close(got, want):
    err = np.abs(got.astype(np.float64) - want)
    bound = FUSED_RTOL * np.maximum(np.abs(want), FUSED_FLOOR)
    assert (err <= bound).all(), f"max err {err.max():.3e}, worst ratio {(err / bound).max():.3f}"


# --------------------------------------------------------------------------
# (a1) signatures
# --------------------------------------------------------------------------

@pytest.mark.parametrize("stride", [16, 32])
def test_pack_staged_and_byte_paths_agree(ctx, torch, stride):
    """Code rows of 32 bytes take the shared-memory staged packer, rows of 33
    bytes the per-byte one; both must give the same records, and the records
    must decode to the input (5-bit codes, length in the top nibbles of words
    0 and 1).  n spans several grid strides and a ragged last block."""
    rng = np.random.default_rng(5 + stride)
    n = 311_373
    max_len = 24 if stride == 16 else 30
    lens = rng.integers(1, max_len + 1, n).astype(np.uint8)
    codes32 = rng.integers(0, 20, (n, 32)).astype(np.uint8)
    codes33 = np.zeros((n, 33), np.uint8)
    codes33[:, :32] = codes32
    a = to_np(ctx.pack(torch.from_numpy(codes32), torch.from_numpy(lens), stride))
    b = to_np(ctx.pack(torch.from_numpy(codes33), torch.from_numpy(lens), stride))
    assert (a == b).all()
    w = np.ascontiguousarray(a).view(np.uint64).reshape(n, stride // 8)
    L = (w[:, 0] >> np.uint64(60)) | ((w[:, 1] >> np.uint64(60)) << np.uint64(4))
    assert (L.astype(np.int64) == lens).all()
    for p in range(max_len):
        code = (w[:, p // 12] >> np.uint64(5 * (p % 12))) & np.uint64(31)
        mask = p < lens
        assert (code[mask].astype(np.int64) == codes32[mask, p]).all()


@pytest.mark.parametrize("k", [1, 2, 3, 4, 6])
def test_sign_bitexact_tiny(ctx, torch, oracle_mod, k):
    rep = synth.tiny_repertoire()
    a, b = synth.hash_coefficients(64, seed=k)
    _, sig = gpu_sig(ctx, torch, rep, k, a, b, 16, 4, 16)
    want = oracle_sig_layout(oracle_mod.sign(rep.codes, rep.lens, k, a, b), 16, 4)
    assert (to_np(sig).view(np.uint32) == want).all()
    ctx.check()


@pytest.mark.parametrize("bands,rows", [(32, 4), (16, 2), (8, 3), (5, 7), (64, 1)])
def test_sign_bitexact_long_sequences_stride32(ctx, torch, oracle_mod, bands, rows):
    rep = synth.zipf_repertoire(3000, seed=1, hi=200)
    assert rep.lens.max() > 24
    a, b = synth.hash_coefficients(bands * rows, seed=2)
    _, sig = gpu_sig(ctx, torch, rep, 3, a, b, bands, rows, 32)
    want = oracle_sig_layout(oracle_mod.sign(rep.codes, rep.lens, 3, a, b), bands, rows)
    assert (to_np(sig).view(np.uint32) == want).all()


def test_sign_extreme_coefficients(ctx, torch, oracle_mod):
    rep = synth.tiny_repertoire()
    P = (1 << 31) - 1
    a = np.array([P - 1, P - 2, 1, 2, (1 << 30) + 7, 123457, P - 1, 1], dtype=np.uint32)
    b = np.array([P - 1, 0, P - 1, 0, P - 2, 7, 0, 0], dtype=np.uint32)
    _, sig = gpu_sig(ctx, torch, rep, 6, a, b, 2, 4, 16)
    want = oracle_sig_layout(oracle_mod.sign(rep.codes, rep.lens, 6, a, b), 2, 4)
    assert (to_np(sig).view(np.uint32) == want).all()


def test_sequence_shorter_than_k_gets_empty_signature(ctx, torch):
    codes, lens = synth.encode(["CA", "CASF"])
    a, b = synth.hash_coefficients(8)
    _, sig = gpu_sig(ctx, torch, synth.Repertoire(codes, lens, np.zeros(2, np.int32), np.zeros(2, np.int32),
                                                  np.ones(20) / 20), 3, a, b, 2, 4, 16)
    s = to_np(sig).view(np.uint32)
    assert (s[:, 0, :] == 0xFFFFFFFF).all()
    assert (s[:, 1, :] != 0xFFFFFFFF).all()


def test_invalid_codes_are_reported(ctx, torch):
    from paper_2602_17330_gb300 import subquad

    codes, lens = synth.encode(["CASSF", "CASSF"])
    codes[1, 2] = 25
    ctx.pack(torch.from_numpy(codes), torch.from_numpy(lens), 16)
    with pytest.raises(subquad.SubquadError) as ei:
        ctx.check()
    assert ei.value.status == subquad.SUBQUAD_ERR_INPUT
    ctx.check()  # the sticky error was cleared
    bad_len = lens.copy()
    bad_len[0] = 25  # > 24 does not fit the 16-byte record
    ctx.pack(torch.from_numpy(codes[:1]), torch.from_numpy(bad_len[:1]), 16)
    with pytest.raises(subquad.SubquadError):
        ctx.check()


# --------------------------------------------------------------------------
# (a2) candidates
# --------------------------------------------------------------------------

def gpu_candidates_from_sig(ctx, torch, sig_np, bands, rows, cap):
    """sig_np: uint32 [n, H] in the oracle's layout."""
    n = sig_np.shape[0]
    lay = np.ascontiguousarray(oracle_sig_layout(sig_np, bands, rows)).view(np.int32)
    sig = torch.from_numpy(lay).to(ctx.device)
    return to_np(ctx.band_candidates(sig, n, bands, rows, cap)).view(np.uint32)


@pytest.mark.parametrize("cap", [0, 1, 2, 3, 7])
def test_candidates_bitexact_planted_buckets(ctx, torch, oracle_mod, cap):
    rng = np.random.default_rng(100 + cap)
    n, bands, rows = 3000, 5, 3
    sig = rng.integers(0, 4, (n, bands * rows)).astype(np.uint32)  # buckets of every size
    sig[:, 1::3] += np.uint32((1 << 31) - 10)
    got = gpu_candidates_from_sig(ctx, torch, sig, bands, rows, cap)
    want = oracle_mod.candidates(sig, bands, rows, cap)
    assert got.shape == want.shape and (got == want).all()


def test_candidates_bitexact_tiny(ctx, torch, oracle_mod):
    rep = synth.tiny_repertoire()
    a, b = synth.hash_coefficients(64)
    _, sig = gpu_sig(ctx, torch, rep, 3, a, b, 16, 4, 16)
    got = to_np(ctx.band_candidates(sig, rep.n, 16, 4, 0)).view(np.uint32)
    want = oracle_mod.candidates(oracle_mod.sign(rep.codes, rep.lens, 3, a, b), 16, 4, 0)
    assert got.shape == want.shape and (got == want).all()


@pytest.mark.parametrize("cap", [0, 2048, 4])
def test_candidates_bitexact_donor_20k(ctx, torch, oracle_mod, cap):
    rep = synth.donor_repertoire(20_000, seed=3)
    a, b = synth.hash_coefficients(64, seed=3)
    _, sig = gpu_sig(ctx, torch, rep, 3, a, b, 16, 4, 16)
    got = to_np(ctx.band_candidates(sig, rep.n, 16, 4, cap)).view(np.uint32)
    want = oracle_mod.candidates(oracle_mod.sign(rep.codes, rep.lens, 3, a, b), 16, 4, cap)
    assert got.shape == want.shape and (got == want).all()


def test_candidates_capacity_error_reports_required_count(ctx, torch, oracle_mod):
    from paper_2602_17330_gb300 import subquad
    import ctypes

    rep = synth.tiny_repertoire()
    a, b = synth.hash_coefficients(64)
    _, sig = gpu_sig(ctx, torch, rep, 3, a, b, 16, 4, 16)
    want = oracle_mod.candidates(oracle_mod.sign(rep.codes, rep.lens, 3, a, b), 16, 4, 0)
    out = torch.empty((5, 2), dtype=torch.int32, device=ctx.device)
    cnt = ctypes.c_int64(0)
    st = subquad.lib().subquad_band_candidates(ctx.handle, ctypes.c_void_p(sig.data_ptr()), rep.n, 16, 4, 0,
                                                ctypes.c_void_p(out.data_ptr()), 5, ctypes.byref(cnt))
    assert st == subquad.SUBQUAD_ERR_CAPACITY and cnt.value == want.shape[0]


def test_candidates_degenerate_inputs(ctx, torch):
    one = torch.zeros((4, 1, 4), dtype=torch.int32, device=ctx.device)
    assert ctx.band_candidates(one, 1, 4, 4, 0).shape[0] == 0
    same = torch.zeros((2, 50, 2), dtype=torch.int32, device=ctx.device)  # one bucket per band
    got = to_np(ctx.band_candidates(same, 50, 2, 2, 0))
    assert got.shape[0] == 50 * 49 // 2
    got = to_np(ctx.band_candidates(same, 50, 2, 2, 10))
    assert got.shape[0] == 5 * 45


@pytest.mark.parametrize("cap", [0, 4])
def test_candidates_split_partitions(ctx, torch, oracle_mod, cap):
    """A partition target of 2^16 keys puts all 20k keys of a band in one
    partition, more distinct keys than one shared-memory table holds: the
    partition is split into fingerprint sub-ranges; the result is unchanged."""
    from paper_2602_17330_gb300 import subquad

    rep = synth.donor_repertoire(20_000, seed=4)
    a, b = synth.hash_coefficients(64, seed=4)
    _, sig = gpu_sig(ctx, torch, rep, 3, a, b, 16, 4, 16)
    want = oracle_mod.candidates(oracle_mod.sign(rep.codes, rep.lens, 3, a, b), 16, 4, cap)
    old = ctx.get_tuning(subquad.TUNE_BAND_PART_LOG2)
    try:
        for part_log2 in (16, 6):
            ctx.set_tuning(subquad.TUNE_BAND_PART_LOG2, part_log2)
            got = to_np(ctx.band_candidates(sig, rep.n, 16, 4, cap)).view(np.uint32)
            assert got.shape == want.shape and (got == want).all()
    finally:
        ctx.set_tuning(subquad.TUNE_BAND_PART_LOG2, old)


def test_candidates_most_partitions(ctx, torch, oracle_mod):
    """A partition target of 2^6 keys over 70,000 sequences asks for more than
    the 1,024 partitions per band the partition pass allows: every band is
    split into 1,024 partitions of about 68 keys (four digits per thread in
    the scatter's scan, digits up to 1,023 in its staged words) over 18
    tiles, the last one ragged."""
    from paper_2602_17330_gb300 import subquad

    rep = synth.donor_repertoire(70_000, seed=6)
    a, b = synth.hash_coefficients(64, seed=6)
    _, sig = gpu_sig(ctx, torch, rep, 3, a, b, 16, 4, 16)
    want = oracle_mod.candidates(oracle_mod.sign(rep.codes, rep.lens, 3, a, b), 16, 4, 0)
    old = ctx.get_tuning(subquad.TUNE_BAND_PART_LOG2)
    try:
        ctx.set_tuning(subquad.TUNE_BAND_PART_LOG2, 6)
        got = to_np(ctx.band_candidates(sig, rep.n, 16, 4, 0)).view(np.uint32)
        assert got.shape == want.shape and (got == want).all()
    finally:
        ctx.set_tuning(subquad.TUNE_BAND_PART_LOG2, old)


FP_MUL = 0x9E3779B1  # the library's fingerprint multiplier


def _premix(w):
    return (w ^ (w >> 16)) & 0xFFFFFFFF  # its own inverse


def test_candidates_fingerprint_clash(ctx, torch, oracle_mod):
    """White-box: distinct 2-row keys built to share the library's 32-bit key
    fingerprint (words pre-mixed by w ^ w >> 16, summed by Horner with an odd
    multiplier mod 2^32, then mixed) must stay in separate buckets.  With at
    most 1024 keys per band (the default partition target) every band is a
    single partition, so the equal fingerprints meet in one table."""
    rng = np.random.default_rng(77)
    n, bands, rows = 1000, 2, 2
    sig = rng.integers(0, 40, (n, bands * rows)).astype(np.uint32)
    groups = []
    for g in range(6):
        k0, k1 = 1000 + 2 * g, 5000 + g
        k0b = 1001 + 2 * g
        # (s + p(k0)) M + p(k1) == (s + p(k0b)) M + p(k1b)  (mod 2^32)
        k1b = _premix((_premix(k1) + (_premix(k0) - _premix(k0b)) * FP_MUL) & 0xFFFFFFFF)
        assert (k0b, k1b) != (k0, k1)
        groups.append(((k0, k1), (k0b, k1b)))
    ids = rng.permutation(n)[:6 * 9]
    for g, ((a0, a1), (b0, b1)) in enumerate(groups):
        for t, i in enumerate(ids[9 * g:9 * g + 9]):
            sig[i, 0:2] = (a0, a1) if t < 5 else (b0, b1)
    for cap in (0, 3):
        got = gpu_candidates_from_sig(ctx, torch, sig, bands, rows, cap)
        want = oracle_mod.candidates(sig, bands, rows, cap)
        assert got.shape == want.shape and (got == want).all()


@pytest.mark.parametrize("cap", [0, 3])
def test_candidates_every_key_twice(ctx, torch, oracle_mod, cap):
    """Every key occurs exactly twice (every key is kept); with a partition
    target of 2^16 keys a band is one partition with 10,000 distinct keys,
    more than one shared-memory table holds: the exact path splits it into
    fingerprint sub-ranges."""
    from paper_2602_17330_gb300 import subquad

    rng = np.random.default_rng(21)
    n, bands, rows = 20_000, 3, 4
    half = rng.integers(0, 1 << 31, (n // 2, bands * rows)).astype(np.uint32)
    sig = np.concatenate([half, half])[rng.permutation(n)]
    want = oracle_mod.candidates(sig, bands, rows, cap)
    old = ctx.get_tuning(subquad.TUNE_BAND_PART_LOG2)
    try:
        for part_log2 in (16, 10, 6):
            ctx.set_tuning(subquad.TUNE_BAND_PART_LOG2, part_log2)
            got = gpu_candidates_from_sig(ctx, torch, sig, bands, rows, cap)
            assert got.shape == want.shape and (got == want).all()
    finally:
        ctx.set_tuning(subquad.TUNE_BAND_PART_LOG2, old)


def test_candidates_row_longer_than_shared_memory(ctx, torch, oracle_mod):
    """Sequence 0 shares a chunk with 19 different sequences in each of 512
    one-row bands: its row has 9,728 partners, more than one CTA sorts in
    shared memory, so the row is sorted in place in global memory."""
    rng = np.random.default_rng(33)
    bands, rows, per = 512, 1, 19
    n = 1 + bands * per
    sig = rng.integers(0, 1 << 31, (n, bands)).astype(np.uint32)
    for b in range(bands):
        sig[1 + per * b: 1 + per * (b + 1), b] = sig[0, b]
    got = gpu_candidates_from_sig(ctx, torch, sig, bands, rows, per + 1)
    want = oracle_mod.candidates(sig, bands, rows, per + 1)
    assert (want[:, 0] == 0).sum() == bands * per
    assert got.shape == want.shape and (got == want).all()


def test_candidates_rows_of_every_size_to_2049(ctx, torch, oracle_mod):
    """One bucket of 2,050 members among 4,000 sequences: its members' rows
    hold 1, 2, ..., 2,049 partners, so the register, warp and CTA row sorts
    all run and both sides of each of their size boundaries (4/5, 8/9,
    16/17, 32/33 and 512/513 partners) occur; the second band adds pairs
    that the first band already owns."""
    rng = np.random.default_rng(2049)
    n, bands, rows = 4_000, 2, 3
    sig = rng.integers(0, 1 << 31, (n, bands * rows)).astype(np.uint32)
    ids = rng.permutation(n)[:2_050]
    sig[ids, 0:rows] = rng.integers(0, 1 << 31, rows)
    sig[ids[:700], rows:] = rng.integers(0, 1 << 31, rows)
    got = gpu_candidates_from_sig(ctx, torch, sig, bands, rows, 0)
    want = oracle_mod.candidates(sig, bands, rows, 0)
    deg = np.bincount(want[:, 0].astype(np.int64), minlength=n)
    assert set(range(1, 2_050)) <= set(deg.tolist())
    assert got.shape == want.shape and (got == want).all()


@pytest.mark.parametrize("n,nbig,size,cap", [(3_000, 3, 300, 64), (20_000, 40, 500, 64), (20_000, 40, 500, 499)])
def test_candidates_several_buckets_above_cap(ctx, torch, oracle_mod, n, nbig, size, cap):
    """Several buckets above the cap in one partition: with 900 repeated keys
    among 3,000 (one partition) the shared-memory fast path sorts three
    buckets one after another; with 40 buckets of 500 among 20,000 (16
    partitions of ~1,250 records, too many repeats for the fast path) the
    exact path does.  Chunks must hold ranks [m cap, (m+1) cap) in id order."""
    rng = np.random.default_rng(n + nbig + cap)
    bands, rows = 3, 2
    sig = rng.integers(0, 1 << 31, (n, bands * rows)).astype(np.uint32)  # singletons
    for b in range(bands):
        ids = rng.permutation(n)[:nbig * size]
        for g in range(nbig):
            sig[ids[g * size:(g + 1) * size], b * rows:(b + 1) * rows] = rng.integers(0, 1 << 31, rows)
    got = gpu_candidates_from_sig(ctx, torch, sig, bands, rows, cap)
    want = oracle_mod.candidates(sig, bands, rows, cap)
    assert got.shape == want.shape and (got == want).all()


@pytest.mark.parametrize("n,cap", [(20_000, 64), (20_000, 1), (3_000, 1_200), (2_500, 0)])
def test_candidates_one_giant_bucket(ctx, torch, oracle_mod, n, cap):
    """Every sequence has the same key in every band: one bucket of n members
    per band, chunked by rank in id order when it exceeds the cap."""
    rng = np.random.default_rng(n + cap)
    sig = np.repeat(rng.integers(0, 1 << 31, (1, 2 * 2)).astype(np.uint32), n, axis=0)
    got = gpu_candidates_from_sig(ctx, torch, sig, 2, 2, cap)
    want = oracle_mod.candidates(sig, 2, 2, cap)
    assert got.shape == want.shape and (got == want).all()


# --------------------------------------------------------------------------
# (a3) alignment
# --------------------------------------------------------------------------

@pytest.mark.parametrize("binned", [False, True])
def test_align_all_pairs_tiny_bitexact(ctx, torch, oracle_mod, binned):
    rep = synth.tiny_repertoire()
    packed = ctx.pack(torch.from_numpy(rep.codes), torch.from_numpy(rep.lens), 16)
    iu, ju = np.triu_indices(rep.n, 1)
    pairs = np.stack([iu, ju], 1).astype(np.uint32)
    got = to_np(ctx.align_score(packed, torch.from_numpy(pairs.view(np.int32)).to(ctx.device), binned=binned))
    want = oracle_mod.sw_pairs(rep.codes, rep.lens, pairs)
    assert (got == want).all()
    self_got = to_np(ctx.self_scores(packed, binned=binned))
    assert (self_got == oracle_mod.self_scores(rep.codes, rep.lens)).all()


@pytest.mark.parametrize("binned", [False, True])
@pytest.mark.parametrize("m", [1, 31, 33, 1000, 4097])
def test_align_ragged_counts_stride32(ctx, torch, oracle_mod, m, binned):
    rep = synth.zipf_repertoire(4000, seed=5, hi=100)
    packed = ctx.pack(torch.from_numpy(rep.codes), torch.from_numpy(rep.lens), 32)
    rng = np.random.default_rng(m)
    pairs = rng.integers(0, rep.n, (m, 2)).astype(np.uint32)
    pairs[0] = [int(np.argmax(rep.lens)), int(np.argmin(rep.lens))]
    got = to_np(ctx.align_score(packed, torch.from_numpy(pairs.view(np.int32)).to(ctx.device), binned=binned))
    assert (got == oracle_mod.sw_pairs(rep.codes, rep.lens, pairs)).all()
    assert (to_np(ctx.self_scores(packed, binned=binned)) == oracle_mod.self_scores(rep.codes, rep.lens)).all()


@pytest.mark.parametrize("binned", [False, True])
@pytest.mark.parametrize("o,e", [(10, 1), (0, 0), (3, 3), (11, 1), (1000, 1000), (5, 2)])
def test_align_gap_parameters(ctx, torch, oracle_mod, o, e, binned):
    rep = synth.tiny_repertoire(seed=2)
    packed = ctx.pack(torch.from_numpy(rep.codes), torch.from_numpy(rep.lens), 16)
    rng = np.random.default_rng(o * 7 + e)
    pairs = rng.integers(0, rep.n, (3000, 2)).astype(np.uint32)
    got = to_np(ctx.align_score(packed, torch.from_numpy(pairs.view(np.int32)).to(ctx.device), o, e, binned=binned))
    assert (got == oracle_mod.sw_pairs(rep.codes, rep.lens, pairs, o, e)).all()


def test_align_custom_matrices(ctx, torch, oracle_mod):
    rep = synth.tiny_repertoire(seed=4)
    packed = ctx.pack(torch.from_numpy(rep.codes), torch.from_numpy(rep.lens), 16)
    rng = np.random.default_rng(9)
    pairs = rng.integers(0, rep.n, (2000, 2)).astype(np.uint32)
    tp = torch.from_numpy(pairs.view(np.int32)).to(ctx.device)
    try:
        ident = np.full((20, 20), -64, dtype=np.int32)
        np.fill_diagonal(ident, 1)
        ctx.set_matrix(ident.ravel())
        got = to_np(ctx.align_score(packed, tp, 1000, 1000))
        assert (got == oracle_mod.sw_pairs(rep.codes, rep.lens, pairs, 1000, 1000, ident)).all()
        asym = rng.integers(-6, 9, (20, 20)).astype(np.int32)  # not symmetric: no operand swap allowed
        ctx.set_matrix(asym.ravel())
        want = oracle_mod.sw_pairs(rep.codes, rep.lens, pairs, 4, 1, asym)
        assert (to_np(ctx.align_score(packed, tp, 4, 1)) == want).all()
        assert (to_np(ctx.align_score(packed, tp, 4, 1, binned=True)) == want).all()
    finally:
        ctx.set_matrix(None)
    got = to_np(ctx.align_score(packed, tp))
    assert (got == oracle_mod.sw_pairs(rep.codes, rep.lens, pairs)).all()


@pytest.mark.parametrize("binned", [False, True])
def test_self_scores_both_paths(ctx, torch, oracle_mod, binned):
    """Self-scores through the diagonal-sum path (BLOSUM62, a diagonally
    dominant custom matrix) and the dynamic programme (a matrix that is not)."""
    rep = synth.zipf_repertoire(3000, seed=8, hi=100)
    packed = ctx.pack(torch.from_numpy(rep.codes), torch.from_numpy(rep.lens), 32)
    rng = np.random.default_rng(3)
    dom = rng.integers(-5, 3, (20, 20)).astype(np.int32)
    np.fill_diagonal(dom, rng.integers(3, 12, 20))
    bad = dom.copy()
    bad[0, 1] = bad[1, 0] = 30
    try:
        for M in (None, dom, bad):
            ctx.set_matrix(None if M is None else M.ravel())
            for o, e in ((10, 1), (0, 0)):
                got = to_np(ctx.self_scores(packed, o, e, binned=binned))
                assert (got == oracle_mod.self_scores(rep.codes, rep.lens, o, e, M)).all()
    finally:
        ctx.set_matrix(None)


@pytest.mark.parametrize("shape", [0, 1, 2])
@pytest.mark.parametrize("stride,maker", [(16, "donor"), (32, "zipf")])
def test_align_binned_launch_shapes(ctx, torch, oracle_mod, shape, stride, maker):
    from paper_2602_17330_gb300 import subquad

    rep = synth.donor_repertoire(6000, seed=11) if maker == "donor" else synth.zipf_repertoire(6000, seed=11, hi=300)
    packed = ctx.pack(torch.from_numpy(rep.codes), torch.from_numpy(rep.lens), stride)
    rng = np.random.default_rng(shape + stride)
    pairs = rng.integers(0, rep.n, (20_011, 2)).astype(np.uint32)
    tp = torch.from_numpy(pairs.view(np.int32)).to(ctx.device)
    old = ctx.get_tuning(subquad.TUNE_ALIGN_SHAPE)
    try:
        ctx.set_tuning(subquad.TUNE_ALIGN_SHAPE, shape)
        got = to_np(ctx.align_score(packed, tp, binned=True))
        self_got = to_np(ctx.self_scores(packed, binned=True))
    finally:
        ctx.set_tuning(subquad.TUNE_ALIGN_SHAPE, old)
    assert (got == oracle_mod.sw_pairs(rep.codes, rep.lens, pairs)).all()
    assert (self_got == oracle_mod.self_scores(rep.codes, rep.lens)).all()


@pytest.mark.parametrize("o,e", [(0, 0), (1000, 1000), (11, 1), (3, 2)])
def test_align_split_shape_gaps_and_matrix(ctx, torch, oracle_mod, o, e):
    """The split-table launch shape with extreme gap costs and an asymmetric
    matrix spanning the allowed score range (negative staged values)."""
    from paper_2602_17330_gb300 import subquad

    rep = synth.zipf_repertoire(4000, seed=o + e, hi=200)
    packed = ctx.pack(torch.from_numpy(rep.codes), torch.from_numpy(rep.lens), 32)
    rng = np.random.default_rng(o + 7 * e)
    pairs = rng.integers(0, rep.n, (9_999, 2)).astype(np.uint32)
    tp = torch.from_numpy(pairs.view(np.int32)).to(ctx.device)
    M = rng.integers(-64, 64, (20, 20)).astype(np.int32)
    old = ctx.get_tuning(subquad.TUNE_ALIGN_SHAPE)
    try:
        ctx.set_tuning(subquad.TUNE_ALIGN_SHAPE, 2)
        ctx.set_matrix(M.reshape(-1).tolist())
        got = to_np(ctx.align_score(packed, tp, o, e, binned=True))
    finally:
        ctx.set_matrix(None)
        ctx.set_tuning(subquad.TUNE_ALIGN_SHAPE, old)
    assert (got == oracle_mod.sw_pairs(rep.codes, rep.lens, pairs, o, e, M)).all()


def test_autotune_picks_a_candidate_and_keeps_results(ctx, torch, oracle_mod):
    from paper_2602_17330_gb300 import autotune, subquad

    rep = synth.donor_repertoire(20_000, seed=12)
    a, b = synth.hash_coefficients(64, seed=12)
    packed, sig = gpu_sig(ctx, torch, rep, 3, a, b, 16, 4, 16)
    pairs = ctx.band_candidates(sig, rep.n, 16, 4, 2048)
    res = autotune.autotune(ctx, packed, pairs, sig=sig, n=rep.n, bands=16, rows=4, bucket_cap=2048, reps=2,
                            use_cache=False)
    assert int(res["choice"][str(subquad.TUNE_ALIGN_SHAPE)]) in (0, 1)
    assert int(res["choice"][str(subquad.TUNE_BAND_PART_LOG2)]) in autotune.CANDIDATES[subquad.TUNE_BAND_PART_LOG2]
    pairs2 = to_np(ctx.band_candidates(sig, rep.n, 16, 4, 2048)).view(np.uint32)
    want = oracle_mod.candidates(oracle_mod.sign(rep.codes, rep.lens, 3, a, b), 16, 4, 2048)
    assert (pairs2 == want).all()
    sw = to_np(ctx.align_score(packed, pairs, binned=True))
    assert (sw == oracle_mod.sw_pairs(rep.codes, rep.lens, want)).all()


def test_align_empty(ctx, torch):
    rep = synth.tiny_repertoire()
    packed = ctx.pack(torch.from_numpy(rep.codes), torch.from_numpy(rep.lens), 16)
    pairs = torch.zeros((0, 2), dtype=torch.int32, device=ctx.device)
    assert ctx.align_score(packed, pairs).shape[0] == 0


# --------------------------------------------------------------------------
# (a4) fusion
# --------------------------------------------------------------------------

def _row_heavy_pairs(rng, n, count):
    """Sorted pairs whose first members have long runs of partners (as in a
    candidate list with large buckets), plus short rows and singletons."""
    heads = rng.choice(n - 1, 40, replace=False)
    parts = []
    for h in heads:
        deg = int(rng.integers(1, 400))
        parts.append(np.stack([np.full(deg, h), rng.integers(h + 1, n, deg)], axis=1))
    parts.append(np.sort(rng.integers(0, n, (count, 2)), axis=1))
    pairs = np.unique(np.concatenate(parts), axis=0)
    return pairs[pairs[:, 0] < pairs[:, 1]].astype(np.uint32)


@pytest.mark.parametrize("lanes", [4, 8])
@pytest.mark.parametrize("d,hidden,scale", [(64, 16, False), (128, 32, True), (4, 1, True), (36, 64, False),
                                            (256, 17, True), (260, 16, False)])
def test_fuse_forward_within_tolerance(ctx, torch, oracle_mod, d, hidden, scale, lanes):
    from paper_2602_17330_gb300 import subquad

    rep = synth.tiny_repertoire()
    packed = ctx.pack(torch.from_numpy(rep.codes), torch.from_numpy(rep.lens), 16)
    rng = np.random.default_rng(d)
    pairs = _row_heavy_pairs(rng, rep.n, 20_001)
    emb = synth.family_embeddings(rep.family, d, seed=d)
    if scale:
        emb = np.ascontiguousarray(emb * rng.uniform(0.2, 5.0, (rep.n, 1)).astype(np.float32))
    params = synth.gate_parameters(hidden, seed=hidden)
    tp = torch.from_numpy(pairs.view(np.int32)).to(ctx.device)
    # both sides take the oracle's alignment scores (inputs of this step)
    sw_o = oracle_mod.sw_pairs(rep.codes, rep.lens, pairs)
    self_o = oracle_mod.self_scores(rep.codes, rep.lens)
    sw = torch.from_numpy(sw_o).to(ctx.device)
    self_sc = torch.from_numpy(self_o).to(ctx.device)
    old = ctx.get_tuning(subquad.TUNE_FUSE_LANES)
    try:
        ctx.set_tuning(subquad.TUNE_FUSE_LANES, lanes)
        fused, alpha = ctx.fuse_forward(tp, sw, self_sc, packed, torch.from_numpy(emb), torch.from_numpy(params),
                                        hidden, want_alpha=True)
        # a ragged tail and an empty list through the same launch shape
        tail = pairs.shape[0] - 13
        fused_t = ctx.fuse_forward(tp[:tail], sw[:tail], self_sc, packed, torch.from_numpy(emb),
                                   torch.from_numpy(params), hidden)
        empty = ctx.fuse_forward(tp[:0], sw[:0], self_sc, packed, torch.from_numpy(emb), torch.from_numpy(params),
                                 hidden)
    finally:
        ctx.set_tuning(subquad.TUNE_FUSE_LANES, old)
    want = oracle_mod.fuse_forward(pairs, sw_o, self_o, rep.lens, emb, params, hidden)
    assert to_np(empty).shape[0] == 0
    assert (to_np(fused_t) == to_np(fused)[:tail]).all()  # a pair's result does not depend on its neighbours
    assert_fused_close(to_np(fused), want["fused"])
    assert_fused_close(to_np(alpha), want["alpha"])


# --------------------------------------------------------------------------
# full-size workload: one donor of 1,000,000 sequences, as the benchmark runs it
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def donor_1m(ctx, torch, oracle_mod):
    from paper_2602_17330_gb300 import pipeline

    rep = synth.donor_repertoire(1_000_000, seed=0)
    cfg = pipeline.DONOR_1M
    a, b = synth.hash_coefficients(cfg.hashes, seed=0)
    emb = synth.unit_embeddings(rep.n, cfg.d, seed=0)
    params = synth.gate_parameters(cfg.hidden, seed=0)
    run = pipeline.Pipeline(ctx, cfg)
    out = run.forward_numpy(rep, a, b, emb, params)
    threads = oracle_mod.host_threads()
    sig_o = oracle_mod.sign_mt(rep.codes, rep.lens, 3, a, b, threads)
    pairs_o = oracle_mod.candidates(sig_o, cfg.bands, cfg.rows, cfg.bucket_cap)
    return dict(rep=rep, a=a, b=b, emb=emb, params=params, out=out, cfg=cfg, sig_o=sig_o, pairs_o=pairs_o)


def test_full_size_signatures_sampled(donor_1m, oracle_mod):
    d = donor_1m
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(d["rep"].n, 20_000, replace=False))
    want = oracle_mod.sign(d["rep"].codes[idx], d["rep"].lens[idx], 3, d["a"], d["b"])
    got = d["out"]["sig"][:, idx, :].transpose(1, 0, 2).reshape(len(idx), -1)
    assert (got == want).all()


def test_full_size_candidates_exact(donor_1m, oracle_mod):
    d = donor_1m
    want = d["pairs_o"]
    got = d["out"]["pairs"]
    assert got.shape == want.shape and (got == want).all()


def test_full_size_scores_and_fusion_sampled(donor_1m, oracle_mod):
    d = donor_1m
    rep, out = d["rep"], d["out"]
    rng = np.random.default_rng(1)
    # the GPU's pair list equals the oracle's (test_full_size_candidates_exact);
    # the sample and every oracle input below come from the oracle side
    assert (out["pairs"] == d["pairs_o"]).all()
    sel = np.sort(rng.choice(d["pairs_o"].shape[0], 30_000, replace=False))
    pairs = d["pairs_o"][sel]
    sw_o = oracle_mod.sw_pairs(rep.codes, rep.lens, pairs)
    assert (out["sw"][sel] == sw_o).all()
    assert (out["sw_plain"][sel] == out["sw"][sel]).all()
    self_o = oracle_mod.self_scores(rep.codes, rep.lens)
    assert (out["self"] == self_o).all()
    want = oracle_mod.fuse_forward(pairs, sw_o, self_o, rep.lens, d["emb"], d["params"], d["cfg"].hidden)
    assert_fused_close(out["fused"][sel], want["fused"])
