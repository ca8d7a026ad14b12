"""The streamed candidate form on a Zipf donor with a bucket of 50,000 members
(200,000 sequences, Zipf(1.2) families up to 50,000, lengths 6-30, and one
planted block of 50,000 identical sequences so every band has a bucket of at
least 50,000): 4 bands of 2 rows, no cap, about 1.3e9 candidate pairs.

Checked against the oracle's signatures (not its pair list, which would not
fit): every pair of a seeded sample of batches shares its key in at least one
band; the batches hold no pair twice (all batches' pairs deduplicated on the
GPU); and their total equals |C| counted independently by inclusion-exclusion
over the bands: |C| = sum over non-empty band sets S of (-1)^(|S|+1) sum over
the buckets of S's combined key of C(size, 2)."""
import itertools

import numpy as np
import pytest

from paper_2602_17330_gb300 import synth

pytestmark = pytest.mark.gpu

BANDS, ROWS, BIG = 4, 2, 50_000


def test_stream_giant_bucket_partitions_candidates(oracle_mod):
    import torch

    from paper_2602_17330_gb300 import _build, subquad

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    _build.build()
    rep = synth.zipf_repertoire(200_000, seed=0, hi=50_000)
    rng = np.random.default_rng(0)
    block = np.sort(rng.choice(rep.n, BIG, replace=False))
    rep.codes[block] = rep.codes[block[0]]
    rep.lens[block] = rep.lens[block[0]]
    a, b = synth.hash_coefficients(BANDS * ROWS, seed=0)
    sig = oracle_mod.sign_mt(rep.codes, rep.lens, 3, a, b, oracle_mod.host_threads())

    # |C| by inclusion-exclusion over the bands (no cap)
    def pairs_sharing(bands):
        keys = np.concatenate([sig[:, b * ROWS:(b + 1) * ROWS] for b in bands], axis=1)
        _, cnt = np.unique(keys, axis=0, return_counts=True)
        return int((cnt.astype(np.int64) * (cnt - 1) // 2).sum()), int(cnt.max())

    want_total, biggest = 0, 0
    for r in range(1, BANDS + 1):
        for S in itertools.combinations(range(BANDS), r):
            c, mx = pairs_sharing(S)
            want_total += (-1) ** (r + 1) * c
            if r == 1:
                biggest = max(biggest, mx)
    assert biggest >= BIG

    with subquad.Context(0) as ctx:
        packed = ctx.pack(torch.from_numpy(rep.codes), torch.from_numpy(rep.lens), 32)
        sig_t = ctx.sign(packed, rep.n, 3, torch.from_numpy(a.view(np.int32)), torch.from_numpy(b.view(np.int32)),
                         BANDS, ROWS)
        assert (sig_t.cpu().numpy().view(np.uint32).transpose(1, 0, 2).reshape(rep.n, -1) == sig).all()
        keys = torch.empty((want_total + 1,), dtype=torch.int64, device=ctx.device)
        total, k, checked = 0, 0, 0
        sample = set(np.random.default_rng(1).choice(150, 12, replace=False).tolist())
        for bt in ctx.band_stream(sig_t, rep.n, BANDS, ROWS, 0, capacity=8_000_000):
            m = int(bt.shape[0])
            assert total + m <= want_total, "more pairs than |C|"
            p64 = bt.to(torch.int64)
            assert bool((p64[:, 0] < p64[:, 1]).all())
            keys[total:total + m] = (p64[:, 0] << 32) | p64[:, 1]
            if k in sample:
                P = bt.cpu().numpy().view(np.uint32)
                share = np.zeros(m, dtype=bool)
                for band in range(BANDS):
                    s0 = sig[P[:, 0], band * ROWS:(band + 1) * ROWS]
                    s1 = sig[P[:, 1], band * ROWS:(band + 1) * ROWS]
                    share |= (s0 == s1).all(axis=1)
                assert share.all(), f"batch {k}: a pair shares no band key"
                checked += m
            total += m
            k += 1
        ctx.check()
        assert total == want_total, (total, want_total)
        assert checked > 0
        distinct = int(torch.unique(keys[:total]).shape[0])
        assert distinct == total, "a pair appears in two batches"
