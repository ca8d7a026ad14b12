"""Output bounds through the C ABI: every output buffer is followed by canary
words, and no entry point may write past the end it was given -- including a
band call whose candidate set does not fit its capacity (the overflow is
reported, nothing is written beyond the buffer)."""
import ctypes

import numpy as np
import pytest

from paper_2602_17330_gb300 import synth

pytestmark = pytest.mark.gpu

CANARY = 0x5AA55AA5
TAIL = 256  # int32 words after every output


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


def guarded(torch, words):
    """(buffer of words + TAIL int32, view of the first words) filled with the canary."""
    buf = torch.full((words + TAIL,), CANARY, dtype=torch.int32, device="cuda")
    return buf, buf[:words]


def tail_intact(buf, words):
    t = buf[words:].cpu().numpy().view(np.uint32)
    return bool((t == CANARY).all())


def test_no_entry_point_writes_past_its_outputs(ctx, torch):
    from paper_2602_17330_gb300 import subquad

    L, P = subquad.lib(), subquad._ptr
    rep = synth.donor_repertoire(20_000, seed=3)
    n, stride, bands, rows, k = rep.n, 16, 16, 4, 3
    codes = torch.from_numpy(rep.codes).cuda()
    lens = torch.from_numpy(rep.lens).cuda()

    pk_buf, pk = guarded(torch, n * stride // 4)
    assert L.subquad_pack(ctx.handle, P(codes), int(codes.shape[1]), P(lens), n, stride, P(pk)) == 0
    torch.cuda.synchronize()
    assert tail_intact(pk_buf, n * stride // 4)

    a, b = synth.hash_coefficients(bands * rows, seed=3)
    ta = torch.from_numpy(a.view(np.int32)).cuda()
    tb = torch.from_numpy(b.view(np.int32)).cuda()
    sg_buf, sg = guarded(torch, bands * n * rows)
    assert L.subquad_sign(ctx.handle, P(pk), stride, n, k, bands, rows, P(ta), P(tb), P(sg)) == 0
    torch.cuda.synchronize()
    assert tail_intact(sg_buf, bands * n * rows)

    # the exact candidate count first, then the same call with that capacity and with half of it
    cnt = ctypes.c_int64(0)
    big = torch.empty((8 * n, 2), dtype=torch.int32, device="cuda")
    assert L.subquad_band_candidates(ctx.handle, P(sg), n, bands, rows, 64, P(big), 8 * n, ctypes.byref(cnt)) == 0
    m = int(cnt.value)
    assert m > 1000
    for cap in (m, m // 2):
        pr_buf, pr = guarded(torch, 2 * cap)
        st = L.subquad_band_candidates(ctx.handle, P(sg), n, bands, rows, 64, P(pr), cap, ctypes.byref(cnt))
        torch.cuda.synchronize()
        assert st == (0 if cap == m else subquad.SUBQUAD_ERR_CAPACITY)
        assert int(cnt.value) == m
        assert tail_intact(pr_buf, 2 * cap)
    dm = torch.zeros((1,), dtype=torch.int64, device="cuda")
    pr_buf, pr = guarded(torch, 2 * (m // 2))
    assert L.subquad_band_candidates_async(ctx.handle, P(sg), n, bands, rows, 64, None, P(pr), m // 2, P(dm)) == 0
    torch.cuda.synchronize()
    assert int(dm.item()) == m
    assert L.subquad_check(ctx.handle) == subquad.SUBQUAD_ERR_CAPACITY  # sticky overflow, read and cleared
    assert tail_intact(pr_buf, 2 * (m // 2))

    pairs = big[:m].contiguous()
    for binned in (False, True):
        sw_buf, sw = guarded(torch, m)
        fn = L.subquad_align_score_binned if binned else L.subquad_align_score
        assert fn(ctx.handle, P(pk), stride, P(pairs), m, 10, 1, P(sw)) == 0
        torch.cuda.synchronize()
        assert tail_intact(sw_buf, m)
    self_buf, self_sc = guarded(torch, n)
    assert L.subquad_self_scores(ctx.handle, P(pk), stride, n, 10, 1, P(self_sc)) == 0
    torch.cuda.synchronize()
    assert tail_intact(self_buf, n)

    d, hidden = 64, 16
    emb = torch.from_numpy(synth.unit_embeddings(n, d, seed=3)).cuda()
    params = torch.from_numpy(synth.gate_parameters(hidden, seed=3)).cuda()
    fu_buf, fu = guarded(torch, m)
    al_buf, al = guarded(torch, m)
    assert L.subquad_fuse_forward(ctx.handle, P(pairs), m, P(sw), P(self_sc), P(pk), stride, P(emb), d, P(params),
                                  hidden, P(fu), P(al)) == 0
    torch.cuda.synchronize()
    assert tail_intact(fu_buf, m) and tail_intact(al_buf, m)
    assert L.subquad_check(ctx.handle) == 0
