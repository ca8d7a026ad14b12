"""GPU parity of the M-channel gated fusion (Eq. wm at M = 3 with the MinHash
Jaccard channel, and M = 2) and its adjoint, through the C ABI, against the
FP64 oracle.  Fused scores and weights: |x - y| <= 1e-5 max(|y|, 1e-3);
gradients: per entry max(1e-4 |g*|, 2^-18 scale) with the oracle's rounding
scale (see test_gpu_training)."""
import numpy as np
import pytest

from paper_2602_17330_gb300 import synth

pytestmark = pytest.mark.gpu

RTOL, FLOOR = 1e-5, 1e-3
GRAD_RTOL, GRAD_KAPPA = 1e-4, 2.0 ** -18


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


def make_case(ctx, torch, oracle_mod, n, bands, rows, stride, d, seed):
    rep = synth.donor_repertoire(n, seed=seed) if stride == 16 else synth.zipf_repertoire(n, seed=seed, hi=300)
    a, b = synth.hash_coefficients(bands * rows, seed=seed)
    packed = ctx.pack(torch.from_numpy(rep.codes), torch.from_numpy(rep.lens), stride)
    sig = ctx.sign(packed, rep.n, 3, torch.from_numpy(a.view(np.int32)), torch.from_numpy(b.view(np.int32)), bands,
                   rows)
    sig_o = oracle_mod.sign(rep.codes, rep.lens, 3, a, b)
    assert (to_np(sig).view(np.uint32).transpose(1, 0, 2).reshape(rep.n, -1) == sig_o).all()
    # the kernels read the sequence-major copy; the oracle's signatures are uploaded for them
    sig_seq = ctx.sig_sequence_major(sig)
    assert (to_np(sig_seq).view(np.uint32) == sig_o).all()
    sig = torch.from_numpy(sig_o.view(np.int32)).to(ctx.device)
    C = oracle_mod.candidates(sig_o, bands, rows, 0)
    sw_o = oracle_mod.sw_pairs(rep.codes, rep.lens, C)
    self_o = oracle_mod.self_scores(rep.codes, rep.lens)
    emb = synth.family_embeddings(rep.family, d, seed=seed)
    emb = np.ascontiguousarray(emb * np.random.default_rng(seed).uniform(0.5, 2.0, (rep.n, 1)).astype(np.float32))
    dev = ctx.device
    return dict(rep=rep, packed=packed, sig=sig, sig_o=sig_o, C=C, C_t=torch.from_numpy(C.view(np.int32)).to(dev),
                sw_o=sw_o, sw_t=torch.from_numpy(sw_o).to(dev), self_o=self_o,
                self_t=torch.from_numpy(self_o).to(dev), emb=emb, emb_t=torch.from_numpy(emb).to(dev))


def assert_close(got, want):
    err = np.abs(got.astype(np.float64) - want)
    bound = RTOL * np.maximum(np.abs(want), FLOOR)
    assert (err <= bound).all(), f"max err {err.max():.3e}, worst ratio {(err / bound).max():.3f}"


@pytest.mark.parametrize("M,bands,rows,stride,d,h", [
    (3, 16, 4, 16, 64, 16), (3, 16, 4, 16, 128, 32), (3, 8, 3, 32, 64, 64), (3, 32, 4, 32, 36, 1),
    (2, 16, 4, 16, 64, 16), (2, 16, 4, 32, 128, 32)])
def test_forward_mc_matches_oracle(ctx, torch, oracle_mod, M, bands, rows, stride, d, h):
    c = make_case(ctx, torch, oracle_mod, 12_000, bands, rows, stride, d, seed=31 + M + rows + d)
    params = synth.gate_parameters_mc(h, M, seed=M + h)
    fused, w = ctx.fuse_forward_mc(c["C_t"], c["sw_t"], c["self_t"], c["packed"], c["emb_t"], c["sig"],
                                   torch.from_numpy(params).to(ctx.device), h, M, want_weights=True)
    want = oracle_mod.fuse_forward_mc(c["C"], c["sw_o"], c["self_o"], c["rep"].lens, c["emb"], c["sig_o"], params, h,
                                      M)
    assert_close(to_np(fused), want["fused"])
    assert_close(to_np(w), want["weights"])
    assert np.allclose(to_np(w).sum(1), 1.0, atol=1e-6)
    if M == 2:  # the two-channel entry point computes the same function
        f2 = ctx.fuse_forward(c["C_t"], c["sw_t"], c["self_t"], c["packed"], c["emb_t"],
                              torch.from_numpy(params).to(ctx.device), h)
        assert_close(to_np(f2), want["fused"])


def grads_ok(got, want, scale):
    err = np.abs(got.astype(np.float64) - want)
    bound = np.maximum(GRAD_RTOL * np.abs(want), GRAD_KAPPA * scale)
    return bool((err <= bound).all()), float((err / np.maximum(bound, 1e-300)).max())


@pytest.mark.parametrize("M,stride,d,h", [(3, 16, 128, 32), (3, 32, 64, 16), (2, 16, 64, 16)])
def test_backward_mc_matches_oracle(ctx, torch, oracle_mod, M, stride, d, h):
    c = make_case(ctx, torch, oracle_mod, 12_000, 16, 4, stride, d, seed=41 + M + d)
    rep = c["rep"]
    params = synth.gate_parameters_mc(h, M, seed=7 + M)
    y, g = oracle_mod.pair_labels(c["C"], rep.family, rep.subgroup)
    wts = oracle_mod.pair_weights(g, int(rep.subgroup.max()) + 1)
    out = oracle_mod.fuse_forward_mc(c["C"], c["sw_o"], c["self_o"], rep.lens, c["emb"], c["sig_o"], params, h, M)
    _, dL = oracle_mod.bce_loss(out["fused"], y, wts)
    dL32 = dL.astype(np.float32)
    args = (c["C"], c["sw_o"], c["self_o"], rep.lens, c["emb"], c["sig_o"], params, h, M, dL32.astype(np.float64))
    want_p, want_e = oracle_mod.fuse_backward_mc(*args)
    scale_p, scale_e = oracle_mod.fuse_backward_mc_scale(*args)
    p_t = torch.from_numpy(params).to(ctx.device)
    dL_t = torch.from_numpy(dL32).to(ctx.device)
    gp, ge = ctx.fuse_backward_mc(c["C_t"], c["sw_t"], c["self_t"], c["packed"], c["emb_t"], c["sig"], p_t, h, M,
                                  dL_t)
    gp2, ge2 = ctx.fuse_backward_mc(c["C_t"], c["sw_t"], c["self_t"], c["packed"], c["emb_t"], c["sig"], p_t, h, M,
                                    dL_t)
    assert torch.equal(gp, gp2) and torch.equal(ge, ge2), "not bitwise reproducible"
    ok, worst = grads_ok(to_np(gp), want_p, scale_p)
    assert ok, f"parameter gradient worst error / bound {worst:.3f}"
    ok, worst = grads_ok(to_np(ge), want_e, scale_e)
    assert ok, f"embedding gradient worst error / bound {worst:.3f}"
    if M == 2:  # and the two-channel adjoint agrees within the same bound
        gq = ctx.fuse_backward(c["C_t"], c["sw_t"], c["self_t"], c["packed"], c["emb_t"], p_t, h, dL_t,
                               want_emb=False)
        ok, worst = grads_ok(to_np(gq), want_p, scale_p)
        assert ok, worst


def test_mc_argument_errors(ctx, torch):
    from paper_2602_17330_gb300 import subquad

    z = torch.zeros(16, dtype=torch.int32, device=ctx.device)
    e = torch.zeros((4, 8), dtype=torch.float32, device=ctx.device)
    pk = torch.zeros((4, 16), dtype=torch.uint8, device=ctx.device)
    par = torch.zeros(64, dtype=torch.float32, device=ctx.device)
    for channels, sig in ((4, None), (1, None), (3, None)):
        with pytest.raises(subquad.SubquadError):
            ctx.fuse_forward_mc(z.view(-1, 2), z[:8], z, pk, e, sig, par, 2, channels)
