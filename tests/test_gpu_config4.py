"""Gate training at its full size: the first 4,000,000 candidate pairs of the
1,000,000-sequence donor, d = 128 family-correlated embeddings, gate 3-32-1,
weighted BCE on family-match labels with inverse-subgroup weights.  The GPU
forward, loss and adjoint (parameters and embeddings) are compared with the
FP64 oracle on the oracle's own candidate list and alignment scores: fused
scores within 1e-5 relative, the loss within 1e-5, gradients per entry within
max(1e-4 |g*|, 2^-18 scale)."""
import numpy as np
import pytest

from paper_2602_17330_gb300 import synth

pytestmark = pytest.mark.gpu

GRAD_RTOL, GRAD_KAPPA = 1e-4, 2.0 ** -18


def test_config4_full_size_gradient(oracle_mod):
    import torch

    from paper_2602_17330_gb300 import _build, subquad

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    _build.build()
    threads = oracle_mod.host_threads()
    rep = synth.donor_repertoire(1_000_000, seed=0)
    a, b = synth.hash_coefficients(64, seed=0)
    sig = oracle_mod.sign_mt(rep.codes, rep.lens, 3, a, b, threads)
    C = oracle_mod.candidates(sig, 16, 4, 2048)[:4_000_000]
    assert C.shape[0] == 4_000_000
    del sig
    sw = oracle_mod.sw_pairs_mt(rep.codes, rep.lens, C, threads)
    self_sc = oracle_mod.self_scores(rep.codes, rep.lens)
    emb = synth.family_embeddings(rep.family, 128, seed=1)
    hidden = 32
    params = synth.gate_parameters(hidden, seed=1)
    y, g = oracle_mod.pair_labels(C, rep.family, rep.subgroup)
    w = oracle_mod.pair_weights(g, int(rep.subgroup.max()) + 1)
    fused_o = oracle_mod.fuse_forward_mt(C, sw, self_sc, rep.lens, emb, params, hidden, threads)
    loss_o, dL_o = oracle_mod.bce_loss(fused_o, y, w)
    dL32 = dL_o.astype(np.float32)

    with subquad.Context(0) as ctx:
        dev = ctx.device
        packed = ctx.pack(torch.from_numpy(rep.codes), torch.from_numpy(rep.lens), 16)
        pairs = torch.from_numpy(C.view(np.int32)).to(dev)
        sw_t = torch.from_numpy(sw).to(dev)
        self_t = torch.from_numpy(self_sc).to(dev)
        emb_t = torch.from_numpy(emb).to(dev)
        par_t = torch.from_numpy(params).to(dev)
        fused = ctx.fuse_forward(pairs, sw_t, self_t, packed, emb_t, par_t, hidden).cpu().numpy()
        err = np.abs(fused.astype(np.float64) - fused_o)
        assert (err <= 1e-5 * np.maximum(np.abs(fused_o), 1e-3)).all(), err.max()
        label = torch.from_numpy(y).to(dev)
        weight = torch.from_numpy(w.astype(np.float32)).to(dev)
        loss, _ = ctx.bce_loss(torch.from_numpy(fused_o.astype(np.float32)).to(dev), label, weight)
        assert abs(float(loss.item()) - loss_o) <= 1e-5 * abs(loss_o)
        gp, ge = ctx.fuse_backward(pairs, sw_t, self_t, packed, emb_t, par_t, hidden,
                                   torch.from_numpy(dL32).to(dev))
        gp, ge = gp.cpu().numpy(), ge.cpu().numpy()
        ctx.check()
    args = (C, sw, self_sc, rep.lens, emb, params, hidden, dL32.astype(np.float64))
    want_p, want_e = oracle_mod.fuse_backward(*args)
    scale_p, scale_e = oracle_mod.fuse_backward_scale(*args)
    for got, want, scale, what in ((gp, want_p, scale_p, "parameters"), (ge, want_e, scale_e, "embeddings")):
        e = np.abs(got.astype(np.float64) - want)
        rel_bound = GRAD_RTOL * np.abs(want)
        bound = np.maximum(rel_bound, GRAD_KAPPA * scale)
        at_rel = (rel_bound >= GRAD_KAPPA * scale) & (want != 0)
        worst_rel = float((e[at_rel] / np.abs(want[at_rel])).max()) if at_rel.any() else 0.0
        print(f"\n4M pairs, {what}: {int(at_rel.sum())}/{e.size} entries at rel 1e-4 (worst rel {worst_rel:.2e}), "
              f"worst err / (u scale) {float((e / np.maximum(scale, 1e-300)).max()) / 2.0 ** -24:.3f}")
        assert (e <= bound).all(), f"{what}: worst error / bound {(e / np.maximum(bound, 1e-300)).max():.3f}"
