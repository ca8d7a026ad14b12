"""GPU parity for gate training (labels, weights, weighted BCE, the fusion
adjoint, Adam) against the FP64 oracle.

Tolerances, derived from the FP32 arithmetic of the kernels:
* loss and dL/dfused: relative 1e-5 (FP32 inputs, FP64 sums);
* parameter and embedding gradients, per entry:
  |g - g*| <= max(1e-4 |g*|, 2^-18 * scale), where scale is the oracle's
  rounding scale of the entry (each pair's term evaluated on operand
  magnitudes): where the pair terms do not cancel the relative 1e-4 applies,
  and where they cancel below 2^-18 scale / 1e-4 no float32 evaluation can
  reach 1e-4 of the result, so the floor is 64 unit roundoffs of the scale.
  The worst observed error / scale is printed (run with -s).
"""
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


@pytest.fixture(scope="module")
def case(ctx, torch, oracle_mod):
    """A donor of 30,000 sequences with its candidate list, family-correlated
    embeddings of d = 128 scaled off unit norm, gate 3-32-1."""
    rep = synth.donor_repertoire(30_000, seed=7)
    a, b = synth.hash_coefficients(64, seed=7)
    packed = ctx.pack(torch.from_numpy(rep.codes), torch.from_numpy(rep.lens), 16)
    # the step's inputs come from the oracle side and are uploaded for the GPU
    pairs_np = oracle_mod.candidates(oracle_mod.sign(rep.codes, rep.lens, 3, a, b), 16, 4, 2048)
    sw_np = oracle_mod.sw_pairs(rep.codes, rep.lens, pairs_np)
    self_np = oracle_mod.self_scores(rep.codes, rep.lens)
    pairs = torch.from_numpy(pairs_np.view(np.int32)).to(ctx.device)
    sw = torch.from_numpy(sw_np).to(ctx.device)
    self_sc = torch.from_numpy(self_np).to(ctx.device)
    emb = synth.family_embeddings(rep.family, 128, seed=7)
    emb = np.ascontiguousarray(emb * np.random.default_rng(7).uniform(0.5, 2.0, (rep.n, 1)).astype(np.float32))
    hidden = 32
    params = synth.gate_parameters(hidden, seed=7)
    return dict(rep=rep, packed=packed, pairs=pairs, pairs_np=pairs_np, sw=sw, sw_np=sw_np, self=self_sc,
                self_np=self_np, emb=emb,
                emb_t=torch.from_numpy(emb).to(ctx.device), hidden=hidden, params=params,
                params_t=torch.from_numpy(params).to(ctx.device))


def test_labels_and_weights(ctx, torch, oracle_mod, case):
    rep = case["rep"]
    label, group = ctx.pair_labels(case["pairs"], torch.from_numpy(rep.family), torch.from_numpy(rep.subgroup))
    y, g = oracle_mod.pair_labels(case["pairs_np"], rep.family, rep.subgroup)
    assert (to_np(label) == y).all() and (to_np(group) == g).all()
    assert y.sum() > 0 and (g > 0).sum() > 0
    w = to_np(ctx.pair_weights(group, 51))
    want = oracle_mod.pair_weights(g, 51)
    assert np.allclose(w, want, rtol=1e-6, atol=0)


def test_bce_loss_and_gradient(ctx, torch, oracle_mod, case):
    """Both sides take the oracle's fused scores (rounded to float32, the
    dtype the fusion writes), labels and weights."""
    rep = case["rep"]
    out = oracle_mod.fuse_forward(case["pairs_np"], case["sw_np"], case["self_np"], rep.lens, case["emb"],
                                  case["params"], case["hidden"])
    f32 = out["fused"].astype(np.float32)
    y, g = oracle_mod.pair_labels(case["pairs_np"], rep.family, rep.subgroup)
    w32 = oracle_mod.pair_weights(g, 51).astype(np.float32)
    dev = ctx.device
    loss, dL = ctx.bce_loss(torch.from_numpy(f32).to(dev), torch.from_numpy(y).to(dev), torch.from_numpy(w32).to(dev))
    want_loss, want_dL = oracle_mod.bce_loss(f32.astype(np.float64), y, w32.astype(np.float64))
    assert abs(float(to_np(loss)[0]) - want_loss) <= 1e-5 * abs(want_loss)
    assert np.allclose(to_np(dL), want_dL, rtol=1e-5, atol=1e-12)


def test_bce_clamp_boundaries(ctx, torch, oracle_mod):
    """Fused scores at and around the loss's clamp points (the float
    neighbours of 1e-7 and 1 - 1e-7, 0, 1, 1/2) with both labels: the
    kernels decide the clamp with float thresholds, which must decide every
    float exactly as the oracle's FP64 comparisons (zero gradients in the same
    places) and give the loss and the gradient within 1e-5."""
    vals = []
    for c in (1e-7, 1.0 - 1e-7):
        f = np.float32(c)
        for k in range(-3, 4):
            v = f
            for _ in range(abs(k)):
                v = np.nextafter(v, np.float32(np.inf if k > 0 else -np.inf), dtype=np.float32)
            vals.append(v)
    vals += [np.float32(0.0), np.float32(1.0), np.float32(0.5), np.float32(1e-30), np.float32(0.999)]
    f32 = np.array(vals * 2, dtype=np.float32)
    y = np.array([0] * len(vals) + [1] * len(vals), dtype=np.uint8)
    w32 = np.random.default_rng(11).uniform(0.5, 2.0, f32.shape[0]).astype(np.float32)
    dev = ctx.device
    loss, dL = ctx.bce_loss(torch.from_numpy(f32).to(dev), torch.from_numpy(y).to(dev), torch.from_numpy(w32).to(dev))
    want_loss, want_dL = oracle_mod.bce_loss(f32.astype(np.float64), y, w32.astype(np.float64))
    got = to_np(dL)
    assert ((got == 0) == (want_dL == 0)).all(), "clamp decided differently"
    assert abs(float(to_np(loss)[0]) - want_loss) <= 1e-5 * abs(want_loss)
    assert np.allclose(got, want_dL, rtol=1e-5, atol=0)


GRAD_RTOL = 1e-4
GRAD_KAPPA = 2.0 ** -18


def grads_close(got, want, scale, what):
    """Per-entry bound max(GRAD_RTOL |g*|, GRAD_KAPPA scale); returns the worst
    error / bound and prints the worst error in units of u * scale and the
    worst relative error among entries checked at the relative bound."""
    err = np.abs(got.astype(np.float64) - want)
    rel_bound = GRAD_RTOL * np.abs(want)
    floor = GRAD_KAPPA * scale
    bound = np.maximum(rel_bound, floor)
    ratio = err / np.maximum(bound, 1e-300)
    checked_rel = (rel_bound >= floor) & (want != 0)
    worst_rel = float((err[checked_rel] / np.abs(want[checked_rel])).max()) if checked_rel.any() else 0.0
    print(f"\n{what}: worst err / (u scale) = {float((err / np.maximum(scale, 1e-300)).max()) / 2.0 ** -24:.3f}, "
          f"{int(checked_rel.sum())}/{err.size} entries at rel {GRAD_RTOL:g} (worst rel {worst_rel:.2e})")
    return bool((err <= bound).all()), float(ratio.max())


def check_backward(ctx, torch, oracle_mod, case, dL, what):
    rep = case["rep"]
    dL_t = torch.from_numpy(dL.astype(np.float32)).to(ctx.device)
    gp, ge = ctx.fuse_backward(case["pairs"], case["sw"], case["self"], case["packed"], case["emb_t"],
                               case["params_t"], case["hidden"], dL_t)
    gp2, ge2 = ctx.fuse_backward(case["pairs"], case["sw"], case["self"], case["packed"], case["emb_t"],
                                 case["params_t"], case["hidden"], dL_t)
    assert torch.equal(gp, gp2) and torch.equal(ge, ge2), "backward is not bitwise reproducible"
    dL64 = dL.astype(np.float32).astype(np.float64)
    args = (case["pairs_np"], case["sw_np"], case["self_np"], rep.lens, case["emb"], case["params"], case["hidden"],
            dL64)
    want_p, want_e = oracle_mod.fuse_backward(*args)
    scale_p, scale_e = oracle_mod.fuse_backward_scale(*args)
    ok, worst = grads_close(to_np(gp), want_p, scale_p, what + ", parameters")
    assert ok, f"parameter gradient worst error / bound = {worst:.3f}"
    ok, worst = grads_close(to_np(ge), want_e, scale_e, what + ", embeddings")
    assert ok, f"embedding gradient worst error / bound = {worst:.3f}"


def test_backward_matches_oracle_and_is_deterministic(ctx, torch, oracle_mod, case):
    """Upstream gradients with random signs: the per-entry sums cancel hard."""
    m = case["pairs_np"].shape[0]
    dL = np.random.default_rng(3).standard_normal(m) / m
    check_backward(ctx, torch, oracle_mod, case, dL, "random-sign dL")


def test_backward_of_weighted_bce_matches_oracle(ctx, torch, oracle_mod, case):
    """The upstream gradient of training: dL/dfused of the weighted BCE at the
    oracle's fused scores (label-dependent signs, little cancellation)."""
    rep = case["rep"]
    y, g = oracle_mod.pair_labels(case["pairs_np"], rep.family, rep.subgroup)
    w = oracle_mod.pair_weights(g, 51)
    out = oracle_mod.fuse_forward(case["pairs_np"], case["sw_np"], case["self_np"], rep.lens, case["emb"],
                                  case["params"], case["hidden"])
    _, dL = oracle_mod.bce_loss(out["fused"], y, w)
    check_backward(ctx, torch, oracle_mod, case, dL, "weighted-BCE dL")


@pytest.mark.parametrize("d", [128, 64, 256, 260])
def test_backward_with_heavy_sequences(ctx, torch, oracle_mod, case, d):
    """Sequences in thousands of pairs (as the members of a bucket of 2,000
    are) take the embedding gradient's block-per-sequence path (rows up to 256
    floats; d = 260 stays on the half-warp path): first members with 1,500 and
    400 partners, a second member with 900, beside ordinary pairs."""
    rep = case["rep"]
    rng = np.random.default_rng(d)
    n = rep.n
    parts = [case["pairs_np"][:20_000].astype(np.int64)]
    for head, deg in ((5, 1500), (777, 400)):
        parts.append(np.stack([np.full(deg, head), rng.choice(np.arange(head + 1, n), deg, replace=False)], 1))
    tail = n - 10
    parts.append(np.stack([rng.choice(np.arange(tail), 900, replace=False), np.full(900, tail)], 1))
    pairs_np = np.unique(np.concatenate(parts), axis=0)
    pairs_np = pairs_np[pairs_np[:, 0] < pairs_np[:, 1]].astype(np.uint32)
    sw_np = oracle_mod.sw_pairs(rep.codes, rep.lens, pairs_np)
    emb = np.ascontiguousarray(synth.family_embeddings(rep.family, d, seed=d) *
                               rng.uniform(0.5, 2.0, (n, 1)).astype(np.float32))
    m = pairs_np.shape[0]
    dL = (rng.standard_normal(m) / m).astype(np.float32)
    dev = ctx.device
    args_t = (torch.from_numpy(pairs_np.view(np.int32)).to(dev), torch.from_numpy(sw_np).to(dev), case["self"],
              case["packed"], torch.from_numpy(emb).to(dev), case["params_t"], case["hidden"],
              torch.from_numpy(dL).to(dev))
    gp, ge = ctx.fuse_backward(*args_t)
    gp2, ge2 = ctx.fuse_backward(*args_t)
    assert torch.equal(gp, gp2) and torch.equal(ge, ge2), "backward is not bitwise reproducible"
    args = (pairs_np, sw_np, case["self_np"], rep.lens, emb, case["params"], case["hidden"], dL.astype(np.float64))
    want_p, want_e = oracle_mod.fuse_backward(*args)
    scale_p, scale_e = oracle_mod.fuse_backward_scale(*args)
    ok, worst = grads_close(to_np(gp), want_p, scale_p, f"heavy sequences d={d}, parameters")
    assert ok, f"parameter gradient worst error / bound = {worst:.3f}"
    ok, worst = grads_close(to_np(ge), want_e, scale_e, f"heavy sequences d={d}, embeddings")
    assert ok, f"embedding gradient worst error / bound = {worst:.3f}"


def test_backward_without_embedding_gradient(ctx, torch, oracle_mod, case):
    m = case["pairs_np"].shape[0]
    dL = torch.full((m,), 1.0 / m, dtype=torch.float32, device=ctx.device)
    gp = ctx.fuse_backward(case["pairs"], case["sw"], case["self"], case["packed"], case["emb_t"], case["params_t"],
                           case["hidden"], dL, want_emb=False)
    gp2, _ = ctx.fuse_backward(case["pairs"], case["sw"], case["self"], case["packed"], case["emb_t"],
                               case["params_t"], case["hidden"], dL)
    assert torch.equal(gp, gp2)


def test_pair_index(ctx, torch, case):
    n = case["rep"].n
    idx = ctx.pair_index(case["pairs"], n)
    P = case["pairs_np"].astype(np.int64)
    for side, col in (("i", 0), ("j", 1)):
        perm = to_np(idx["perm_" + side]).view(np.uint32)[: P.shape[0]]
        off = to_np(idx["off_" + side]).view(np.uint32)
        want_perm = np.argsort(P[:, col], kind="stable")
        assert (perm == want_perm).all()
        want_off = np.concatenate([[0], np.cumsum(np.bincount(P[:, col], minlength=n))])
        assert (off == want_off).all()


@pytest.mark.parametrize("P", [1000, 1003, 3])
def test_adam_against_oracle(ctx, torch, oracle_mod, P):
    """Four elements per thread on 16-byte aligned buffers, a scalar tail;
    buffers one element off alignment take the scalar kernel throughout and
    must give the same bits."""
    rng = np.random.default_rng(4)
    p0 = rng.standard_normal(P).astype(np.float32)
    p_t = torch.from_numpy(p0.copy()).cuda()
    m1 = torch.zeros_like(p_t)
    m2 = torch.zeros_like(p_t)
    # the same state one element into a larger buffer (4-byte aligned only)
    big = torch.zeros((4, P + 1), dtype=torch.float32, device="cuda")
    big[0, 1:] = p_t
    pu, m1u, m2u, gu = big[0, 1:], big[1, 1:], big[2, 1:], big[3, 1:]
    pw, a1, a2 = p0.astype(np.float64), np.zeros(P), np.zeros(P)
    for t in range(1, 31):
        g = rng.standard_normal(P).astype(np.float32)
        ctx.adam_step(p_t, torch.from_numpy(g).cuda(), m1, m2, t, lr=1e-2)
        gu.copy_(torch.from_numpy(g))
        ctx.adam_step(pu, gu, m1u, m2u, t, lr=1e-2)
        oracle_mod.adam_step(pw, g.astype(np.float64), a1, a2, t, lr=1e-2)
    assert np.allclose(to_np(p_t), pw, rtol=0, atol=2e-5)
    assert torch.equal(pu, p_t) and torch.equal(m1u, m1) and torch.equal(m2u, m2)


def test_training_steps_track_oracle(ctx, torch, oracle_mod, case):
    """Twenty full-batch steps (gate and embeddings trained) on the GPU and,
    independently, in the FP64 oracle from the same start (its forward, loss,
    adjoint and Adam; parameters rounded to float32 for each forward like the
    GPU's): the losses agree within 1e-4 relative at every step."""
    from paper_2602_17330_gb300 import train

    rep = case["rep"]
    label, group = ctx.pair_labels(case["pairs"], torch.from_numpy(rep.family), torch.from_numpy(rep.subgroup))
    weight = ctx.pair_weights(group, 51)
    y, g = oracle_mod.pair_labels(case["pairs_np"], rep.family, rep.subgroup)
    w = oracle_mod.pair_weights(g, 51)
    tr = train.GateTrainer(ctx, case["pairs"], case["sw"], case["self"], case["packed"], case["emb_t"],
                           case["params_t"], case["hidden"], label, weight, lr=1e-3, train_emb=True)
    p = case["params"].astype(np.float64)
    e = case["emb"].astype(np.float64)
    m1p, m2p, m1e, m2e = np.zeros_like(p), np.zeros_like(p), np.zeros_like(e), np.zeros_like(e)
    losses, drift = [], []
    for t in range(1, 21):
        loss = float(to_np(tr.step())[0])
        out = oracle_mod.fuse_forward(case["pairs_np"], case["sw_np"], case["self_np"], rep.lens,
                                      e.astype(np.float32), p.astype(np.float32), case["hidden"])
        want, dL = oracle_mod.bce_loss(out["fused"], y, w)
        gp, ge = oracle_mod.fuse_backward(case["pairs_np"], case["sw_np"], case["self_np"], rep.lens,
                                          e.astype(np.float32), p.astype(np.float32), case["hidden"], dL)
        oracle_mod.adam_step(p, gp, m1p, m2p, t)
        ef, gf = e.reshape(-1), np.ascontiguousarray(ge.reshape(-1))
        oracle_mod.adam_step(ef, gf, m1e.reshape(-1), m2e.reshape(-1), t)
        drift.append(abs(loss - want) / abs(want))
        losses.append(loss)
    print(f"\n20-step trajectory: worst loss drift {max(drift):.2e}")
    assert max(drift) <= 1e-4, drift
    assert losses[-1] < losses[0], "training did not reduce the loss"


def test_autograd_function_matches_direct_calls(ctx, torch, case):
    from paper_2602_17330_gb300 import train

    emb = case["emb_t"].clone().requires_grad_(True)
    params = case["params_t"].clone().requires_grad_(True)
    fused = train.fuse(ctx, case["pairs"], case["sw"], case["self"], case["packed"], emb, params, case["hidden"])
    m = fused.shape[0]
    wts = torch.linspace(-1, 1, m, device=ctx.device)
    (fused * wts).sum().backward()
    gp, ge = ctx.fuse_backward(case["pairs"], case["sw"], case["self"], case["packed"], case["emb_t"],
                               case["params_t"], case["hidden"], wts.contiguous())
    assert torch.equal(params.grad, gp) and torch.equal(emb.grad, ge)


@pytest.mark.parametrize("train_emb", [True, False])
def test_resume_from_checkpoint_is_bit_identical(ctx, torch, case, tmp_path, train_emb):
    """Six steps in one run against three steps, a checkpoint written to disk,
    a fresh trainer restored from it and three more steps: parameters,
    embeddings, Adam moments and the last loss agree bit for bit."""
    from paper_2602_17330_gb300 import train

    rep = case["rep"]
    label, group = ctx.pair_labels(case["pairs"], torch.from_numpy(rep.family), torch.from_numpy(rep.subgroup))
    weight = ctx.pair_weights(group, 51)

    def trainer():
        return train.GateTrainer(ctx, case["pairs"], case["sw"], case["self"], case["packed"], case["emb_t"],
                                 case["params_t"], case["hidden"], label, weight, lr=1e-3, train_emb=train_emb)

    full = trainer()
    for _ in range(6):
        loss_full = full.step().clone()
    first = trainer()
    for _ in range(3):
        first.step()
    path = str(tmp_path / "gate.ckpt")
    first.save(path)
    resumed = trainer()
    resumed.load(path)
    assert resumed.t == 3
    for _ in range(3):
        loss_resumed = resumed.step().clone()
    a, b = full.state(), resumed.state()
    assert a["t"] == b["t"] == 6
    for k in a:
        if torch.is_tensor(a[k]):
            assert torch.equal(a[k], b[k]), k
    assert torch.equal(loss_full, loss_resumed)
    other = train.GateTrainer(ctx, case["pairs"], case["sw"], case["self"], case["packed"], case["emb_t"],
                              case["params_t"], case["hidden"], label, weight, lr=1e-3, train_emb=not train_emb)
    with pytest.raises(ValueError):
        other.restore(first.checkpoint())
