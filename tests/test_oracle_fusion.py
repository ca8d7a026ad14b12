"""Pins for the oracle's gated fusion (Eq. alpha, Eq. wm, Eq. afused), its
adjoint, the gate-training loss, Adam and cross-donor top-k."""
import numpy as np
import pytest
import scipy.special
import scipy.spatial.distance

from paper_2602_17330_gb300 import synth


@pytest.fixture(scope="module")
def small(oracle_mod):
    rep = synth.make_repertoire(300, 30, seed=2)
    a, b = synth.hash_coefficients(32, seed=2)
    sig = oracle_mod.sign(rep.codes, rep.lens, 3, a, b)
    C = oracle_mod.candidates(sig, 16, 2, 0)
    sw = oracle_mod.sw_pairs(rep.codes, rep.lens, C)
    self_sc = oracle_mod.self_scores(rep.codes, rep.lens)
    emb = synth.family_embeddings(rep.family, 24, seed=2)
    emb *= np.linspace(0.5, 2.0, rep.n, dtype=np.float32)[:, None]  # not unit norm
    return dict(rep=rep, C=C, sw=sw, self=self_sc, emb=np.ascontiguousarray(emb))


def params_from(W1, b1, w2, b2):
    return np.concatenate([np.asarray(W1, np.float64).ravel(), b1, w2, [b2]]).astype(np.float32)


def test_alpha_is_two_way_softmax_of_gate_bias(oracle_mod, small):
    h = 8
    for b2 in (-3.0, -0.25, 0.0, 0.7, 4.0):
        p = params_from(np.zeros((h, 3)), np.zeros(h), np.ones(h), b2)
        out = oracle_mod.fuse_forward(small["C"], small["sw"], small["self"], small["rep"].lens, small["emb"], p, h)
        want = scipy.special.softmax([np.float32(b2), 0.0])[0]
        assert np.allclose(out["alpha"], want, rtol=0, atol=1e-15)


def test_alpha_two_way_softmax_through_hidden_layer(oracle_mod, small):
    rng = np.random.default_rng(0)
    h = 6
    b1 = rng.normal(size=h).astype(np.float32)
    w2 = rng.normal(size=h).astype(np.float32)
    p = params_from(np.zeros((h, 3)), b1, w2, 0.3)
    out = oracle_mod.fuse_forward(small["C"], small["sw"], small["self"], small["rep"].lens, small["emb"], p, h)
    g = float(np.dot(w2.astype(np.float64), np.maximum(b1.astype(np.float64), 0))) + float(np.float32(0.3))
    assert np.allclose(out["alpha"], scipy.special.softmax([g, 0.0])[0], rtol=0, atol=1e-15)


def test_feature_order_s_c_delta(oracle_mod, small):
    """One hidden unit reading exactly one feature pins the order [s, c, |dL|]."""
    C, lens = small["C"], small["rep"].lens
    s_ref = small["sw"] / np.sqrt(small["self"][C[:, 0]].astype(np.float64) * small["self"][C[:, 1]])
    e = small["emb"].astype(np.float64)
    c_ref = np.array([1.0 - scipy.spatial.distance.cosine(e[i], e[j]) for i, j in C])
    d_ref = np.abs(lens[C[:, 0]].astype(np.float64) - lens[C[:, 1]])
    for col, feat, bias in ((0, s_ref, 0.0), (1, c_ref + 1.0, 1.0), (2, d_ref, 0.0)):
        W1 = np.zeros((1, 3))
        W1[0, col] = 1.0
        p = params_from(W1, [bias], [1.0], 0.0)
        out = oracle_mod.fuse_forward(C, small["sw"], small["self"], lens, small["emb"], p, 1)
        assert np.allclose(out["alpha"], scipy.special.expit(feat), rtol=0, atol=1e-12)


def test_limits_and_channels(oracle_mod, small):
    C, lens = small["C"], small["rep"].lens
    e = small["emb"].astype(np.float64)
    c_ref = np.array([1.0 - scipy.spatial.distance.cosine(e[i], e[j]) for i, j in C])
    s_ref = small["sw"] / np.sqrt(small["self"][C[:, 0]].astype(np.float64) * small["self"][C[:, 1]])
    h = 4
    hi = oracle_mod.fuse_forward(C, small["sw"], small["self"], lens, small["emb"],
                                 params_from(np.zeros((h, 3)), np.zeros(h), np.zeros(h), 80.0), h)
    lo = oracle_mod.fuse_forward(C, small["sw"], small["self"], lens, small["emb"],
                                 params_from(np.zeros((h, 3)), np.zeros(h), np.zeros(h), -80.0), h)
    assert np.allclose(hi["fused"], s_ref, rtol=0, atol=1e-12)
    assert np.allclose(lo["fused"], (1.0 + c_ref) / 2.0, rtol=0, atol=1e-12)
    assert np.allclose(hi["c"], c_ref, atol=1e-12) and np.allclose(hi["s"], s_ref, atol=1e-15)
    assert (s_ref >= 0).all() and (s_ref <= 1).all()
    mid = oracle_mod.fuse_forward(C, small["sw"], small["self"], lens, small["emb"], synth.gate_parameters(h), h)
    assert (mid["fused"] >= 0).all() and (mid["fused"] <= 1).all()


def loss_of(oracle_mod, d, params, emb, y, w, h):
    out = oracle_mod.fuse_forward(d["C"], d["sw"], d["self"], d["rep"].lens, emb, params, h)
    return oracle_mod.bce_loss(out["fused"], y, w)[0]


def test_backward_matches_central_differences(oracle_mod, small):
    """FP64 central differences, h = 1e-6, relative tolerance 1e-4, on every
    gate parameter and a sample of embedding coordinates.  Parameters and
    embeddings are float32, so the step actually taken is the float32
    difference, which the quotient uses."""
    d = small
    h = 8
    params = synth.gate_parameters(h, seed=5)
    y, g = oracle_mod.pair_labels(d["C"], d["rep"].family, d["rep"].subgroup)
    w = oracle_mod.pair_weights(g, 1)
    out = oracle_mod.fuse_forward(d["C"], d["sw"], d["self"], d["rep"].lens, d["emb"], params, h)
    _, dL = oracle_mod.bce_loss(out["fused"], y, w)
    gp, ge = oracle_mod.fuse_backward(d["C"], d["sw"], d["self"], d["rep"].lens, d["emb"], params, h, dL)
    step = 1e-6

    def fd(get_plus_minus):
        (pp, ep), (pm, em), delta = get_plus_minus()
        return (loss_of(oracle_mod, d, pp, ep, y, w, h) - loss_of(oracle_mod, d, pm, em, y, w, h)) / delta

    for k in range(params.shape[0]):
        def pm(k=k):
            up, dn = params.copy(), params.copy()
            up[k] = np.float32(params[k] + step)
            dn[k] = np.float32(params[k] - step)
            return (up, d["emb"]), (dn, d["emb"]), float(up[k]) - float(dn[k])
        num = fd(pm)
        assert abs(num - gp[k]) <= 1e-4 * abs(gp[k]) + 1e-9, (k, num, gp[k])
    rng = np.random.default_rng(9)
    used = np.unique(d["C"].ravel())
    for _ in range(25):
        i = int(rng.choice(used))
        c = int(rng.integers(0, d["emb"].shape[1]))

        def pe(i=i, c=c):
            up, dn = d["emb"].copy(), d["emb"].copy()
            up[i, c] = np.float32(d["emb"][i, c] + step)
            dn[i, c] = np.float32(d["emb"][i, c] - step)
            return (params, up), (params, dn), float(up[i, c]) - float(dn[i, c])
        num = fd(pe)
        assert abs(num - ge[i, c]) <= 1e-4 * abs(ge[i, c]) + 1e-9, (i, c, num, ge[i, c])


def test_bce_and_weights_against_torch(oracle_mod):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    m = 500
    fused = rng.uniform(0.001, 0.999, m)
    fused[:3] = [0.0, 1.0, 0.5]
    y = rng.integers(0, 2, m).astype(np.uint8)
    group = rng.choice([0, 1, 2, 5], m, p=[0.85, 0.08, 0.05, 0.02]).astype(np.int32)
    w = oracle_mod.pair_weights(group, 8)
    assert abs(w.sum() - m) < 1e-9
    counts = np.bincount(group, minlength=8)
    prod = w * counts[group]
    assert np.allclose(prod, prod[0])
    loss, dL = oracle_mod.bce_loss(fused, y, w)
    ft = torch.tensor(np.clip(fused, 1e-7, 1 - 1e-7), dtype=torch.float64, requires_grad=True)
    yt = torch.tensor(y, dtype=torch.float64)
    wt = torch.tensor(w, dtype=torch.float64)
    lt = torch.nn.functional.binary_cross_entropy(ft, yt, weight=wt, reduction="sum") / wt.sum()
    lt.backward()
    assert abs(loss - lt.item()) < 1e-12
    inside = (fused > 1e-7) & (fused < 1 - 1e-7)
    assert np.allclose(dL[inside], ft.grad.numpy()[inside], rtol=1e-10, atol=1e-15)
    assert (dL[~inside] == 0).all()


def test_adam_against_torch(oracle_mod):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    P = 17
    p0 = rng.normal(size=P)
    param, m1, m2 = p0.copy(), np.zeros(P), np.zeros(P)
    tp = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    for t in range(1, 31):
        g = rng.normal(size=P)
        oracle_mod.adam_step(param, np.ascontiguousarray(g), m1, m2, t)
        opt.zero_grad()
        tp.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        assert np.allclose(param, tp.detach().numpy(), rtol=0, atol=1e-13)


def test_topk_against_brute_force(oracle_mod):
    rng = np.random.default_rng(12)
    n, m, k = 80, 600, 5
    i = rng.integers(0, n, m)
    j = rng.integers(0, n, m)
    keep = i < j
    pairs = np.unique(np.stack([i[keep], j[keep]], 1), axis=0).astype(np.uint32)
    scores = rng.integers(0, 6, pairs.shape[0]).astype(np.int32)  # many ties
    donor = rng.integers(0, 4, n).astype(np.int32)
    queries = np.arange(0, n, 3, dtype=np.uint32)
    ids, sc = oracle_mod.topk(pairs, scores, donor, queries, k)
    for qi, q in enumerate(queries):
        cand = []
        for (a, b), s in zip(pairs, scores):
            other = b if a == q else a if b == q else None
            if other is not None and donor[other] != donor[q]:
                cand.append((-int(s), int(other)))
        cand.sort()
        want = cand[:k] + [(1, 0xFFFFFFFF)] * (k - len(cand[:k]))
        assert [(-int(s), int(x)) for s, x in zip(sc[qi], ids[qi])] == want


# Tolerance of a float32 adjoint against the FP64 oracle, per gradient entry:
#   |g - g*| <= max(GRAD_RTOL |g*|, GRAD_KAPPA * scale),
# where scale is the oracle's rounding scale of that entry (every pair's term
# evaluated on operand magnitudes, see oracle_fuse_backward_scale).  Where the
# terms do not cancel, GRAD_RTOL |g*| is the larger and the relative 1e-4
# applies; where they cancel to below GRAD_KAPPA * scale / GRAD_RTOL, float32
# cannot deliver 1e-4 of the result and the floor is the rounding error a
# correct float32 evaluation may carry.  GRAD_KAPPA = 2^-18 = 64 unit
# roundoffs; a float32 evaluation of the chain measures below 0.2 u * scale
# (the test below), while the first-order worst case with every rounding
# aligned is a few hundred u at h = 64 and length differences near 20.
GRAD_RTOL = 1e-4
GRAD_KAPPA = 2.0 ** -18


def float32_adjoint(C, sw, self_sc, lens, emb, params, h, dL):
    """The adjoint's parameter gradient with every per-pair quantity rounded to
    float32 (numpy), the per-pair terms summed in float64."""
    f32 = np.float32
    i, j = C[:, 0].astype(np.int64), C[:, 1].astype(np.int64)
    s = sw.astype(f32) / np.sqrt(self_sc[i].astype(f32) * self_sc[j].astype(f32))
    ei, ej = emb[i], emb[j]
    dot = (ei * ej).sum(1, dtype=f32)
    c = dot / np.sqrt((ei * ei).sum(1, dtype=f32) * (ej * ej).sum(1, dtype=f32))
    delta = np.abs(lens[i].astype(f32) - lens[j].astype(f32))
    W1 = params[: 3 * h].reshape(h, 3)
    b1, w2, b2 = params[3 * h: 4 * h], params[4 * h: 5 * h], params[5 * h]
    z = (W1[:, 0][None] * s[:, None] + W1[:, 1][None] * c[:, None] + W1[:, 2][None] * delta[:, None]
         + b1[None]).astype(f32)
    g = (np.maximum(z, f32(0)) * w2[None]).sum(1, dtype=f32) + b2
    a = f32(1) / (f32(1) + np.exp(-g))
    d_g = dL.astype(f32) * (s - f32(0.5) * (f32(1) + c)) * a * (f32(1) - a)
    dz = np.where(z > 0, d_g[:, None] * w2[None], f32(0)).astype(f32)
    out = np.zeros(5 * h + 1)
    out[0:3 * h:3] = (dz * s[:, None]).astype(np.float64).sum(0)
    out[1:3 * h:3] = (dz * c[:, None]).astype(np.float64).sum(0)
    out[2:3 * h:3] = (dz * delta[:, None]).astype(np.float64).sum(0)
    out[3 * h:4 * h] = dz.astype(np.float64).sum(0)
    out[4 * h:5 * h] = (d_g[:, None] * np.maximum(z, f32(0))).astype(np.float64).sum(0)
    out[5 * h] = d_g.astype(np.float64).sum()
    return out


@pytest.mark.parametrize("d,h", [(24, 8), (128, 32)])
def test_gradient_rounding_scale_bounds_float32_chain(oracle_mod, small, d, h):
    """The scale bounds the exact gradient (triangle inequality), and a float32
    evaluation of the chain lies within GRAD_KAPPA * scale of the FP64
    gradient even when the per-pair upstream gradients have random signs (the
    sum then cancels to far below its terms)."""
    rep = small["rep"]
    emb = synth.family_embeddings(rep.family, d, seed=4) * np.float32(1.7)
    params = synth.gate_parameters(h, seed=4)
    dL = np.random.default_rng(4).standard_normal(small["C"].shape[0])
    gp, _ = oracle_mod.fuse_backward(small["C"], small["sw"], small["self"], rep.lens, emb, params, h, dL,
                                     with_emb=False)
    scale, se = oracle_mod.fuse_backward_scale(small["C"], small["sw"], small["self"], rep.lens, emb, params, h, dL)
    assert (np.abs(gp) <= scale * (1 + 1e-12)).all()
    _, ge = oracle_mod.fuse_backward(small["C"], small["sw"], small["self"], rep.lens, emb, params, h, dL)
    assert (np.abs(ge) <= se * (1 + 1e-12) + 1e-300).all()
    g32 = float32_adjoint(small["C"], small["sw"], small["self"], rep.lens, emb, params, h, dL.astype(np.float32))
    err = np.abs(g32 - gp)
    assert (err <= GRAD_KAPPA * scale).all(), float((err / scale).max())
    assert (err <= 2.0 ** -22 * scale).all(), "float32 chain error above 0.25 u * scale"
