"""Pins for the oracle's M-channel gated fusion (Eq. wm at M = 3, Eq. afused):
channels s (normalised alignment), c' = (1 + c)/2 (embedding cosine) and J
(MinHash estimate of the k-mer Jaccard index), softmax weights over the logits
(g1, 0, g3) of a two-layer gate MLP on [s, c, |dL|, J]."""
import numpy as np
import pytest
import scipy.special
import scipy.spatial.distance

from paper_2602_17330_gb300 import synth


@pytest.fixture(scope="module")
def small(oracle_mod):
    rep = synth.make_repertoire(300, 30, seed=12)
    a, b = synth.hash_coefficients(64, seed=12)
    sig = oracle_mod.sign(rep.codes, rep.lens, 3, a, b)
    C = oracle_mod.candidates(sig, 32, 2, 0)
    sw = oracle_mod.sw_pairs(rep.codes, rep.lens, C)
    self_sc = oracle_mod.self_scores(rep.codes, rep.lens)
    emb = synth.family_embeddings(rep.family, 20, seed=12)
    emb *= np.linspace(0.5, 2.0, rep.n, dtype=np.float32)[:, None]
    return dict(rep=rep, sig=sig, C=C, sw=sw, self=self_sc, emb=np.ascontiguousarray(emb))


def mc_params(W1, b1, W2, b2):
    return np.concatenate([np.asarray(W1, np.float64).ravel(), np.asarray(b1, np.float64).ravel(),
                           np.asarray(W2, np.float64).ravel(), np.asarray(b2, np.float64).ravel()]).astype(np.float32)


def fwd(oracle_mod, d, params, h, M):
    return oracle_mod.fuse_forward_mc(d["C"], d["sw"], d["self"], d["rep"].lens, d["emb"], d["sig"], params, h, M)


def channels(d):
    C = d["C"]
    s = d["sw"] / np.sqrt(d["self"][C[:, 0]].astype(np.float64) * d["self"][C[:, 1]])
    e = d["emb"].astype(np.float64)
    c = np.array([1.0 - scipy.spatial.distance.cosine(e[i], e[j]) for i, j in C])
    J = np.array([scipy.spatial.distance.hamming(d["sig"][i], d["sig"][j]) for i, j in C])
    return s, (1.0 + c) / 2.0, 1.0 - J


def test_two_channels_equal_the_two_channel_gate(oracle_mod, small):
    h = 7
    params = synth.gate_parameters(h, seed=3)  # layout W1 [h][3], b1, w2, b2 == M = 2 layout
    assert params.shape[0] == oracle_mod.mc_param_count(h, 2)
    got = fwd(oracle_mod, small, params, h, 2)
    want = oracle_mod.fuse_forward(small["C"], small["sw"], small["self"], small["rep"].lens, small["emb"], params, h)
    assert np.allclose(got["fused"], want["fused"], rtol=0, atol=1e-14)
    assert np.allclose(got["weights"][:, 0], want["alpha"], rtol=0, atol=1e-14)


def test_weights_are_the_softmax_of_the_logits(oracle_mod, small):
    """With W1 = 0 and b1 = 1 every hidden unit is 1, so the logits are the
    row sums of W2 plus b2: the weights must be scipy's softmax of (g1, 0, g3)."""
    h = 5
    rng = np.random.default_rng(1)
    for _ in range(5):
        W2 = rng.normal(size=(2, h)).astype(np.float32)
        b2 = rng.normal(size=2).astype(np.float32)
        p = mc_params(np.zeros((h, 4)), np.ones(h), W2, b2)
        out = fwd(oracle_mod, small, p, h, 3)
        g = W2.astype(np.float64).sum(1) + b2
        want = scipy.special.softmax([g[0], 0.0, g[1]])
        assert np.allclose(out["weights"], want[None, :], rtol=0, atol=1e-15)
        assert np.allclose(out["weights"].sum(1), 1.0, rtol=0, atol=1e-15)


def test_channels_and_limits(oracle_mod, small):
    s, cp, J = channels(small)
    h = 3
    out = fwd(oracle_mod, small, mc_params(np.zeros((h, 4)), np.zeros(h), np.zeros((2, h)), [0.0, 0.0]), h, 3)
    assert np.allclose(out["jaccard"], J, rtol=0, atol=1e-15)
    assert np.allclose(out["fused"], (s + cp + J) / 3.0, rtol=0, atol=1e-12)
    for b2, want in (([80.0, 0.0], s), ([0.0, 80.0], J), ([-80.0, -80.0], cp)):
        out = fwd(oracle_mod, small, mc_params(np.zeros((h, 4)), np.zeros(h), np.zeros((2, h)), b2), h, 3)
        assert np.allclose(out["fused"], want, rtol=0, atol=1e-12)
    mid = fwd(oracle_mod, small, synth.gate_parameters_mc(8, 3, seed=2), 8, 3)
    assert (mid["fused"] >= 0).all() and (mid["fused"] <= 1).all()


def test_feature_order_s_c_delta_j(oracle_mod, small):
    """One hidden unit reading one feature, feeding the channel-1 logit only,
    with channel 3 switched off: the channel-1 weight is sigmoid(feature)."""
    s, cp, J = channels(small)
    C, lens = small["C"], small["rep"].lens
    c = 2.0 * cp - 1.0
    dl = np.abs(lens[C[:, 0]].astype(np.float64) - lens[C[:, 1]])
    for col, feat, bias in ((0, s, 0.0), (1, c + 1.0, 1.0), (2, dl, 0.0), (3, J, 0.0)):
        W1 = np.zeros((1, 4))
        W1[0, col] = 1.0
        p = mc_params(W1, [bias], [[1.0], [0.0]], [0.0, -200.0])
        out = fwd(oracle_mod, small, p, 1, 3)
        assert np.allclose(out["weights"][:, 0], scipy.special.expit(feat), rtol=0, atol=1e-12)


def test_jaccard_estimate_tracks_exact_kmer_jaccard(oracle_mod, small):
    """MinHash: E[J_hat] = J exactly for min-wise hashing; over the candidate
    pairs the mean bias stays within the appendix bound 1/sqrt(H) / sqrt(m)
    (four standard errors) plus the linear family's eps_impl = 0.02."""
    rep = small["rep"]
    h = 2
    out = fwd(oracle_mod, small, mc_params(np.zeros((h, 4)), np.zeros(h), np.zeros((2, h)), [0.0, 0.0]), h, 3)

    def kset(r):
        return {tuple(rep.codes[r, p:p + 3]) for p in range(int(rep.lens[r]) - 2)}

    exact = np.array([len(kset(i) & kset(j)) / len(kset(i) | kset(j)) for i, j in small["C"]])
    bias = (out["jaccard"] - exact).mean()
    assert abs(bias) <= 4.0 / np.sqrt(64) / np.sqrt(exact.size) + 0.02, bias


def loss_of(oracle_mod, d, params, emb, y, w, h, M):
    out = oracle_mod.fuse_forward_mc(d["C"], d["sw"], d["self"], d["rep"].lens, emb, d["sig"], params, h, M)
    return oracle_mod.bce_loss(out["fused"], y, w)[0]


@pytest.mark.parametrize("M", [2, 3])
def test_backward_matches_central_differences(oracle_mod, small, M):
    d = small
    h = 6
    params = synth.gate_parameters_mc(h, M, seed=5)
    y, g = oracle_mod.pair_labels(d["C"], d["rep"].family, d["rep"].subgroup)
    w = oracle_mod.pair_weights(g, 1)
    out = oracle_mod.fuse_forward_mc(d["C"], d["sw"], d["self"], d["rep"].lens, d["emb"], d["sig"], params, h, M)
    _, dL = oracle_mod.bce_loss(out["fused"], y, w)
    gp, ge = oracle_mod.fuse_backward_mc(d["C"], d["sw"], d["self"], d["rep"].lens, d["emb"], d["sig"], params, h,
                                         M, dL)
    if M == 2:
        gp2, ge2 = oracle_mod.fuse_backward(d["C"], d["sw"], d["self"], d["rep"].lens, d["emb"], params, h, dL)
        assert np.allclose(gp, gp2, rtol=1e-12, atol=1e-15) and np.allclose(ge, ge2, rtol=1e-12, atol=1e-15)
    step = 1e-6
    for k in range(params.shape[0]):
        up, dn = params.copy(), params.copy()
        up[k] = np.float32(params[k] + step)
        dn[k] = np.float32(params[k] - step)
        num = (loss_of(oracle_mod, d, up, d["emb"], y, w, h, M) - loss_of(oracle_mod, d, dn, d["emb"], y, w, h, M)) / (
            float(up[k]) - float(dn[k]))
        assert abs(num - gp[k]) <= 1e-4 * abs(gp[k]) + 1e-9, (k, num, gp[k])
    rng = np.random.default_rng(9)
    used = np.unique(d["C"].ravel())
    for _ in range(15):
        i = int(rng.choice(used))
        c = int(rng.integers(0, d["emb"].shape[1]))
        up, dn = d["emb"].copy(), d["emb"].copy()
        up[i, c] = np.float32(d["emb"][i, c] + step)
        dn[i, c] = np.float32(d["emb"][i, c] - step)
        num = (loss_of(oracle_mod, d, params, up, y, w, h, M) - loss_of(oracle_mod, d, params, dn, y, w, h, M)) / (
            float(up[i, c]) - float(dn[i, c]))
        assert abs(num - ge[i, c]) <= 1e-4 * abs(ge[i, c]) + 1e-9, (i, c, num, ge[i, c])


def test_mc_rounding_scale_bounds_the_gradient(oracle_mod, small):
    """The M-channel rounding scale bounds every gradient entry (each pair
    term is bounded by its operand-magnitude evaluation)."""
    d = small
    h = 6
    for M in (2, 3):
        params = synth.gate_parameters_mc(h, M, seed=6)
        dL = np.random.default_rng(6).standard_normal(d["C"].shape[0])
        args = (d["C"], d["sw"], d["self"], d["rep"].lens, d["emb"], d["sig"], params, h, M, dL)
        gp, ge = oracle_mod.fuse_backward_mc(*args)
        sc, se = oracle_mod.fuse_backward_mc_scale(*args)
        assert (np.abs(gp) <= sc * (1 + 1e-12)).all() and (np.abs(ge) <= se * (1 + 1e-12) + 1e-300).all()
