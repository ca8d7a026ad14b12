"""GPU parity of the graph step (components, RMT threshold scan, pruning) and
of the cluster-mass Jensen-Shannon repertoire distance against the oracle.
Components, level counts, component sizes, the chosen threshold and the
pruned graph are exact; <r> within 1e-9 (FP64 Jacobi against LAPACK);
distances within 1e-12."""
import math

import numpy as np
import pytest

from oracle import graph as G
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


def dev(torch, ctx, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a).astype(dtype)).to(ctx.device)


def to_np(t):
    return t.detach().cpu().numpy()


def random_graph(rng, n, m):
    i = rng.integers(0, n, m)
    j = rng.integers(0, n, m)
    keep = i < j
    p = np.unique(np.stack([i[keep], j[keep]], 1), axis=0).astype(np.uint32)
    return p, rng.uniform(0, 1, p.shape[0]).astype(np.float32)


@pytest.mark.parametrize("n,m,tau", [(1, 0, 0.5), (50, 10, 0.0), (5000, 4000, 0.3), (100_000, 300_000, 0.7),
                                     (100_000, 300_000, 0.0)])
def test_components_exact(ctx, torch, n, m, tau):
    rng = np.random.default_rng(n + m)
    p, w = random_graph(rng, n, m) if m else (np.zeros((0, 2), np.uint32), np.zeros(0, np.float32))
    lab, sizes = ctx.graph_components(dev(torch, ctx, p.view(np.int32).reshape(-1, 2), np.int32),
                                      dev(torch, ctx, w, np.float32), n, tau, want_sizes=True)
    ctx.check()
    want = G.components(n, p, w.astype(np.float64), tau)
    assert (to_np(lab).astype(np.int64) == want).all()
    assert (to_np(sizes)[want] == np.bincount(want, minlength=n)[want]).all()


def check_scan(ctx, torch, n, p, w, taus, s_max=64):
    res = ctx.rmt_threshold(dev(torch, ctx, p.view(np.int32).reshape(-1, 2), np.int32), dev(torch, ctx, w, np.float32),
                            n, taus, s_max)
    want_tau, stats = G.rmt_threshold(n, p, w.astype(np.float64), taus, s_max)
    assert res["tau_star"] == want_tau
    for t, st in enumerate(stats):
        assert res["max_comp"][t] == st["max_comp"], t
        if st["evaluable"]:
            assert res["num_levels"][t] == st["levels"].size
            assert res["num_ratios"][t] == st["n_r"]
            if st["n_r"]:
                assert abs(res["r_mean"][t] - st["r_mean"]) <= 1e-9, (t, res["r_mean"][t], st["r_mean"])
        else:
            assert math.isnan(res["r_mean"][t])
    for t in range(len(stats), len(taus)):  # not reached
        assert res["max_comp"][t] == -1
    return res


def test_rmt_threshold_planted(ctx, torch):
    import test_oracle_graph as T

    rng = np.random.default_rng(4)
    n, p, w = T.planted(rng)
    taus = np.round(np.arange(0.30, 0.91, 0.05), 2)
    res = check_scan(ctx, torch, n, p.astype(np.uint32), w.astype(np.float32), taus)
    assert 0.45 <= res["tau_star"] <= 0.6


def test_rmt_threshold_on_fused_donor_graph(ctx, torch, oracle_mod):
    """A 100,000-sequence donor's candidate graph weighted by the oracle's
    fused scores (rounded to float32, the dtype the fusion writes): the full
    scan, then G."""
    rep = synth.donor_repertoire(100_000, seed=3)
    a, b = synth.hash_coefficients(64, seed=3)
    sig = oracle_mod.sign_mt(rep.codes, rep.lens, 3, a, b, 16)
    C = oracle_mod.candidates(sig, 16, 4, 2048)
    sw = oracle_mod.sw_pairs_mt(rep.codes, rep.lens, C, 16)
    self_sc = oracle_mod.self_scores(rep.codes, rep.lens)
    emb = synth.unit_embeddings(rep.n, 64, seed=3)
    fused = oracle_mod.fuse_forward_mt(C, sw, self_sc, rep.lens, emb, synth.gate_parameters(16, seed=0), 16, 16)
    w = fused.astype(np.float32)
    taus = np.round(np.arange(0.40, 0.91, 0.02), 2)
    res = check_scan(ctx, torch, rep.n, C, w, taus)
    gp, gw = ctx.graph_prune(dev(torch, ctx, C.view(np.int32), np.int32), dev(torch, ctx, w, np.float32),
                             res["tau_star"])
    wp, ww = G.prune(C, w, res["tau_star"])
    assert (to_np(gp).view(np.uint32) == wp).all() and (to_np(gw) == ww).all()


def test_prune_edge_cases(ctx, torch):
    rng = np.random.default_rng(7)
    p, w = random_graph(rng, 1000, 3000)
    for tau in (-1.0, 0.5, 2.0):
        gp, gw = ctx.graph_prune(dev(torch, ctx, p.view(np.int32), np.int32), dev(torch, ctx, w, np.float32), tau)
        wp, ww = G.prune(p, w, tau)
        assert gp.shape[0] == wp.shape[0] and (to_np(gp).view(np.uint32) == wp).all() and (to_np(gw) == ww).all()


@pytest.mark.parametrize("n,D,K", [(1000, 3, 50), (200_000, 64, 20_000), (50_000, 7, 10)])
def test_cluster_js_matches_oracle(ctx, torch, n, D, K):
    rng = np.random.default_rng(n + D)
    labels = rng.integers(0, K, n).astype(np.uint32) * 7 + 3  # arbitrary label ids
    donor = rng.integers(0, D, n).astype(np.int32)
    got = to_np(ctx.cluster_js(dev(torch, ctx, labels.view(np.int32), np.int32), dev(torch, ctx, donor, np.int32), D))
    ctx.check()
    want = G.js_distance_matrix(labels.astype(np.int64), donor, D)
    assert np.allclose(got, want, rtol=0, atol=1e-12), np.abs(got - want).max()


def test_cluster_js_empty_donor_and_disjoint(ctx, torch):
    labels = np.array([0, 0, 1, 1, 2, 2], np.uint32)
    donor = np.array([0, 0, 0, 0, 2, 2], np.int32)  # donor 1 has no sequences
    got = to_np(ctx.cluster_js(dev(torch, ctx, labels.view(np.int32), np.int32), dev(torch, ctx, donor, np.int32), 3))
    assert np.isnan(got[1]).all() and np.isnan(got[:, 1]).all()
    assert abs(got[0, 2] - math.sqrt(math.log(2))) < 1e-15 and got[0, 0] == 0.0
