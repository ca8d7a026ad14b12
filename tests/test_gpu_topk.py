"""GPU parity for cross-donor retrieval: top-k from the candidate graph and
the exhaustive top-k, both bit-exact (ids and scores) against the oracle."""
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
def pooled(ctx, torch, oracle_mod):
    """Pooled donors with the oracle's candidate list and scores (the inputs
    of the retrieval step), uploaded for the GPU."""
    rep = synth.pooled_repertoire(8, 300, 3000, n_public=40, public_lo=0.3, public_hi=0.6, seed=3)
    a, b = synth.hash_coefficients(64, seed=3)
    packed = ctx.pack(torch.from_numpy(rep.codes), torch.from_numpy(rep.lens), 16)
    pairs_o = oracle_mod.candidates(oracle_mod.sign(rep.codes, rep.lens, 3, a, b), 16, 4, 0)
    scores_o = oracle_mod.sw_pairs(rep.codes, rep.lens, pairs_o)
    pairs = torch.from_numpy(pairs_o.view(np.int32)).to(ctx.device)
    scores = torch.from_numpy(scores_o).to(ctx.device)
    return dict(rep=rep, packed=packed, pairs=pairs, scores=scores, pairs_o=pairs_o, scores_o=scores_o)


@pytest.mark.parametrize("k", [1, 5, 50, 200])
def test_topk_candidates_against_oracle(ctx, torch, oracle_mod, pooled, k):
    rep = pooled["rep"]
    queries = synth.sample_queries(rep.n, 700, seed=k)
    ids, sc = ctx.topk_candidates(pooled["pairs"], pooled["scores"], rep.n, torch.from_numpy(rep.donor),
                                  torch.from_numpy(queries.view(np.int32)), k)
    ctx.check()
    want_ids, want_sc = oracle_mod.topk(pooled["pairs_o"], pooled["scores_o"], rep.donor, queries, k)
    assert (to_np(ids).view(np.uint32) == want_ids).all()
    assert (to_np(sc) == want_sc).all()
    assert (want_sc[:, 0] >= 0).mean() > 0.1  # a good share of queries have cross-donor candidates


def test_topk_bruteforce_against_oracle(ctx, torch, oracle_mod):
    rep = synth.pooled_repertoire(4, 200, 500, n_public=20, public_lo=5e-2, public_hi=2e-1, seed=5)
    packed = ctx.pack(torch.from_numpy(rep.codes), torch.from_numpy(rep.lens), 16)
    iu, ju = np.triu_indices(rep.n, 1)
    all_pairs = np.stack([iu, ju], 1).astype(np.uint32)
    all_scores = oracle_mod.sw_pairs(rep.codes, rep.lens, all_pairs)
    queries = synth.sample_queries(rep.n, 300, seed=5)
    for k in (3, 50):
        ids, sc = ctx.topk_bruteforce(packed, torch.from_numpy(rep.donor), torch.from_numpy(queries.view(np.int32)),
                                      k)
        want_ids, want_sc = oracle_mod.topk(all_pairs, all_scores, rep.donor, queries, k)
        assert (to_np(ids).view(np.uint32) == want_ids).all()
        assert (to_np(sc) == want_sc).all()


def test_bruteforce_dominates_candidates(ctx, torch, pooled):
    """Every score the candidate route retrieves at rank r is at most the
    exhaustive score at rank r (the candidate set is a subset)."""
    rep = pooled["rep"]
    queries = synth.sample_queries(rep.n, 400, seed=9)
    q = torch.from_numpy(queries.view(np.int32))
    _, sc_c = ctx.topk_candidates(pooled["pairs"], pooled["scores"], rep.n, torch.from_numpy(rep.donor), q, 20)
    _, sc_b = ctx.topk_bruteforce(pooled["packed"], torch.from_numpy(rep.donor), q, 20)
    assert (to_np(sc_c) <= to_np(sc_b)).all()
