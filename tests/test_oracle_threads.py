"""The oracle's multi-threaded runners (the CPU baseline over all host cores)
split index ranges over threads and call the single-threaded routines, so
their results must equal the single-threaded calls exactly."""
import numpy as np
import pytest

from paper_2602_17330_gb300 import synth


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_threaded_runners_equal_single_thread(oracle_mod, threads):
    rep = synth.donor_repertoire(6_000, seed=3)
    a, b = synth.hash_coefficients(64, seed=3)
    sig = oracle_mod.sign(rep.codes, rep.lens, 3, a, b)
    assert (oracle_mod.sign_mt(rep.codes, rep.lens, 3, a, b, threads) == sig).all()
    C = oracle_mod.candidates(sig, 16, 4, 2048)
    assert np.array_equal(oracle_mod.candidates_mt(sig, 16, 4, 2048, threads), C)
    # a cap that splits buckets, no cap, and bands of other shapes
    for bands, rows, cap in ((16, 4, 3), (32, 2, 0), (5, 3, 0)):
        assert np.array_equal(oracle_mod.candidates_mt(sig, bands, rows, cap, threads),
                              oracle_mod.candidates(sig, bands, rows, cap))
    sw = oracle_mod.sw_pairs(rep.codes, rep.lens, C)
    assert (oracle_mod.sw_pairs_mt(rep.codes, rep.lens, C, threads) == sw).all()
    self_sc = oracle_mod.self_scores(rep.codes, rep.lens)
    emb = synth.unit_embeddings(rep.n, 64, seed=3)
    params = synth.gate_parameters(16, seed=3)
    want = oracle_mod.fuse_forward(C, sw, self_sc, rep.lens, emb, params, 16)["fused"]
    assert (oracle_mod.fuse_forward_mt(C, sw, self_sc, rep.lens, emb, params, 16, threads) == want).all()
    # fewer items than threads
    few = C[:2]
    assert (oracle_mod.sw_pairs_mt(rep.codes, rep.lens, few, threads) == sw[:2]).all()


def test_threaded_parameter_gradient(oracle_mod):
    rep = synth.donor_repertoire(6_000, seed=4)
    a, b = synth.hash_coefficients(64, seed=4)
    C = oracle_mod.candidates(oracle_mod.sign(rep.codes, rep.lens, 3, a, b), 16, 4, 2048)
    sw = oracle_mod.sw_pairs(rep.codes, rep.lens, C)
    self_sc = oracle_mod.self_scores(rep.codes, rep.lens)
    emb = synth.family_embeddings(rep.family, 32, seed=4)
    params = synth.gate_parameters(8, seed=4)
    dL = np.random.default_rng(4).standard_normal(C.shape[0])
    want, _ = oracle_mod.fuse_backward(C, sw, self_sc, rep.lens, emb, params, 8, dL, with_emb=False)
    for threads in (1, 5):
        got = oracle_mod.fuse_backward_params_mt(C, sw, self_sc, rep.lens, emb, params, 8, dL, threads)
        assert np.allclose(got, want, rtol=1e-12, atol=1e-15)
