"""Recall of the candidate set on the 1,000-sequence workload (seed 0: 100
families, 3-mers, 64 hashes in 16 bands of 4, no cap) against brute force.

T = {i < j : s_ij >= 0.7}, s_ij = S_ij / sqrt(S_ii S_jj) from the affine-gap
local alignment of ALL 499,500 pairs (tau = 0.7 is the paper's fused-score
threshold of its parameter study).  Reported: |C n T| / |T| and the recall of
same-family pairs.  The value is then explained independently: for a pair
with exact k-mer Jaccard J, banding with B bands of R rows makes it a
candidate with probability 1 - (1 - J^R)^B (over the draw of the min-wise
hash family); averaged over 20 hash draws, |C n T| must agree with that sum
within four standard errors plus the min-wise implementation bias (the
appendix's sampling-error bound allows an eps_impl; 0.02 per pair here).
"""
import numpy as np
import pytest

from paper_2602_17330_gb300 import synth

TAU = 0.7
K, BANDS, ROWS = 3, 16, 4


@pytest.fixture(scope="module")
def tiny(oracle_mod):
    rep = synth.tiny_repertoire(seed=0)
    n = rep.n
    iu, ju = np.triu_indices(n, 1)
    allp = np.stack([iu, ju], 1).astype(np.uint32)
    S = oracle_mod.sw_pairs(rep.codes, rep.lens, allp)
    self_sc = oracle_mod.self_scores(rep.codes, rep.lens)
    s = S / np.sqrt(self_sc[iu].astype(np.float64) * self_sc[ju])
    return dict(rep=rep, n=n, iu=iu, ju=ju, s=s, key=iu.astype(np.int64) * n + ju)


def candidate_keys(oracle_mod, rep, seed):
    a, b = synth.hash_coefficients(BANDS * ROWS, seed=seed)
    C = oracle_mod.candidates(oracle_mod.sign(rep.codes, rep.lens, K, a, b), BANDS, ROWS, 0)
    return C, C[:, 0].astype(np.int64) * rep.n + C[:, 1]


def test_recall_against_all_pairs(oracle_mod, tiny):
    rep, n = tiny["rep"], tiny["n"]
    C, ckey = candidate_keys(oracle_mod, rep, 0)
    # C is a set of distinct pairs i < j < n, so it is a subset of all pairs
    assert (C[:, 0] < C[:, 1]).all() and (C[:, 1] < n).all() and np.unique(ckey).size == ckey.size
    in_c = np.isin(tiny["key"], ckey)
    T = tiny["s"] >= TAU
    fam = (rep.family[tiny["iu"]] >= 0) & (rep.family[tiny["iu"]] == rep.family[tiny["ju"]])
    recall = (in_c & T).sum() / T.sum()
    fam_recall = (in_c & fam).sum() / fam.sum()
    assert np.isfinite(recall) and 0.0 <= recall <= 1.0 and 0.0 <= fam_recall <= 1.0
    assert T.sum() > 0 and fam.sum() == 1000
    print(f"\n|C| = {C.shape[0]}, |T| = {T.sum()}, |C n T| = {(in_c & T).sum()}, recall = {recall:.4f}; "
          f"same-family pairs {fam.sum()}, recall {fam_recall:.4f}")


def test_recall_follows_banding_s_curve(oracle_mod, tiny):
    rep = tiny["rep"]
    Tq = np.flatnonzero(tiny["s"] >= TAU)

    def kmer_set(r):
        c = rep.codes[r]
        return {tuple(c[p:p + K]) for p in range(int(rep.lens[r]) - K + 1)}

    sets = {}
    for r in np.unique(np.concatenate([tiny["iu"][Tq], tiny["ju"][Tq]])):
        sets[int(r)] = kmer_set(int(r))
    J = np.array([len(sets[int(tiny["iu"][q])] & sets[int(tiny["ju"][q])]) /
                  len(sets[int(tiny["iu"][q])] | sets[int(tiny["ju"][q])]) for q in Tq])
    P = 1.0 - (1.0 - J ** ROWS) ** BANDS
    expected = P.sum()
    hits = []
    for seed in range(1001, 1021):
        _, ckey = candidate_keys(oracle_mod, rep, seed)
        hits.append(int(np.isin(tiny["key"][Tq], ckey).sum()))
    hits = np.array(hits, dtype=np.float64)
    sem = np.sqrt((P * (1 - P)).sum()) / np.sqrt(hits.size)
    bias = 0.02 * Tq.size * ROWS * BANDS * np.mean(J ** (ROWS - 1))  # eps_impl on each row collision
    assert abs(hits.mean() - expected) <= 4 * sem + bias, (hits.mean(), expected, sem, bias)
