"""Pins for the oracle's MinHash signatures and LSH candidate list."""
import itertools
import math

import numpy as np
import pytest

from paper_2602_17330_gb300 import synth

P31 = (1 << 31) - 1


def enc(s):
    codes, lens = synth.encode([s] if isinstance(s, str) else s)
    return codes, lens


# --- k-mer code and hash --------------------------------------------------------

@pytest.mark.parametrize("kmer,value", [("CAS", 415), ("AAA", 0), ("YYY", 7999), ("WYV", 7597), ("ACD", 22)])
def test_kmer_code_hand_values(oracle_mod, kmer, value):
    # base-20 with the first residue most significant; worked by hand from the
    # code order ACDEFGHIKLMNPQRSTVWY (A=0, C=1, D=2, S=15, V=17, W=18, Y=19)
    codes, lens = enc(kmer)
    assert oracle_mod.kmer_code(codes[0], 3) == value
    one = np.array([1], dtype=np.uint32)
    zero = np.array([0], dtype=np.uint32)
    assert oracle_mod.sign(codes, lens, 3, one, zero)[0, 0] == value


def test_hash_is_exact_modular_arithmetic_at_extremes(oracle_mod):
    # a, b near 2^31 make a*x + b exceed 2^44: compare with Python integers
    codes, lens = enc("YYYWYVCAS")
    a = np.array([P31 - 1, P31 - 2, 1 << 30, 123456789], dtype=np.uint32)
    b = np.array([P31 - 1, 0, P31 - 2, 987654321], dtype=np.uint32)
    sig = oracle_mod.sign(codes, lens, 3, a, b)[0]
    s = "YYYWYVCAS"
    xs = []
    for p in range(len(s) - 2):
        x = 0
        for ch in s[p:p + 3]:
            x = x * 20 + synth.ALPHABET.index(ch)
        xs.append(x)
    for t in range(4):
        assert int(sig[t]) == min((int(a[t]) * x + int(b[t])) % P31 for x in xs)


def test_signature_of_union_is_min_of_parts(oracle_mod):
    # the k-mer set of s is the union of the k-mer sets of two overlapping
    # pieces, so the signature must be the elementwise min of theirs
    rep = synth.tiny_repertoire()
    a, b = synth.hash_coefficients(64, seed=3)
    k = 3
    for i in range(0, 200, 7):
        s = rep.strings([i])[0]
        cut = len(s) // 2
        left, right = s[: cut + k - 1], s[cut:]
        codes, lens = enc([s, left, right])
        sig = oracle_mod.sign(codes, lens, k, a, b)
        assert (sig[0] == np.minimum(sig[1], sig[2])).all()


def test_minhash_collision_rate_tracks_jaccard(oracle_mod):
    # P[sig_t(A) = sig_t(B)] ~ J(A, B); the appendix bounds the estimate's error
    # by 1/sqrt(M) + eps_impl.  Over T = 10,000 seeded hash draws the empirical
    # rate must lie within 4 binomial standard errors plus eps_impl = 0.02 (the
    # linear family is not exactly min-wise independent).
    rng = np.random.default_rng(0)
    T = 10_000
    a = rng.integers(1, P31, T, dtype=np.int64).astype(np.uint32)
    b = rng.integers(0, P31, T, dtype=np.int64).astype(np.uint32)
    pairs = [("CASSLGQGAYEQYF", "CASSLGQGAYEQYF"),
             ("CASSLGQGAYEQYF", "CASSLGRGAYEQYF"),
             ("CASSLGQGAYEQYF", "CASSPGQGTYEQYF"),
             ("CASSLGQGAYEQYF", "CASRDWNTEAFF"),
             ("CAWSVGQGNTIYF", "CAWSVGQGNTLYF"),
             ("CASSQDRGHEQFF", "CSARDRTGNGYTF")]
    worst_bias = 0.0
    for s, t in pairs:
        ks = {s[p:p + 3] for p in range(len(s) - 2)}
        kt = {t[p:p + 3] for p in range(len(t) - 2)}
        J = len(ks & kt) / len(ks | kt)
        codes, lens = enc([s, t])
        sig = oracle_mod.sign(codes, lens, 3, a, b)
        rate = float((sig[0] == sig[1]).mean())
        tol = 4.0 * math.sqrt(J * (1.0 - J) / T) + 0.02
        worst_bias = max(worst_bias, abs(rate - J))
        assert abs(rate - J) <= tol, (s, t, J, rate)
    assert worst_bias < 0.05


# --- banding and candidate emission ----------------------------------------------

def brute_force_candidates(sig, bands, rows, cap):
    """Definition written pairwise: i < j is a candidate iff some band gives
    them equal R-tuples and equal chunk index, the chunk index of a member being
    (number of bucket members with smaller id) // cap."""
    n = sig.shape[0]
    out = set()
    for b in range(bands):
        keys = [tuple(int(v) for v in sig[i, b * rows:(b + 1) * rows]) for i in range(n)]
        rank = [sum(1 for u in range(i) if keys[u] == keys[i]) for i in range(n)]
        for i in range(n):
            for j in range(i + 1, n):
                if keys[i] == keys[j]:
                    if cap <= 0 or rank[i] // cap == rank[j] // cap:
                        out.add((i, j))
    return sorted(out)


@pytest.mark.parametrize("cap", [0, 1, 2, 3, 5])
def test_candidates_match_pairwise_definition_planted_buckets(oracle_mod, cap):
    rng = np.random.default_rng(cap + 10)
    n, bands, rows = 60, 5, 3
    # few distinct values, so buckets of many sizes appear in every band
    sig = rng.integers(0, 3, (n, bands * rows)).astype(np.uint32)
    sig[:, ::2] += np.uint32(P31 - 5)  # exercise values near 2^31
    got = oracle_mod.candidates(sig, bands, rows, cap)
    want = brute_force_candidates(sig, bands, rows, cap)
    assert [tuple(map(int, p)) for p in got] == want


def test_candidates_match_pairwise_definition_real_signatures(oracle_mod):
    rep = synth.make_repertoire(150, 15, seed=4)
    a, b = synth.hash_coefficients(16, seed=4)
    sig = oracle_mod.sign(rep.codes, rep.lens, 3, a, b)
    for bands, rows, cap in [(8, 2, 0), (4, 4, 0), (16, 1, 3)]:
        got = oracle_mod.candidates(sig, bands, rows, cap)
        want = brute_force_candidates(sig, bands, rows, cap)
        assert [tuple(map(int, p)) for p in got] == want
        assert len(want) > 0


def test_candidates_sorted_unique_and_ordered(oracle_mod):
    rep = synth.tiny_repertoire()
    a, b = synth.hash_coefficients(64)
    sig = oracle_mod.sign(rep.codes, rep.lens, 3, a, b)
    C = oracle_mod.candidates(sig, 16, 4, 0)
    assert (C[:, 0] < C[:, 1]).all()
    key = C[:, 0].astype(np.int64) * rep.n + C[:, 1]
    assert (np.diff(key) > 0).all()
