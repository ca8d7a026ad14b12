"""Pins for the oracle's edit distance (the GPU appendix's edit-distance
recurrence): hand-worked values, brute-force enumeration of every alignment
path on short strings, the Hamming and LCS reductions, metric axioms, and the
default biochemical substitution costs."""
import itertools
import os

import numpy as np
import pytest

from paper_2602_17330_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
ALPHA = synth.ALPHABET


def enc(s):
    return np.array([ALPHA.index(ch) for ch in s], dtype=np.uint8)


UNIT = (np.ones((20, 20), np.uint8) - np.eye(20, dtype=np.uint8))


def golden():
    rows = []
    for line in open(os.path.join(HERE, "golden", "edit_hand_worked.txt")):
        if line.strip() and not line.startswith("#"):
            a, b, u, d = line.split()
            rows.append((a, b, int(u), int(d)))
    return rows


@pytest.mark.parametrize("a,b,unit,default", golden())
def test_hand_worked(oracle_mod, a, b, unit, default):
    assert oracle_mod.edit(enc(a), enc(b), 1, UNIT) == unit
    assert oracle_mod.edit(enc(a), enc(b)) == default


def brute_force(a, b, indel, sub):
    """Minimum cost over every monotone alignment path (match/substitute,
    delete, insert), enumerated recursively without memoisation."""
    def go(x, y):
        if x == len(a) and y == len(b):
            return 0
        best = 1 << 30
        if x < len(a):
            best = min(best, indel + go(x + 1, y))
        if y < len(b):
            best = min(best, indel + go(x, y + 1))
        if x < len(a) and y < len(b):
            c = 0 if a[x] == b[y] else int(sub[a[x], b[y]])
            best = min(best, c + go(x + 1, y + 1))
        return best
    return go(0, 0)


def test_brute_force_on_short_strings(oracle_mod):
    rng = np.random.default_rng(0)
    for _ in range(300):
        a = rng.integers(0, 4, rng.integers(0, 6)).astype(np.uint8)
        b = rng.integers(0, 4, rng.integers(0, 6)).astype(np.uint8)
        indel = int(rng.integers(0, 5))
        sub = rng.integers(0, 9, (20, 20)).astype(np.uint8)
        assert oracle_mod.edit(a, b, indel, sub) == brute_force(a, b, indel, sub)


def test_prohibitive_indels_give_hamming(oracle_mod):
    rng = np.random.default_rng(1)
    sub = oracle_mod.default_edit_costs()
    for L in range(1, 25):
        a = rng.integers(0, 20, L).astype(np.uint8)
        b = rng.integers(0, 20, L).astype(np.uint8)
        want = int(sum(0 if x == y else sub[x, y] for x, y in zip(a, b)))
        assert oracle_mod.edit(a, b, 255, sub) == want


def lcs_brute(a, b):
    best = 0
    for r in range(len(a), 0, -1):
        subs = {tuple(c) for c in itertools.combinations(a, r)}
        if any(tuple(c) in subs for c in itertools.combinations(b, r)):
            return r
    return best


def test_prohibitive_substitutions_give_lcs(oracle_mod):
    rng = np.random.default_rng(2)
    sub = np.full((20, 20), 200, np.uint8)
    for _ in range(100):
        a = rng.integers(0, 5, rng.integers(0, 8)).astype(np.uint8)
        b = rng.integers(0, 5, rng.integers(0, 8)).astype(np.uint8)
        assert oracle_mod.edit(a, b, 3, sub) == 3 * (len(a) + len(b) - 2 * lcs_brute(list(a), list(b)))


def test_metric_axioms_unit_costs(oracle_mod):
    rng = np.random.default_rng(3)
    seqs = [rng.integers(0, 20, rng.integers(1, 16)).astype(np.uint8) for _ in range(40)]
    d = np.array([[oracle_mod.edit(x, y, 1, UNIT) for y in seqs] for x in seqs])
    assert (d == d.T).all() and (np.diag(d) == 0).all()
    assert (d[~np.eye(len(seqs), dtype=bool)] > 0).all() or any(
        (x.shape == y.shape and (x == y).all()) for x, y in itertools.combinations(seqs, 2))
    # d(a, c) <= d(a, b) + d(b, c), indexed [a, b, c]
    assert (d[:, None, :] <= d[:, :, None] + d[None, :, :]).all()


def test_default_costs(oracle_mod):
    S = oracle_mod.default_edit_costs()
    M = oracle_mod.blosum62()
    assert (S == S.T).all() and (np.diag(S) == 0).all()
    off = ~np.eye(20, dtype=bool)
    assert set(np.unique(S[off]).tolist()) == {1, 2}
    assert ((S[off] == 1) == (M[off] > 0)).all()
    assert S[ALPHA.index("I"), ALPHA.index("V")] == 1 and S[ALPHA.index("W"), ALPHA.index("A")] == 2
