"""Pins for the oracle's alignment channel (affine-gap local alignment with
BLOSUM62) against values and routines that do not come from the oracle."""
import difflib
import itertools
import os

import numpy as np
import pytest

from paper_2602_17330_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sw_hand_worked.txt")


def codes_of(s):
    return np.array([synth.ALPHABET.index(c) for c in s], dtype=np.uint8)


# --- BLOSUM62 ---------------------------------------------------------------

def test_blosum62_shape_symmetry_and_diagonal(oracle_mod):
    M = oracle_mod.blosum62()
    assert M.shape == (20, 20)
    assert (M == M.T).all()
    for a in range(20):
        row = M[a].copy()
        assert row[a] > 0
        row[a] = -1000
        assert M[a, a] > row.max(), "diagonal must be the strict row maximum"


@pytest.mark.parametrize("x,y,v", [("W", "W", 11), ("C", "C", 9), ("A", "A", 4), ("H", "H", 8),
                                   ("P", "P", 7), ("Y", "Y", 7), ("G", "G", 6), ("I", "V", 3),
                                   ("W", "G", -2), ("D", "E", 2), ("F", "Y", 3), ("K", "R", 2),
                                   ("W", "D", -4), ("C", "E", -4), ("L", "I", 2), ("S", "T", 1)])
def test_blosum62_spot_entries(oracle_mod, x, y, v):
    M = oracle_mod.blosum62()
    a, b = synth.ALPHABET.index(x), synth.ALPHABET.index(y)
    assert M[a, b] == v and M[b, a] == v


# --- hand-worked alignments ---------------------------------------------------

def golden_cases():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            a, b, o, e, score, alt = line.split()[:6]
            rows.append((a, b, int(o), int(e), int(score), int(alt)))
    return rows


@pytest.mark.parametrize("a,b,o,e,score,alt", golden_cases())
def test_hand_worked_alignments(oracle_mod, a, b, o, e, score, alt):
    assert oracle_mod.sw(codes_of(a), codes_of(b), o, e) == score


# --- exhaustive enumeration of local alignments --------------------------------

def brute_force_local(a, b, M, o, e):
    """Max over every local alignment path (start cell, then any sequence of
    match / gap-in-a / gap-in-b columns), each maximal gap run of length l
    costing o + (l-1) e; the empty alignment scores 0."""
    la, lb = len(a), len(b)
    best = 0

    def walk(i, j, last, run, score):
        nonlocal best
        best = max(best, score)
        if i < la and j < lb:
            walk(i + 1, j + 1, "M", 0, score + M[a[i], b[j]])
        if j < lb:  # b_j against a gap
            cost = e if last == "I" else o
            walk(i, j + 1, "I", run + 1 if last == "I" else 1, score - cost)
        if i < la:  # a_i against a gap
            cost = e if last == "D" else o
            walk(i + 1, j, "D", run + 1 if last == "D" else 1, score - cost)

    for i0 in range(la + 1):
        for j0 in range(lb + 1):
            walk(i0, j0, "S", 0, 0)
    return best


def test_enumeration_matches_on_random_short_strings(oracle_mod):
    rng = np.random.default_rng(7)
    for trial in range(60):
        la, lb = rng.integers(1, 6), rng.integers(1, 6)
        a = rng.integers(0, 20, la).astype(np.uint8)
        b = rng.integers(0, 20, lb).astype(np.uint8)
        # a random small integer matrix (not symmetric) and small gap costs,
        # so that gapped alignments often win
        M = rng.integers(-3, 8, (20, 20)).astype(np.int32)
        o = int(rng.integers(0, 6))
        e = int(rng.integers(0, 4))
        assert oracle_mod.sw(a, b, o, e, M) == brute_force_local(a, b, M, o, e), (trial, a, b, o, e)


def test_enumeration_matches_with_blosum(oracle_mod):
    rng = np.random.default_rng(11)
    M = oracle_mod.blosum62()
    for trial in range(30):
        la, lb = rng.integers(2, 6), rng.integers(2, 6)
        a = rng.integers(0, 20, la).astype(np.uint8)
        b = rng.integers(0, 20, lb).astype(np.uint8)
        o, e = (10, 1) if trial % 2 == 0 else (2, 1)
        assert oracle_mod.sw(a, b, o, e) == brute_force_local(a, b, M, o, e)


# --- textbook reductions ------------------------------------------------------

def kadane_diagonals(a, b, M):
    """Ungapped local alignment: best maximum-subarray sum over every diagonal."""
    best = 0
    for off in range(-len(a) + 1, len(b)):
        run = 0
        for i in range(len(a)):
            j = i + off
            if 0 <= j < len(b):
                run = max(0, run + int(M[a[i], b[j]]))
                best = max(best, run)
    return best


def test_infinite_gap_cost_reduces_to_kadane(oracle_mod):
    rng = np.random.default_rng(3)
    M = oracle_mod.blosum62()
    for _ in range(40):
        a = rng.integers(0, 20, rng.integers(5, 25)).astype(np.uint8)
        b = rng.integers(0, 20, rng.integers(5, 25)).astype(np.uint8)
        assert oracle_mod.sw(a, b, 1_000_000, 1_000_000) == kadane_diagonals(a, b, M)


def test_identity_matrix_reduces_to_longest_common_substring(oracle_mod):
    rng = np.random.default_rng(5)
    ident = np.full((20, 20), -1000, dtype=np.int32)
    np.fill_diagonal(ident, 1)
    for _ in range(40):
        a = rng.integers(0, 4, rng.integers(3, 30)).astype(np.uint8)
        b = rng.integers(0, 4, rng.integers(3, 30)).astype(np.uint8)
        sa = "".join(synth.ALPHABET[x] for x in a)
        sb = "".join(synth.ALPHABET[x] for x in b)
        lcs = difflib.SequenceMatcher(None, sa, sb, autojunk=False).find_longest_match(0, len(sa), 0, len(sb)).size
        assert oracle_mod.sw(a, b, 1000, 1000, ident) == lcs


# --- invariants ---------------------------------------------------------------

def test_self_score_is_diagonal_sum_and_bounds(oracle_mod):
    rep = synth.tiny_repertoire()
    M = oracle_mod.blosum62()
    self_sc = oracle_mod.self_scores(rep.codes, rep.lens)
    for i in range(0, rep.n, 37):
        L = rep.lens[i]
        assert self_sc[i] == int(sum(M[c, c] for c in rep.codes[i, :L]))
    rng = np.random.default_rng(1)
    pairs = rng.integers(0, rep.n, (400, 2)).astype(np.uint32)
    s_ij = oracle_mod.sw_pairs(rep.codes, rep.lens, pairs)
    s_ji = oracle_mod.sw_pairs(rep.codes, rep.lens, pairs[:, ::-1])
    assert (s_ij == s_ji).all()
    assert (s_ij >= 0).all()
    assert (s_ij <= np.minimum(self_sc[pairs[:, 0]], self_sc[pairs[:, 1]])).all()


def test_self_score_shortcut_condition(oracle_mod):
    """The library scores a sequence against itself as the sum of its diagonal
    entries when every diagonal entry is positive and 2 M(a,b) <= M(a,a) +
    M(b,b) (then no alignment beats the ungapped identity alignment).
    BLOSUM62 satisfies it; a matrix that breaks it has self-scores above the
    diagonal sum, computed here by the full dynamic programme."""
    M = oracle_mod.blosum62().astype(np.int64)
    d = np.diag(M)
    assert (d > 0).all() and (2 * M <= d[:, None] + d[None, :]).all()
    bad = np.full((20, 20), -4, dtype=np.int32)
    np.fill_diagonal(bad, 1)
    bad[0, 1] = bad[1, 0] = 10  # A-C far above the diagonal
    codes = np.zeros((1, 32), dtype=np.uint8)
    codes[0, :6] = [0, 1, 0, 1, 0, 1]  # ACACAC
    lens = np.array([6], dtype=np.uint8)
    sc = oracle_mod.self_scores(codes, lens, 10, 1, bad)
    assert sc[0] > 6  # the shifted alignment A-C, C-A, ... wins
