"""Seeded synthetic repertoires and random draws for the affinity stage.

This module is the one piece shared by the CUDA path, the oracle, the tests and
the benchmark.  It holds none of the method's arithmetic: it only draws random
CDR3-like sequences, family/subgroup labels, hash coefficients, embeddings and
gate parameters, and returns them as plain numpy arrays.  Everything the method
computes from them (k-mers, hashes, bands, alignments, the gate) lives in the
library and, independently, in the oracle.

Workload shapes (the paper's data are VDJdb / McPAS-TCR / NEPdb CDR3 beta
repertoires, which these stand in for):

* lengths ~ round(N(15, 2)) clipped to a range, optionally with a heavy tail of
  uniformly drawn longer sequences;
* every sequence starts with C and ends with F (CDR3 junction anchors);
* interior residues are i.i.d. from a seeded Dirichlet(alpha=2) frequency vector
  over the 20 amino acids;
* clonotype families: a seed sequence (not itself emitted) and members made from
  it by 1-3 substitutions at distinct interior positions, each new residue drawn
  from the frequency vector conditioned on differing from the old one;
* background sequences are singletons;
* ids are a seeded permutation, so family members are scattered.

Residue codes follow the alphabetical one-letter order ``ACDEFGHIKLMNPQRSTVWY``
(code 0..19).  Sequences are stored as a ``uint8 [n, CODE_STRIDE]`` matrix whose
positions past the length hold ``PAD``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

ALPHABET = "ACDEFGHIKLMNPQRSTVWY"
CODE_C = ALPHABET.index("C")
CODE_F = ALPHABET.index("F")
CODE_STRIDE = 32
PAD = 31
MERSENNE31 = (1 << 31) - 1

# independent random streams per component, so that changing one draw does not
# shift the others
_STREAM = {"freq": 1, "background": 2, "families": 3, "members": 4, "shuffle": 5,
           "subgroups": 6, "hash": 7, "emb": 8, "gate": 9, "sizes": 10, "tail": 11,
           "donors": 12, "public": 13, "queries": 14, "sample": 15}


def rng_for(seed: int, stream: str) -> np.random.Generator:
    return np.random.default_rng([int(seed), _STREAM[stream]])


@dataclass
class Repertoire:
    codes: np.ndarray      # uint8 [n, CODE_STRIDE]
    lens: np.ndarray       # uint8 [n]
    family: np.ndarray     # int32 [n], -1 for background singletons
    subgroup: np.ndarray   # int32 [n], 0 = not in a rare subgroup
    freq: np.ndarray       # float64 [20], interior residue frequencies
    donor: np.ndarray | None = field(default=None)   # int32 [n] for pooled donors

    @property
    def n(self) -> int:
        return int(self.lens.shape[0])

    def strings(self, idx=None) -> list[str]:
        rows = range(self.n) if idx is None else idx
        return ["".join(ALPHABET[c] for c in self.codes[r, : self.lens[r]]) for r in rows]


def encode(seqs: list[str]) -> tuple[np.ndarray, np.ndarray]:
    """Letters -> (codes uint8 [n, CODE_STRIDE], lens uint8 [n])."""
    codes = np.full((len(seqs), CODE_STRIDE), PAD, dtype=np.uint8)
    lens = np.zeros(len(seqs), dtype=np.uint8)
    for r, s in enumerate(seqs):
        if len(s) > CODE_STRIDE:
            raise ValueError("sequence longer than CODE_STRIDE")
        codes[r, : len(s)] = [ALPHABET.index(ch) for ch in s]
        lens[r] = len(s)
    return codes, lens


def _draw_residues(rng, freq, shape) -> np.ndarray:
    cdf = np.cumsum(freq)
    u = rng.random(shape)
    return np.minimum(np.searchsorted(cdf, u, side="right"), 19).astype(np.uint8)


def _draw_lengths(rng, count, len_min, len_max, tail_frac, tail_range) -> np.ndarray:
    lens = np.clip(np.rint(15.0 + 2.0 * rng.standard_normal(count)), len_min, len_max)
    if tail_frac > 0.0:
        tail = rng.random(count) < tail_frac
        lens[tail] = rng.integers(tail_range[0], tail_range[1] + 1, int(tail.sum()))
    return lens.astype(np.uint8)


def _draw_sequences(rng, freq, lens) -> np.ndarray:
    count = lens.shape[0]
    codes = _draw_residues(rng, freq, (count, CODE_STRIDE))
    pos = np.arange(CODE_STRIDE)[None, :]
    L = lens.astype(np.int64)[:, None]
    codes[:, 0] = CODE_C
    codes[pos == (L - 1)] = CODE_F
    codes[pos >= L] = PAD
    return codes


def _substitute(rng, freq, codes, lens) -> None:
    """1-3 substitutions at distinct interior positions, in place."""
    m = codes.shape[0]
    if m == 0:
        return
    k = rng.integers(1, 4, m)
    keys = rng.random((m, CODE_STRIDE))
    pos = np.arange(CODE_STRIDE)[None, :]
    L = lens.astype(np.int64)[:, None]
    keys[(pos == 0) | (pos >= L - 1)] = 2.0
    order = np.argsort(keys, axis=1, kind="stable")
    rows = np.arange(m)
    for t in range(3):
        sel = rows[k > t]
        p = order[sel, t]
        old = codes[sel, p]
        new = _draw_residues(rng, freq, sel.shape[0])
        bad = new == old
        while bad.any():
            new[bad] = _draw_residues(rng, freq, int(bad.sum()))
            bad = new == old
        codes[sel, p] = new


def zipf_family_sizes(total: int, s: float, lo: int, hi: int, rng) -> np.ndarray:
    """Family sizes from Zipf(s) truncated to [lo, hi] until they sum to total."""
    support = np.arange(lo, hi + 1, dtype=np.float64)
    pmf = support ** (-s)
    cdf = np.cumsum(pmf / pmf.sum())
    sizes: list[np.ndarray] = []
    acc = 0
    while acc < total:
        draw = np.minimum(np.searchsorted(cdf, rng.random(100_000), side="right"), hi - lo) + lo
        csum = acc + np.cumsum(draw)
        cut = int(np.searchsorted(csum, total, side="left"))
        if cut < draw.shape[0]:
            draw = draw[: cut + 1].copy()
            draw[-1] -= int(csum[cut] - total)
            sizes.append(draw)
            acc = total
        else:
            sizes.append(draw)
            acc = int(csum[-1])
    out = np.concatenate(sizes).astype(np.int64)
    return out[out >= lo] if out[-1] < lo else out


def make_repertoire(n: int, n_families: int = 0, *, seed: int = 0, member_frac: float = 0.5,
                    len_min: int = 8, len_max: int = 24, tail_frac: float = 0.0,
                    tail_range: tuple[int, int] = (25, 30), family_sizes: np.ndarray | None = None,
                    rare_subgroups: int = 0, rare_subgroup_size: int = 0,
                    freq: np.ndarray | None = None) -> Repertoire:
    """One seeded synthetic repertoire of ``n`` CDR3-like sequences."""
    if freq is None:
        freq = rng_for(seed, "freq").dirichlet(np.full(20, 2.0))
    if family_sizes is None:
        members = int(round(member_frac * n)) if n_families > 0 else 0
        family_sizes = np.full(n_families, members // max(n_families, 1), dtype=np.int64)
        family_sizes[: members - int(family_sizes.sum())] += 1
    family_sizes = np.asarray(family_sizes, dtype=np.int64)
    n_members = int(family_sizes.sum())
    if n_members > n:
        raise ValueError("family members exceed n")
    nf = family_sizes.shape[0]

    rf = rng_for(seed, "families")
    seed_lens = _draw_lengths(rf, nf, len_min, len_max, tail_frac, tail_range)
    seed_codes = _draw_sequences(rf, freq, seed_lens)
    fam_of_member = np.repeat(np.arange(nf, dtype=np.int32), family_sizes)
    m_codes = seed_codes[fam_of_member]
    m_lens = seed_lens[fam_of_member]
    _substitute(rng_for(seed, "members"), freq, m_codes, m_lens)

    rb = rng_for(seed, "background")
    nb = n - n_members
    b_lens = _draw_lengths(rb, nb, len_min, len_max, tail_frac, tail_range)
    b_codes = _draw_sequences(rb, freq, b_lens)

    codes = np.concatenate([m_codes, b_codes])
    lens = np.concatenate([m_lens, b_lens])
    family = np.concatenate([fam_of_member, np.full(nb, -1, dtype=np.int32)])
    fam_subgroup = np.zeros(nf, dtype=np.int32)
    if rare_subgroups > 0:
        # rare subgroups are assigned at family level: whole families, in a
        # seeded order, until each subgroup holds rare_subgroup_size sequences
        order = rng_for(seed, "subgroups").permutation(nf)
        fill = np.zeros(rare_subgroups + 1, dtype=np.int64)
        g = 1
        for f in order:
            if g > rare_subgroups:
                break
            fam_subgroup[f] = g
            fill[g] += family_sizes[f]
            if fill[g] >= rare_subgroup_size:
                g += 1
    subgroup = np.concatenate([fam_subgroup[fam_of_member], np.zeros(nb, dtype=np.int32)])

    perm = rng_for(seed, "shuffle").permutation(n)
    return Repertoire(codes=np.ascontiguousarray(codes[perm]), lens=np.ascontiguousarray(lens[perm]),
                      family=np.ascontiguousarray(family[perm]),
                      subgroup=np.ascontiguousarray(subgroup[perm]), freq=freq)


def hash_coefficients(H: int, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """a_t uniform on [1, 2^31-2], b_t uniform on [0, 2^31-2] (uint32)."""
    r = rng_for(seed, "hash")
    a = r.integers(1, MERSENNE31, H, dtype=np.int64).astype(np.uint32)
    b = r.integers(0, MERSENNE31, H, dtype=np.int64).astype(np.uint32)
    return a, b


def unit_embeddings(n: int, d: int, seed: int = 0) -> np.ndarray:
    """i.i.d. Gaussian rows scaled to unit norm (float32 [n, d])."""
    r = rng_for(seed, "emb")
    z = r.standard_normal((n, d), dtype=np.float32)
    z /= np.linalg.norm(z, axis=1, keepdims=True)
    return np.ascontiguousarray(z)


def family_embeddings(family: np.ndarray, d: int, seed: int = 0) -> np.ndarray:
    """normalise(c_family + z): a shared Gaussian centre per family, so the
    cosine channel carries family signal; background rows are normalise(z)."""
    r = rng_for(seed, "emb")
    nf = int(family.max()) + 1 if family.size else 0
    centres = r.standard_normal((max(nf, 1), d), dtype=np.float32)
    z = r.standard_normal((family.shape[0], d), dtype=np.float32)
    fam = family >= 0
    z[fam] += centres[family[fam]]
    z /= np.linalg.norm(z, axis=1, keepdims=True)
    return np.ascontiguousarray(z)


def gate_parameters(hidden: int, seed: int = 0) -> np.ndarray:
    """Flat float32 [W1 (hidden x 3, row-major), b1 (hidden), w2 (hidden), b2],
    each layer uniform on +-1/sqrt(fan_in)."""
    r = rng_for(seed, "gate")
    w1 = r.uniform(-1.0, 1.0, (hidden, 3)) / np.sqrt(3.0)
    b1 = r.uniform(-1.0, 1.0, hidden) / np.sqrt(3.0)
    w2 = r.uniform(-1.0, 1.0, hidden) / np.sqrt(hidden)
    b2 = r.uniform(-1.0, 1.0, 1) / np.sqrt(hidden)
    return np.concatenate([w1.ravel(), b1, w2, b2]).astype(np.float32)


def gate_param_count(hidden: int) -> int:
    return 3 * hidden + hidden + hidden + 1


def gate_parameters_mc(hidden: int, channels: int, seed: int = 0) -> np.ndarray:
    """Flat float32 parameters of the M-channel gate: [W1 (hidden x (M+1),
    row-major), b1 (hidden), W2 ((M-1) x hidden, row-major), b2 (M-1)], each
    layer uniform on +-1/sqrt(fan_in).  For M = 2 this equals gate_parameters."""
    if channels == 2:
        return gate_parameters(hidden, seed)
    r = rng_for(seed, "gate")
    F = channels + 1
    w1 = r.uniform(-1.0, 1.0, (hidden, F)) / np.sqrt(F)
    b1 = r.uniform(-1.0, 1.0, hidden) / np.sqrt(F)
    w2 = r.uniform(-1.0, 1.0, (channels - 1, hidden)) / np.sqrt(hidden)
    b2 = r.uniform(-1.0, 1.0, channels - 1) / np.sqrt(hidden)
    return np.concatenate([w1.ravel(), b1, w2.ravel(), b2]).astype(np.float32)


# ---------------------------------------------------------------------------
# The five workloads, by what they are
# ---------------------------------------------------------------------------

def tiny_repertoire(seed: int = 0) -> Repertoire:
    """1,000 sequences, 100 families (half of the sequences), lengths 8-24."""
    return make_repertoire(1000, 100, seed=seed)


def donor_repertoire(n: int = 1_000_000, seed: int = 0) -> Repertoire:
    """One donor: n sequences, families of 25 members covering half of them, and
    50 rare subgroups of 0.1% of n each, assigned at family level."""
    n_fam = max(1, int(round(0.5 * n / 25)))
    return make_repertoire(n, n_fam, seed=seed, rare_subgroups=50,
                           rare_subgroup_size=max(1, n // 1000))


def zipf_repertoire(n: int = 10_000_000, seed: int = 0, hi: int = 50_000) -> Repertoire:
    """Lengths 6-30 (2% drawn uniformly from 25-30), Zipf(1.2) family sizes on
    [2, hi] until half of the sequences are family members."""
    sizes = zipf_family_sizes(n // 2, 1.2, 2, hi, rng_for(seed, "sizes"))
    return make_repertoire(n, seed=seed, len_min=6, len_max=24, tail_frac=0.02,
                           tail_range=(25, 30), family_sizes=sizes)


def pooled_repertoire(n_donors: int = 64, size_lo: int = 50_000, size_hi: int = 2_000_000, n_public: int = 500,
                      public_lo: float = 1e-4, public_hi: float = 1e-2, seed: int = 0,
                      family_size: int = 25) -> Repertoire:
    """Many donors pooled into one repertoire (``donor`` gives each sequence's
    donor).  Donor sizes are log-uniform on [size_lo, size_hi]; every donor has
    its own residue frequencies and private families (families of
    ``family_size`` covering half of its private sequences), and shares
    ``n_public`` public families: each donor's total public fraction f_d is
    log-uniform on [public_lo, public_hi] and its public members are spread
    uniformly over the public families (each a 1-3 substitution variant of the
    family's seed).  Family ids: public families 0..n_public-1, private ones
    after them."""
    r = rng_for(seed, "donors")
    sizes = np.exp(r.uniform(np.log(size_lo), np.log(size_hi), n_donors)).astype(np.int64)
    fracs = np.exp(r.uniform(np.log(public_lo), np.log(public_hi), n_donors))
    rp = rng_for(seed, "public")
    pub_freq = rp.dirichlet(np.full(20, 2.0))
    pub_lens = _draw_lengths(rp, n_public, 8, 24, 0.0, (25, 30))
    pub_codes = _draw_sequences(rp, pub_freq, pub_lens)
    codes, lens, family, subgroup, donor = [], [], [], [], []
    next_family = n_public
    for d in range(n_donors):
        n_d = int(sizes[d])
        n_pub = min(n_d, int(round(fracs[d] * n_d)))
        n_priv = n_d - n_pub
        n_fam = max(1, int(round(0.5 * n_priv / family_size)))
        rep = make_repertoire(n_priv, n_fam, seed=int(seed) * 100_003 + d + 1)
        rd = rng_for(int(seed) * 100_003 + d + 1, "public")
        pf = rd.integers(0, n_public, n_pub)
        pc = pub_codes[pf].copy()
        pl = pub_lens[pf].copy()
        _substitute(rd, pub_freq, pc, pl)
        fam = np.where(rep.family >= 0, rep.family + next_family, -1).astype(np.int32)
        next_family += n_fam
        c = np.concatenate([rep.codes, pc])
        l = np.concatenate([rep.lens, pl])
        f = np.concatenate([fam, pf.astype(np.int32)])
        perm = rd.permutation(n_d)
        codes.append(c[perm])
        lens.append(l[perm])
        family.append(f[perm])
        subgroup.append(np.zeros(n_d, dtype=np.int32))
        donor.append(np.full(n_d, d, dtype=np.int32))
    return Repertoire(codes=np.ascontiguousarray(np.concatenate(codes)), lens=np.ascontiguousarray(np.concatenate(lens)),
                      family=np.ascontiguousarray(np.concatenate(family)),
                      subgroup=np.ascontiguousarray(np.concatenate(subgroup)), freq=pub_freq,
                      donor=np.ascontiguousarray(np.concatenate(donor)))


def sample_queries(n: int, count: int, seed: int = 0) -> np.ndarray:
    """`count` distinct sequence ids drawn without replacement (uint32)."""
    return np.sort(rng_for(seed, "queries").choice(n, size=min(count, n), replace=False)).astype(np.uint32)
