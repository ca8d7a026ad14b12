"""Pins for the oracle of the graph step (RMT-based thresholding of the fused
similarity matrix) and of the cluster-mass Jensen-Shannon repertoire
distance."""
import math

import numpy as np
import pytest
import scipy.spatial.distance

from oracle import graph as G


def test_reference_constants():
    assert abs(G.R_POISSON - 0.3862943611198906) < 1e-15
    assert abs(G.R_GOE - 0.5358983848622456) < 1e-15


def test_r_statistic_poisson_levels():
    """Uncorrelated levels (exponential spacings): <r> = 2 ln 2 - 1."""
    rng = np.random.default_rng(0)
    N = 400_000
    r, nr = G.r_statistic(np.cumsum(rng.exponential(size=N)))
    assert nr == N - 2
    # sd of r under Poisson is about 0.28; neighbouring ratios share a spacing
    assert abs(r - G.R_POISSON) < 8 * 0.28 / math.sqrt(N)


def test_r_statistic_goe_and_superposition():
    """A large GOE matrix has level repulsion (<r> near 0.53); a union of many
    independent GOE blocks has none across blocks (<r> near the Poisson
    value), which is what a block-diagonal thresholded matrix gives."""
    rng = np.random.default_rng(1)
    X = rng.normal(size=(2000, 2000))
    r_goe, _ = G.r_statistic(np.linalg.eigvalsh((X + X.T) / 2))
    assert 0.52 < r_goe < 0.545
    blocks = []
    for _ in range(2000):
        Y = rng.normal(size=(20, 20))
        blocks.append(np.linalg.eigvalsh((Y + Y.T) / 2))
    r_sup, _ = G.r_statistic(np.concatenate(blocks))
    assert abs(r_sup - G.R_POISSON) < 0.01


def test_degenerate_levels_are_merged():
    r, nr = G.r_statistic([0.5, -0.5] * 100)
    assert nr == 0 and math.isnan(r)
    r, nr = G.r_statistic([0.0, 1.0, 1.0 + 1e-12, 3.0, 3.0])
    assert nr == 1 and abs(r - 0.5) < 1e-15  # levels 0, 1, 3: spacings 1, 2


def bfs_labels(n, pairs, w, tau):
    adj = [[] for _ in range(n)]
    for (i, j), x in zip(pairs, w):
        if x >= tau:
            adj[i].append(j)
            adj[j].append(i)
    lab = [-1] * n
    for s in range(n):
        if lab[s] >= 0:
            continue
        lab[s] = s
        stack = [s]
        while stack:
            u = stack.pop()
            for v in adj[u]:
                if lab[v] < 0:
                    lab[v] = s
                    stack.append(v)
    return np.array(lab)


def random_graph(rng, n, m):
    i = rng.integers(0, n, m)
    j = rng.integers(0, n, m)
    keep = i < j
    p = np.unique(np.stack([i[keep], j[keep]], 1), axis=0)
    return p, rng.uniform(0, 1, p.shape[0])


def test_components_against_bfs():
    rng = np.random.default_rng(2)
    for _ in range(20):
        n = int(rng.integers(1, 200))
        p, w = random_graph(rng, n, int(rng.integers(0, 3 * n)))
        tau = float(rng.uniform(0, 1))
        assert (G.components(n, p, w, tau) == bfs_labels(n, p, w, tau)).all()


def test_spectrum_moments():
    """trace A = 0 and trace A^2 = 2 sum w^2 over the kept edges."""
    rng = np.random.default_rng(3)
    n = 300
    p, w = random_graph(rng, n, 250)
    st = G.threshold_spectrum(n, p, w, 0.3, 64)
    assert st["evaluable"]
    keep = w >= 0.3
    assert abs(st["levels"].sum()) < 1e-10
    assert abs((st["levels"] ** 2).sum() - 2 * (w[keep] ** 2).sum()) < 1e-9


def planted(rng, n_cliques=300, noise_deg=3.0):
    sizes = rng.integers(4, 16, n_cliques)
    n = int(sizes.sum()) + 2000
    pairs, w = [], []
    base = 0
    for s in sizes:
        for a in range(s):
            for b in range(a + 1, s):
                pairs.append((base + a, base + b))
                w.append(rng.uniform(0.6, 0.9))
        base += s
    m_noise = int(noise_deg * n / 2)
    i = rng.integers(0, n, m_noise)
    j = rng.integers(0, n, m_noise)
    for a, b in zip(i, j):
        if a != b:
            pairs.append((min(a, b), max(a, b)))
            w.append(rng.uniform(0.2, 0.45))
    p = np.array(pairs)
    uniq, first = np.unique(p, axis=0, return_index=True)
    return n, uniq, np.array(w)[first]


def test_threshold_separates_planted_cliques_from_noise():
    """Cliques with weights in [0.6, 0.9] plus a percolating random graph of
    weights in [0.2, 0.45]: the scan stops between the two ranges, and G keeps
    exactly the clique edges."""
    rng = np.random.default_rng(4)
    n, p, w = planted(rng)
    taus = np.round(np.arange(0.30, 0.91, 0.05), 2)
    tau_star, stats = G.rmt_threshold(n, p, w, taus, 64)
    assert 0.45 <= tau_star <= 0.6
    assert not stats[0]["evaluable"]  # the noise percolates at the lowest threshold
    assert stats[-1]["r_mean"] <= G.R_MID
    gp, gw = G.prune(p, w, tau_star)
    assert (gw >= 0.6).all() and gp.shape[0] == int((w >= 0.6).sum())


def test_js_distance_against_scipy():
    rng = np.random.default_rng(5)
    for _ in range(50):
        K = int(rng.integers(1, 30))
        pA = rng.dirichlet(np.ones(K)) * (rng.uniform(size=K) > 0.3)
        pB = rng.dirichlet(np.ones(K)) * (rng.uniform(size=K) > 0.3)
        if pA.sum() == 0 or pB.sum() == 0:
            continue
        pA, pB = pA / pA.sum(), pB / pB.sum()
        want = scipy.spatial.distance.jensenshannon(pA, pB)  # natural log, sqrt of the divergence
        assert abs(math.sqrt(G.js_divergence(pA, pB)) - want) < 1e-12


def test_js_matrix_special_cases():
    labels = np.array([0, 0, 1, 1, 2, 2, 3, 3, 4, 4])
    donor = np.array([0, 0, 0, 0, 1, 1, 1, 1, 2, 2])
    D = G.js_distance_matrix(labels, donor, 3)
    assert abs(D[0, 1] - math.sqrt(math.log(2))) < 1e-15  # disjoint clusters
    assert (np.diag(D) == 0).all() and np.allclose(D, D.T)
    same = G.js_distance_matrix(np.array([0, 1, 0, 1]), np.array([0, 0, 1, 1]), 2)
    assert same[0, 1] == 0.0
    masses = G.cluster_mass(labels, donor, 3)
    assert np.allclose(sum(masses.values()), 1.0)
