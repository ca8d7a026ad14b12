"""Oracle for the graph step of Algorithm 1: the fused similarity matrix A
and its RMT-based thresholding into the sparse graph G (the section on graph
construction and RMT-based thresholding), and the cluster-mass Jensen-Shannon
repertoire distance of the appendix on repertoire-level distances.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): plain, slow numpy /
scipy, FP64, no code shared with the CUDA path.

Readings (the paper states the three steps -- eigenvalue spectrum of A, bulk
cutoff estimated from it, edges below the resulting threshold removed -- and
names MetaNet's random-matrix thresholding as its model):

* A is symmetric with A_ij = A_ji = fused(i, j) on the candidate pairs and 0
  elsewhere (including the diagonal).
* The threshold is scanned over a grid tau_1 < tau_2 < ...; A_tau keeps the
  entries >= tau.  A_tau is block-diagonal over the connected components of
  its graph, so its spectrum is the union of the components' spectra
  (isolated vertices are left out: they only add zero levels).
* The spectral statistic is the mean ratio of consecutive level spacings,
  <r> = mean_k min(d_k, d_{k+1}) / max(d_k, d_{k+1}) over the sorted spectrum
  (Oganesyan-Huse; it needs no unfolding).  Its reference values are
  2 ln 2 - 1 = 0.3863 for uncorrelated (Poisson) levels and 4 - 2 sqrt 3 =
  0.5359 for the Gaussian orthogonal ensemble (Wigner-like surmise of Atas et
  al.).  Levels within EPS_LEVEL of their predecessor are one degenerate
  level (dropped before the spacings are taken).
* The bulk cutoff is the random-matrix (GOE) to localized (Poisson)
  transition: tau* is the smallest grid threshold whose spectrum is closer to
  Poisson than to GOE, <r> <= R_MID = midpoint of the two reference values.
  A threshold at which some component has more than s_max vertices is not
  evaluated (a percolating component is the random-matrix regime).  If no
  grid value qualifies, tau* is the largest grid value.
* G keeps the candidate pairs with fused >= tau*, with their fused weights.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

R_POISSON = 2.0 * math.log(2.0) - 1.0
R_GOE = 4.0 - 2.0 * math.sqrt(3.0)
R_MID = 0.5 * (R_POISSON + R_GOE)
EPS_LEVEL = 1e-9


def components(n: int, pairs, weights, tau: float) -> np.ndarray:
    """Component label of every vertex in the graph of the pairs with weight
    >= tau; the label is the smallest vertex id of the component."""
    p = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    w = np.asarray(weights, dtype=np.float64)
    keep = w >= tau
    g = sp.coo_matrix((np.ones(int(keep.sum())), (p[keep, 0], p[keep, 1])), shape=(n, n))
    _, lab = connected_components(g, directed=False)
    first = np.full(lab.max() + 1 if n else 0, n, dtype=np.int64)
    np.minimum.at(first, lab, np.arange(n))
    return first[lab].astype(np.int64)


def r_statistic(levels) -> tuple[float, int]:
    """(<r>, number of ratios) of a spectrum: sort, drop levels within
    EPS_LEVEL of their predecessor, spacings d_k, ratios min/max of
    neighbouring spacings, mean.  NaN with fewer than three kept levels."""
    lv = np.sort(np.asarray(levels, dtype=np.float64))
    if lv.size == 0:
        return float("nan"), 0
    keep = np.ones(lv.size, dtype=bool)
    keep[1:] = np.diff(lv) > EPS_LEVEL
    lv = lv[keep]
    if lv.size < 3:
        return float("nan"), 0
    d = np.diff(lv)
    r = np.minimum(d[:-1], d[1:]) / np.maximum(d[:-1], d[1:])
    return float(r.mean()), int(r.size)


def threshold_spectrum(n: int, pairs, weights, tau: float, s_max: int) -> dict:
    """Spectrum of A_tau as the union of its components' spectra (numpy's
    symmetric eigensolver on each component's dense block)."""
    p = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    w = np.asarray(weights, dtype=np.float64)
    lab = components(n, p, w, tau)
    sizes = np.bincount(lab, minlength=n)
    max_comp = int(sizes.max()) if n else 0
    active = np.flatnonzero(sizes >= 2)
    out = {"tau": tau, "max_comp": max_comp if active.size else 0, "components": int(active.size),
           "evaluable": bool(active.size == 0 or sizes[active].max() <= s_max)}
    if not out["evaluable"]:
        out.update(levels=None, r_mean=float("nan"), n_r=0)
        return out
    keep = np.flatnonzero(w >= tau)
    edge_comp = lab[p[keep, 0]]
    by_comp = keep[np.argsort(edge_comp, kind="stable")]
    bounds = np.searchsorted(np.sort(edge_comp), active)
    ends = np.searchsorted(np.sort(edge_comp), active, side="right")
    vorder = np.argsort(lab, kind="stable")
    vstart = np.searchsorted(lab[vorder], active)
    levels = []
    for c, e0, e1, v0 in zip(active, bounds, ends, vstart):
        verts = vorder[v0:v0 + sizes[c]]
        local = {int(v): k for k, v in enumerate(verts)}
        M = np.zeros((verts.size, verts.size))
        for q in by_comp[e0:e1]:
            i, j = int(p[q, 0]), int(p[q, 1])
            M[local[i], local[j]] = w[q]
            M[local[j], local[i]] = w[q]
        levels.append(np.linalg.eigvalsh(M))
    lv = np.sort(np.concatenate(levels)) if levels else np.zeros(0)
    r, nr = r_statistic(lv)
    out.update(levels=lv, r_mean=r, n_r=nr)
    return out


def rmt_threshold(n: int, pairs, weights, taus, s_max: int = 64):
    """(tau*, [per-threshold dicts]) of the scan described in the module
    docstring; the scan stops at the first qualifying threshold."""
    stats = []
    for tau in taus:
        st = threshold_spectrum(n, pairs, weights, float(tau), s_max)
        stats.append(st)
        if st["evaluable"] and st["n_r"] > 0 and st["r_mean"] <= R_MID:
            return float(tau), stats
    return float(taus[-1]), stats


def prune(pairs, weights, tau: float):
    """G: the pairs with weight >= tau, in input order, with their weights."""
    p = np.asarray(pairs).reshape(-1, 2)
    w = np.asarray(weights)
    keep = w >= tau
    return p[keep], w[keep]


# --------------------------------------------------------------------------
# Cluster-mass Jensen-Shannon repertoire distance (appendix on
# repertoire-level distances).  Reading: the K-partition shared by all
# repertoires is the connected components of G built over the pooled
# repertoires (so cluster k means the same cluster for every repertoire);
# p_A^(k) = |C^(k) n V_A| / |V_A|; natural logarithm; D = sqrt(JS).
# --------------------------------------------------------------------------

def cluster_mass(labels, donor, num_donors: int):
    """dict cluster label -> float64 [num_donors] masses p_d(k) (columns sum
    to one over k for every donor with sequences)."""
    labels = np.asarray(labels)
    donor = np.asarray(donor)
    sizes = np.bincount(donor, minlength=num_donors).astype(np.float64)
    masses = {}
    for k in np.unique(labels):
        cnt = np.bincount(donor[labels == k], minlength=num_donors).astype(np.float64)
        masses[int(k)] = np.divide(cnt, sizes, out=np.zeros(num_donors), where=sizes > 0)
    return masses


def js_divergence(pA, pB) -> float:
    """Jensen-Shannon divergence (natural log) of two discrete distributions:
    1/2 KL(pA || M) + 1/2 KL(pB || M), M = (pA + pB) / 2, with 0 log 0 = 0."""
    pA = np.asarray(pA, dtype=np.float64)
    pB = np.asarray(pB, dtype=np.float64)
    M = 0.5 * (pA + pB)
    total = 0.0
    for P in (pA, pB):
        nz = P > 0
        total += 0.5 * float(np.sum(P[nz] * np.log(P[nz] / M[nz])))
    return total


def js_distance_matrix(labels, donor, num_donors: int) -> np.ndarray:
    """float64 [num_donors, num_donors]: sqrt of the JS divergence between the
    cluster-mass vectors of every pair of donors."""
    masses = cluster_mass(labels, donor, num_donors)
    K = sorted(masses)
    P = np.stack([masses[k] for k in K], axis=1) if K else np.zeros((num_donors, 0))  # [donor, cluster]
    D = np.zeros((num_donors, num_donors))
    for a in range(num_donors):
        for b in range(num_donors):
            D[a, b] = math.sqrt(max(js_divergence(P[a], P[b]), 0.0))
    return D
