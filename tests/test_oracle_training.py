"""Pins for the oracle's pair labels and pair groups, the inputs of the gate
objective (family-match labels, subgroup reweighting).

The expected labels and groups are written out by hand from the definition:
a pair is a positive iff both members belong to the same clonotype family
(background sequences, family -1, are singletons and never match, not even
each other); the pair's group is the first member's subgroup when that is
nonzero, else the second member's.
"""
import numpy as np

#            id:   0   1   2   3   4   5   6   7
FAMILY = np.array([3,  3, -1, -1,  7,  7,  3,  0], dtype=np.int32)
SUBGROUP = np.array([0, 2,  0,  5,  0,  4,  1,  0], dtype=np.int32)

# (i, j, label, group), by hand
HAND = [
    (0, 1, 1, 2),  # same family 3; subgroup(0) = 0 -> subgroup(1) = 2
    (1, 6, 1, 2),  # same family 3; subgroup(1) = 2 taken first
    (0, 6, 1, 1),  # same family 3; falls back to subgroup(6) = 1
    (2, 3, 0, 5),  # both background: no match; subgroup(2) = 0 -> 5
    (3, 2, 0, 5),  # order reversed: subgroup(3) = 5 taken first
    (2, 2, 0, 0),  # a background sequence is not its own family
    (4, 5, 1, 4),  # family 7; subgroup(4) = 0 -> 4
    (5, 4, 1, 4),  # subgroup(5) = 4 taken first
    (0, 4, 0, 0),  # families 3 and 7: no match; both subgroups 0
    (6, 7, 0, 1),  # families 3 and 0: no match; subgroup(6) = 1
    (7, 7, 1, 0),  # family 0 is a real family (not background): self pair matches
    (3, 5, 0, 5),  # background vs family 7
    (4, 2, 0, 0),  # family 7 vs background; both subgroups 0
]


def test_pair_labels_and_groups_by_hand(oracle_mod):
    pairs = np.array([(i, j) for i, j, _, _ in HAND], dtype=np.uint32)
    y, g = oracle_mod.pair_labels(pairs, FAMILY, SUBGROUP)
    assert y.tolist() == [lab for _, _, lab, _ in HAND]
    assert g.tolist() == [grp for _, _, _, grp in HAND]


def test_pair_labels_empty(oracle_mod):
    y, g = oracle_mod.pair_labels(np.zeros((0, 2), np.uint32), FAMILY, SUBGROUP)
    assert y.shape == (0,) and g.shape == (0,)
