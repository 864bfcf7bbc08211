"""Pins of level-0 standard aggregation with repeated passes (Section 3.3).

* a path of 27 nodes, worked by hand: one pass gives {0,1}, {2,3,4}, ..., {23,24,25,26} (9 aggregates); the
  second pass aggregates that 9-node path the same way, giving nodes 0-4, 5-13 and 14-26; a third pass merges
  everything;
* an isolated node (a D1-only unknown) is an aggregate of its own;
* invariants on the 2D workloads: every node aggregated, every aggregate connected in the graph of A, ids
  0..nagg-1 all used, and each aggregate of pass p + 1 a union of aggregates of pass p.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

from oracle.construct import row_groups_from_csr
from oracle.structure import standard_aggregation, structural_adjacency
from inputs import fd_2d, q1_2d, rotated_sqrtK


def _path(n):
    return [np.array([i, i + 1]) for i in range(n - 1)]


def test_path_one_pass():
    agg, n = standard_aggregation(_path(27), 27, 1)
    want = [0, 0] + sum(([k] * 3 for k in range(1, 8)), []) + [8] * 4
    assert n == 9 and agg.tolist() == want


def test_path_two_and_three_passes():
    agg, n = standard_aggregation(_path(27), 27, 2)
    assert n == 3 and agg.tolist() == [0] * 5 + [1] * 9 + [2] * 13
    agg, n = standard_aggregation(_path(27), 27, 3)
    assert n == 1 and agg.tolist() == [0] * 27


def test_isolated_node():
    sups = _path(4) + [np.array([5])]  # node 4 touches no row; node 5 only its own (D1-like) row
    agg, n = standard_aggregation(sups, 6, 1)
    assert agg[4] != agg[5] and agg[4] not in agg[:4] and agg[5] not in agg[:4]
    assert n == len(set(agg.tolist()))


@pytest.mark.parametrize("make", [lambda: fd_2d(20, math.pi / 6, 1e-4),
                                  lambda: q1_2d(17, rotated_sqrtK(0.4, 1e-3))])
@pytest.mark.parametrize("passes", [1, 2, 3])
def test_invariants(make, passes):
    p = make()
    sups, _ = row_groups_from_csr(p.rowptr, p.col, p.val, p.n, p.D1)
    adj = structural_adjacency(sups, p.n)
    agg, n = standard_aggregation(sups, p.n, passes)
    assert agg.min() == 0 and set(agg.tolist()) == set(range(n))
    for a in range(n):
        nodes = np.flatnonzero(agg == a)
        sub = adj[nodes][:, nodes]
        assert connected_components(sub, directed=False)[0] == 1
    if passes > 1:
        prev, _ = standard_aggregation(sups, p.n, passes - 1)
        for a in np.unique(prev):
            assert np.unique(agg[prev == a]).shape[0] == 1
