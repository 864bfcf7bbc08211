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


def _lexicographic_mis_of_square(adj):
    """The first maximal independent set, in ascending order, of the graph joining vertices within distance 2."""
    A = (adj != 0).astype(np.int64)
    A.setdiag(1)
    A2 = (A @ A).tocsr()
    chosen, blocked = [], np.zeros(adj.shape[0], dtype=bool)
    for v in range(adj.shape[0]):
        if not blocked[v]:
            chosen.append(v)
            blocked[A2.indices[A2.indptr[v]:A2.indptr[v + 1]]] = True
    return chosen


@pytest.mark.parametrize("seed", range(6))
def test_pass_one_roots_are_the_first_independent_set_of_the_squared_graph(seed):
    """A characterisation of pass 1 independent of its loop: a vertex roots an aggregate exactly when no
    lower-index root lies within distance 2 (a vertex is aggregated only by an adjacent root), so the roots
    are the ascending-order maximal independent set of the distance-2 graph; and with every edge strong no
    vertex is left for pass 3 (a vertex that is no root had an aggregated neighbour at its visit).  Pass 1
    creates id t at its t-th root, so the t-th vertex of that set must carry id t, with its neighbours, and
    the count of aggregates must equal the set's size."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(40, 400))
    sups = [np.unique(rng.integers(0, n, size=int(rng.integers(1, 5)))) for _ in range(int(rng.integers(n // 2, 2 * n)))]
    adj = structural_adjacency(sups, n).tocsr()
    adj.setdiag(0)
    adj.eliminate_zeros()
    roots = _lexicographic_mis_of_square(adj)
    agg, nagg = standard_aggregation(sups, n, 1)
    # pass 1 made exactly len(roots) aggregates (pass 3 none): each root's id is its rank, and it holds its root
    assert nagg == len(roots)
    for t, r in enumerate(roots):
        assert agg[r] == t
    # each root's neighbours share its aggregate (pass 1 takes the whole closed neighbourhood)
    for r in roots:
        nb = adj.indices[adj.indptr[r]:adj.indptr[r + 1]]
        assert np.all(agg[nb] == agg[r])


def test_planted_pass_one_mistake_is_caught(monkeypatch):
    """A pass 1 that roots an aggregate whenever the node itself is free (ignoring its neighbours) breaks the
    characterisation above."""
    import oracle.structure as ostruct

    def greedy_free_only(adj_nodiag):
        A = adj_nodiag.tocsr()
        n = A.shape[0]
        agg = -np.ones(n, dtype=np.int64)
        nxt = 0
        for j in range(n):
            if agg[j] >= 0:
                continue
            nb = A.indices[A.indptr[j]:A.indptr[j + 1]]
            agg[j] = nxt
            agg[nb[agg[nb] < 0]] = nxt
            nxt += 1
        return agg, nxt

    monkeypatch.setattr(ostruct, "vanek_aggregation", greedy_free_only)
    with pytest.raises(AssertionError):
        for seed in range(6):
            test_pass_one_roots_are_the_first_independent_set_of_the_squared_graph(seed)
