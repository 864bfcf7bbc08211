"""Pins of the oracle's structural part (bit-exact by definition).

* Omega_i against breadth-first hops on the literal pattern of G^T G;
* the Boolean partition of unity sums to the identity (Eq. PoU, pou2);
* every row of nz_i lies inside Omega_i (the property that lets the
  splitting of the Lemma live on Omega_i);
* the multiplicity M against a row-by-row count (Lemma);
* cleanup and standard aggregation against hand-worked graphs.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from inputs import block_aggregates_2d, q1_2d, rotated_sqrtK
from oracle.structure import (
    cleanup_aggregates,
    multiplicity_and_nz,
    overlapping_subdomains,
    row_groups_from_csr,
    structural_adjacency,
    vanek_aggregation,
)
from tests import _brute


def _tiny(N=9, bs=3, d1=None, theta=math.pi / 6, eps=1e-2):
    agg = block_aggregates_2d(N, bs)
    D1 = None if d1 is None else np.full((N - 1) ** 2, d1)
    return q1_2d(N, rotated_sqrtK(theta, eps), D1=D1, agg=agg)


@pytest.mark.parametrize("overlap", [1, 2])
@pytest.mark.parametrize("d1", [None, 0.5])
def test_omega_matches_bfs(overlap, d1):
    p = _tiny(d1=d1)
    sups, grams = row_groups_from_csr(p.rowptr, p.col, p.val, p.n, p.D1)
    adj = structural_adjacency(sups, p.n)
    agg, nagg = cleanup_aggregates(p.agg, adj)
    om, ga, Om = overlapping_subdomains(agg, nagg, adj, overlap)
    G, P = _brute.dense_G(p)
    ref = _brute.omega_sets(P, agg, overlap)
    for i in range(nagg):
        assert np.array_equal(om[i], ref[i][0])
        assert np.array_equal(ga[i], ref[i][1])
        assert np.array_equal(Om[i], np.concatenate([ref[i][0], ref[i][1]]))


def test_partition_of_unity_identity():
    p = _tiny()
    h = oracle.setup(p.rowptr, p.col, p.val, p.n, p.D1, p.agg, overlap=1, n_coarse=10, L_max=2)
    L = h.levels[0]
    S = np.zeros((p.n, p.n), dtype=np.int64)
    for i in range(L.nagg):
        D = np.zeros(L.Omega[i].shape[0], dtype=np.int64)
        D[:L.omega[i].shape[0]] = 1
        R = np.zeros((L.Omega[i].shape[0], p.n), dtype=np.int64)
        R[np.arange(L.Omega[i].shape[0]), L.Omega[i]] = 1
        S += R.T @ np.diag(D) @ R
    assert np.array_equal(S, np.eye(p.n, dtype=np.int64))


def test_nz_rows_inside_Omega_and_multiplicity():
    p = _tiny(d1=0.1)
    G, P = _brute.dense_G(p)
    sups, grams = row_groups_from_csr(p.rowptr, p.col, p.val, p.n, p.D1)
    adj = structural_adjacency(sups, p.n)
    agg, nagg = cleanup_aggregates(p.agg, adj)
    M, nz, touched = multiplicity_and_nz(sups, agg, nagg)
    Mref = _brute.row_multiplicity(P, agg)
    # every literal row maps to the group with its support, with the same M
    key = {tuple(s.tolist()): g for g, s in enumerate(sups)}
    for l in range(P.shape[0]):
        g = key[tuple(np.nonzero(P[l])[0].tolist())]
        assert M[g] == Mref[l]
    _, _, Om = overlapping_subdomains(agg, nagg, adj, 1)
    for i in range(nagg):
        rows = _brute.nz_rows(P, agg, i)
        inside = set(Om[i].tolist())
        for l in rows:
            assert set(np.nonzero(P[l])[0].tolist()) <= inside
        # groups in nz_i are exactly the supports of the literal rows in nz_i
        assert {tuple(sups[g].tolist()) for g in nz[i]} == {tuple(np.nonzero(P[l])[0].tolist()) for l in rows}


def test_row_groups_sum_outer_products():
    p = _tiny(d1=0.3)
    G, P = _brute.dense_G(p)
    sups, grams = row_groups_from_csr(p.rowptr, p.col, p.val, p.n, p.D1)
    A = np.zeros((p.n, p.n))
    for s, H in zip(sups, grams):
        A[np.ix_(s, s)] += H
    assert np.abs(A - G.T @ G).max() <= 1e-14 * np.abs(G.T @ G).max()


def _graph(n, edges):
    r = [a for a, b in edges] + [b for a, b in edges]
    c = [b for a, b in edges] + [a for a, b in edges]
    return sp.csr_matrix((np.ones(len(r)), (r, c)), shape=(n, n))


def test_vanek_path():
    # 0-1-2-3-4-5-6: roots 0 -> {0,1}; 3 -> {2,3,4}; 6 -> {5,6}
    agg, n = vanek_aggregation(_graph(7, [(i, i + 1) for i in range(6)]))
    assert n == 3 and agg.tolist() == [0, 0, 1, 1, 1, 2, 2]


def test_vanek_pass_two():
    # star: 0,1,2 hang off 3; 4 links 3 to 5 and 6.
    # pass 1: root 0 -> {0,3}; root 5 -> {4,5}; pass 2: 1,2 -> agg of 3; 6 -> agg of 4
    agg, n = vanek_aggregation(_graph(7, [(0, 3), (1, 3), (2, 3), (3, 4), (4, 5), (4, 6)]))
    assert n == 2 and agg.tolist() == [0, 0, 0, 0, 1, 1, 1]


def test_vanek_isolated_node():
    agg, n = vanek_aggregation(_graph(3, [(0, 1)]))
    assert n == 2 and agg.tolist() == [0, 0, 1]


def test_cleanup_unaggregated():
    # path 0-1-2-3-4 with ids [-1, 5, -1, -1, 9]: relabel 5->0, 9->1;
    # node 0 joins 0 (neighbour 1); node 2 joins 0 (neighbour 1);
    # node 3: neighbours 2 (now 0) and 4 (1) -> smallest id 0
    adj = _graph(5, [(i, i + 1) for i in range(4)]) + sp.identity(5)
    agg, n = cleanup_aggregates(np.array([-1, 5, -1, -1, 9]), adj.tocsr())
    assert n == 2 and agg.tolist() == [0, 0, 0, 0, 1]


def test_cleanup_isolated_unaggregated():
    adj = (_graph(3, [(0, 1)]) + sp.identity(3)).tocsr()
    agg, n = cleanup_aggregates(np.array([0, 0, -1]), adj)
    assert n == 2 and agg.tolist() == [0, 0, 1]


def test_coarse_blocks_stay_whole():
    N = 12
    p = q1_2d(N, rotated_sqrtK(0.4, 0.05), agg=block_aggregates_2d(N, 2))
    h = oracle.setup(p.rowptr, p.col, p.val, p.n, p.D1, p.agg, overlap=1, c_min=(2,), n_coarse=15, L_max=5)
    assert len(h.levels) >= 3
    L0, L1 = h.levels[0], h.levels[1]
    for a in range(L0.nagg):
        ids = L1.agg[L0.col0[a]:L0.col0[a + 1]]
        assert np.all(ids == ids[0])


def test_coarse_overlap_hops_per_level():
    """overlap = 2 on level 0 and coarse_overlap = 1 above: Omega_i on each
    level against breadth-first hops of that depth on the literal pattern of
    that level's row supports."""
    p = _tiny(N=17, bs=4)
    h = oracle.setup(p.rowptr, p.col, p.val, p.n, p.D1, p.agg, overlap=2, coarse_overlap=1, c_min=(2,),
                     n_coarse=20)
    assert len(h.levels) >= 3
    for lvl, L in enumerate(h.levels[:-1]):
        hops = 2 if lvl == 0 else 1
        P = np.zeros((len(L.sups), L.n), dtype=bool)
        for g, sup in enumerate(L.sups):
            P[g, np.asarray(sup)] = True
        ref = _brute.omega_sets(P, np.asarray(L.agg), hops)
        for i in range(L.nagg):
            assert np.array_equal(L.omega[i], ref[i][0])
            assert np.array_equal(L.gamma[i], ref[i][1])
