"""Planted mistakes in the oracle's threshold, colouring, aggregation and row-form code (CPU only).

Each mistake is planted with monkeypatch where the code under test looks the function up, and the pin that
must catch it is run expecting its assertion to fail.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle.construct as osetup
import oracle.structure as ostruct
from tests import test_oracle_aggregation as TA
from tests import test_oracle_kappa as TK
from tests import test_oracle_schur_rows as TR
from inputs import fd_2d, fd_block_aggregates


def _fd13():
    return fd_2d(13, 0.5, 1e-3, agg=fd_block_aggregates(13, 2))


def test_colouring_by_shared_nodes_only_is_caught(monkeypatch):
    orig = ostruct.subdomain_colouring

    def shared_only(Omega, adj, n):  # forgets the coupling through A, keeps only common nodes
        return orig(Omega, sp.identity(n, format="csr", dtype=bool), n)

    monkeypatch.setattr(TK, "subdomain_colouring", shared_only)
    with pytest.raises(AssertionError):
        TK.test_colouring_is_proper_and_greedy(_fd13)


def test_colouring_that_is_not_smallest_free_is_caught(monkeypatch):
    def not_greedy(Omega, adj, n):
        nagg = len(Omega)
        rows = np.concatenate([np.full(o.shape[0], i) for i, o in enumerate(Omega)])
        T = sp.csr_matrix((np.ones(rows.shape[0]), (rows, np.concatenate(Omega))), shape=(nagg, n))
        C = (T @ adj.astype(float) @ T.T).tocsr()
        colour = np.zeros(nagg, dtype=np.int64)
        for i in range(nagg):
            nb = [j for j in C.indices[C.indptr[i]:C.indptr[i + 1]] if j < i]
            colour[i] = 1 + max((colour[j] for j in nb), default=-1)  # one above the largest, not the smallest free
        return colour, int(colour.max()) + 1

    monkeypatch.setattr(TK, "subdomain_colouring", not_greedy)
    with pytest.raises(AssertionError):
        TK.test_colouring_is_proper_and_greedy(_fd13)


def test_swapped_counts_in_threshold_are_caught(monkeypatch):
    monkeypatch.setattr(osetup, "kappa_threshold", lambda k, nc, nm: max(0.1, (k - nm) / (nc * nm)))
    with pytest.raises(AssertionError):
        TK.test_fd_blocks_need_four_colours_and_multiplicity_three()


def test_missing_floor_is_caught(monkeypatch):
    monkeypatch.setattr(TK, "kappa_threshold", lambda k, nc, nm: (k - nc) / (nc * nm))
    with pytest.raises(AssertionError):
        TK.test_floor()


def test_second_pass_on_the_wrong_graph_is_caught(monkeypatch):
    def wrong_graph(sups, n, passes=1):  # pass 2 on T^T T (aggregates never share nodes) instead of T^T A T
        adj = ostruct.structural_adjacency(sups, n).astype(np.int32)
        off = adj.copy()
        off.setdiag(0)
        off.eliminate_zeros()
        agg, nagg = ostruct.vanek_aggregation(off)
        for _ in range(passes - 1):
            T = sp.csr_matrix((np.ones(n, dtype=np.int32), (np.arange(n), agg)), shape=(n, nagg))
            C = (T.T @ T).tocsr()
            C.setdiag(0)
            C.eliminate_zeros()
            bagg, nagg = ostruct.vanek_aggregation(C)
            agg = bagg[agg]
        return agg, nagg

    monkeypatch.setattr(TA, "standard_aggregation", wrong_graph)
    with pytest.raises(AssertionError):
        TA.test_path_two_and_three_passes()


def test_unscaled_rows_are_caught(monkeypatch):
    orig = osetup.local_splitting_rows
    monkeypatch.setattr(TR, "local_splitting_rows",
                        lambda Om, nz, sups, rows, M: orig(Om, nz, sups, rows, np.ones_like(M)))
    with pytest.raises(AssertionError):
        TR.test_rows_reproduce_grams_and_splitting()


def test_row_route_without_projection_is_caught(monkeypatch):
    # S~ = X^T X (the Gamma rows ignored) no longer matches the Gram route where the gap is clean
    monkeypatch.setattr(osetup, "schur_complement_rows", lambda Y, no, sv: Y[:, :no].T @ Y[:, :no])
    with pytest.raises(AssertionError):
        TR.test_rows_match_gram_route_on_clean_gap()
