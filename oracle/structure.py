"""Structural part of the oracle (integer work; test infrastructure only).

* row groups of G (rows with identical structural support) with their
  outer-product sums -- the form in which the oracle holds G_l;
* the structural graph of A = G^T G: j ~ k iff some row of G has both j and
  k in its support (Section 2.2 builds Gamma_i from "neighbouring nodes in
  the sparsity graph of A");
* cleanup of unaggregated nodes (Section 3.3: unaggregated fine nodes join
  an aggregate of a neighbour);
* overlapping subdomains Omega_i = omega_i u Gamma_i, with Gamma_i the
  nodes within `overlap` graph hops of omega_i (Section 2.2; Algorithm 1,
  "Overlapping subdomains"); local order omega_i ascending, then Gamma_i
  ascending (the omega/Gamma/Delta ordering of Eq. permutation_matrix);
* row multiplicity M(l) and the row sets nz_i (Section 3.1, Lemma);
* standard (Vanek) aggregation passes on a graph whose edges are all strong
  (Section 2.1 describes the passes), used on the coarse-level block graph.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def row_groups_from_csr(rowptr, col, val, n, D1=None, with_rows=False):
    """Group the rows of G (and the rows sqrt(D1_jj) e_j^T) by support.

    Returns (supports, grams): supports[g] is the sorted int64 column list
    shared by every row of group g, grams[g] = sum over those rows of
    g_l^T g_l restricted to the support (dense, symmetric).  Section 1
    writes A = D1 + B^T D2^{-1} B = G^T G with G^T = [sqrt(D1), ...], so the
    D1 rows are ordinary rows of G with a one-node support.  With_rows adds
    a third list: the group's rows themselves (count x support size).
    """
    rowptr = np.asarray(rowptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    val = np.asarray(val, dtype=np.float64)
    lens = np.diff(rowptr)
    sups, grams, rws = [], [], []
    # rows of equal length are handled together; identical supports merge
    extra = None
    if D1 is not None:
        d = np.asarray(D1, dtype=np.float64)
        extra = (np.arange(n, dtype=np.int64)[:, None], np.sqrt(d)[:, None])
    for s in np.unique(lens):
        if s == 0:
            continue
        rows = np.nonzero(lens == s)[0]
        idx = rowptr[rows][:, None] + np.arange(s)[None, :]
        C = col[idx]
        V = val[idx]
        order = np.argsort(C, axis=1, kind="stable")
        C = np.take_along_axis(C, order, axis=1)
        V = np.take_along_axis(V, order, axis=1)
        if extra is not None and s == 1:
            C = np.concatenate([C, extra[0]])
            V = np.concatenate([V, extra[1]])
            extra = None
        _append_groups(C, V, sups, grams, rws)
    if extra is not None:
        _append_groups(extra[0], extra[1], sups, grams, rws)
    return (sups, grams, rws) if with_rows else (sups, grams)


def _append_groups(C, V, sups, grams, rws):
    uniq, inv = np.unique(C, axis=0, return_inverse=True)
    inv = inv.ravel()
    outer = V[:, :, None] * V[:, None, :]
    H = np.zeros((uniq.shape[0],) + outer.shape[1:])
    np.add.at(H, inv, outer)
    order = np.argsort(inv, kind="stable")
    starts = np.searchsorted(inv[order], np.arange(uniq.shape[0] + 1))
    for g in range(uniq.shape[0]):
        sups.append(uniq[g].astype(np.int64))
        grams.append(H[g])
        rws.append(V[order[starts[g]:starts[g + 1]]])


def incidence(sups, n):
    """Boolean group-by-node incidence E (E[g, j] = 1 iff j in support g)."""
    lens = np.array([len(s) for s in sups], dtype=np.int64)
    indptr = np.zeros(len(sups) + 1, dtype=np.int64)
    np.cumsum(lens, out=indptr[1:])
    indices = np.concatenate(sups) if sups else np.zeros(0, dtype=np.int64)
    data = np.ones(indices.shape[0], dtype=np.int8)
    return sp.csr_matrix((data, indices, indptr), shape=(len(sups), n))


def structural_adjacency(sups, n):
    """Structural graph of A = G^T G (diagonal included), boolean CSR."""
    E = incidence(sups, n).astype(np.int32)
    adj = (E.T @ E).tocsr()
    adj = adj + sp.identity(n, dtype=np.int32, format="csr")
    adj.data[:] = 1
    adj.eliminate_zeros()
    return adj.astype(bool).tocsr()


def cleanup_aggregates(agg, adj):
    """Relabel aggregate ids to 0..nagg-1 and attach unaggregated (-1) nodes.

    Reading of Section 3.3 ("assign any unaggregated fine nodes ... to one of
    the aggregates of their neighbors"): nodes are visited in ascending
    order, and a node with id -1 joins the smallest aggregate id among its
    already-aggregated structural neighbours; sweeps repeat while they make
    progress, and nodes that never see an aggregated neighbour become
    singleton aggregates (appended ids, ascending node order).  Ids with no
    node are removed by relabelling in ascending id order.
    """
    agg = np.array(agg, dtype=np.int64)
    n = agg.shape[0]
    adj = adj.tocsr()
    while True:
        todo = np.nonzero(agg < 0)[0]
        if todo.size == 0:
            break
        progress = False
        for j in todo:
            nb = adj.indices[adj.indptr[j]:adj.indptr[j + 1]]
            ids = agg[nb]
            ids = ids[ids >= 0]
            if ids.size:
                agg[j] = ids.min()
                progress = True
        if not progress:
            nxt = agg.max() + 1 if (agg >= 0).any() else 0
            for j in np.nonzero(agg < 0)[0]:
                agg[j] = nxt
                nxt += 1
    uniq, inv = np.unique(agg, return_inverse=True)
    return inv.astype(np.int64).reshape(n), int(uniq.shape[0])


def overlapping_subdomains(agg, nagg, adj, overlap):
    """omega_i, Gamma_i and Omega_i (local order: omega asc., then Gamma asc.)."""
    n = agg.shape[0]
    T = sp.csr_matrix((np.ones(n, dtype=np.int32), (np.arange(n), agg)), shape=(n, nagg))
    mask = T.tocsc()
    A = adj.astype(np.int32)
    for _ in range(overlap):
        mask = (A @ mask).tocsc()
        mask.data[:] = 1
    mask.sort_indices()
    omegas, gammas, Omegas = [], [], []
    order = np.argsort(agg, kind="stable")
    starts = np.searchsorted(agg[order], np.arange(nagg + 1))
    for i in range(nagg):
        om = np.sort(order[starts[i]:starts[i + 1]]).astype(np.int64)
        allnodes = mask.indices[mask.indptr[i]:mask.indptr[i + 1]].astype(np.int64)
        ga = np.setdiff1d(allnodes, om, assume_unique=True)
        omegas.append(om)
        gammas.append(ga)
        Omegas.append(np.concatenate([om, ga]))
    return omegas, gammas, Omegas


def multiplicity_and_nz(sups, agg, nagg):
    """M(l) and nz_i of the Lemma (Section 3.1), per row group.

    M counts the distinct (nonoverlapping) aggregates omega_k that the row's
    support touches, i.e. M(l) = |{k : l in nz_k}| with nz_k the rows that
    are nonzero on omega_k (the reading under which the splitting sums back
    to A).  Returns (M, nz, touched) with touched[g] the sorted aggregate ids
    of group g and nz[i] the ascending group ids in nz_i.
    """
    touched = [np.unique(agg[s]) for s in sups]
    M = np.array([t.shape[0] for t in touched], dtype=np.int64)
    rows = np.repeat(np.arange(len(sups)), M)
    cols = np.concatenate(touched) if touched else np.zeros(0, dtype=np.int64)
    F = sp.csc_matrix((np.ones(rows.shape[0], dtype=np.int8), (rows, cols)), shape=(len(sups), nagg))
    F.sort_indices()
    nz = [F.indices[F.indptr[i]:F.indptr[i + 1]].astype(np.int64) for i in range(nagg)]
    return M, nz, touched


def standard_aggregation(sups, n, passes=1):
    """Level-0 aggregates from the graph of A itself, no strength of connection
    (Section 3.3: the standard routine on the matrix entries), repeated
    `passes` times on the aggregates (aggregating aggregates): T_1 from the
    graph of A, T_2 from the graph of T_1^T A T_1, and so on; the aggregation
    matrix is T_1 T_2 ...  Returns (agg, nagg) with ids in creation order of
    the last pass."""
    if passes < 1:
        raise ValueError("passes must be >= 1")
    adj = structural_adjacency(sups, n).astype(np.int32)
    off = adj.copy()
    off.setdiag(0)
    off.eliminate_zeros()
    off.sort_indices()
    agg, nagg = vanek_aggregation(off)
    for _ in range(passes - 1):
        T = sp.csr_matrix((np.ones(n, dtype=np.int32), (np.arange(n), agg)), shape=(n, nagg))
        C = (T.T @ adj @ T).tocsr()
        C.setdiag(0)
        C.eliminate_zeros()
        C.sort_indices()
        bagg, nagg = vanek_aggregation(C)
        agg = bagg[agg]
    return agg.astype(np.int64), int(nagg)


def subdomain_colouring(Omega, adj, n):
    """Greedy colouring of the overlapping subdomains Omega_i (Section 3.4's n_color).

    Reading: Omega_i and Omega_j need distinct colours when A couples them, i.e.
    A(Omega_i, Omega_j) has a structural nonzero (the A-orthogonality of
    same-coloured subdomains in the cited bound); sharing a node is such a
    coupling since A's diagonal is nonzero.  Subdomains are coloured in
    ascending index, each with the smallest colour no earlier coupled subdomain
    holds.  Returns (colour per subdomain, number of colours)."""
    nagg = len(Omega)
    if nagg == 0:
        return np.zeros(0, dtype=np.int64), 0
    rows = np.concatenate([np.full(o.shape[0], i, dtype=np.int64) for i, o in enumerate(Omega)])
    cols = np.concatenate(Omega).astype(np.int64)
    T = sp.csr_matrix((np.ones(rows.shape[0], dtype=np.int32), (rows, cols)), shape=(nagg, n))
    C = (T @ adj.astype(np.int32) @ T.T).tocsr()
    colour = np.full(nagg, -1, dtype=np.int64)
    for i in range(nagg):
        nb = C.indices[C.indptr[i]:C.indptr[i + 1]]
        used = {int(colour[j]) for j in nb if j < i}
        c = 0
        while c in used:
            c += 1
        colour[i] = c
    return colour, int(colour.max()) + 1


def kappa_threshold(kappa, n_color, n_mult):
    """Local eigenvalue threshold from a target condition number (Section 3.4):
    max{0.1, (kappa - n_color) / (n_color n_multiplicity)}."""
    return max(0.1, (kappa - n_color) / (n_color * n_mult))


def vanek_aggregation(adj_nodiag):
    """Standard aggregation with every edge strong (Section 2.1).

    Pass 1: visit nodes in ascending order; an unaggregated node whose
    neighbours are all unaggregated becomes a root, and root + neighbours
    form a new aggregate.  Pass 2: every node still unaggregated joins the
    aggregate of its lowest-index neighbour that was aggregated in pass 1.
    Pass 3: any node left (possible only without such a neighbour) starts a
    new aggregate with its still-unaggregated neighbours.  Aggregate ids are
    numbered in creation order.
    """
    A = adj_nodiag.tocsr()
    n = A.shape[0]
    agg = -np.ones(n, dtype=np.int64)
    nxt = 0
    for j in range(n):
        if agg[j] >= 0:
            continue
        nb = A.indices[A.indptr[j]:A.indptr[j + 1]]
        nb = nb[nb != j]
        if np.all(agg[nb] < 0):
            agg[j] = nxt
            agg[nb] = nxt
            nxt += 1
    after1 = agg.copy()
    for j in range(n):
        if agg[j] >= 0:
            continue
        nb = np.sort(A.indices[A.indptr[j]:A.indptr[j + 1]])
        nb = nb[nb != j]
        cand = nb[after1[nb] >= 0]
        if cand.size:
            agg[j] = after1[cand[0]]
    for j in range(n):
        if agg[j] >= 0:
            continue
        nb = A.indices[A.indptr[j]:A.indptr[j + 1]]
        nb = nb[(nb != j) & (agg[nb] < 0)]
        agg[j] = nxt
        agg[nb] = nxt
        nxt += 1
    return agg, nxt
