"""Pins of the oracle's coarse-level structure and of its metrics.

Coarse aggregation (Algorithm 1, aggregation step on levels >= 1, read as the
block graph of the previous level's aggregates).  The oracle builds the block
graph from its row-group bookkeeping (`touched`, the aggregates a row group
covers).  Here the same graph is rebuilt from the literal structural pattern
of G_l = G_{l-1} P_{l-1}: the dense m x n pattern of G_0, multiplied as
Boolean matrices by the block pattern of P (row j of P_{l-1} spans the
columns of the aggregate that owns j, Eq. mg-p), level after level.  Two
coarse blocks (previous-level aggregates that kept k_i > 0 columns,
numbered in ascending order) are adjacent when one row of G_l has columns in
both.  Standard aggregation of that graph, spread over each block's columns,
must reproduce the oracle's coarse aggregates id for id.  The same literal
pattern also fixes the row supports of G_l and the pattern of A_l = G_l^T G_l.

Metrics (Section 4): the operator complexity sum_l nnz(A_l) / nnz(A_0) against
a hand count on a two-level block hierarchy (the 9-point pattern on level 0,
the king's-move pattern of 4 x 4 blocks on level 1, each coupling of blocks
a, b contributing k_a k_b entries), and the average convergence factor
(||r_k|| / ||r_0||)^{1/k} against residual norms recomputed from the iterate.
Planted mistakes show that each pin catches its plausible error.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import oracle.construct as oconstruct
import oracle.cycle as ocycle
from inputs import block_aggregates_2d, q1_2d, rotated_sqrtK, seeded_rhs
from inputs.fd import fd_2d, fd_block_aggregates
from oracle.structure import vanek_aggregation
from tests import _brute


def _q1_case(bs, overlap):
    p = q1_2d(16, rotated_sqrtK(math.pi / 6, 1e-2), agg=block_aggregates_2d(16, bs))
    return p, dict(overlap=overlap, coarse_overlap=1, c_min=(2, 3, 4), n_coarse=10, L_max=5)


def _fd_k0_case():
    # isotropic finite differences with kappa = 50: 11 of the 36 level-0 blocks keep no vector
    p = fd_2d(16, math.pi / 6, 1.0, agg=fd_block_aggregates(16, 3))
    return p, dict(overlap=1, c_min=(2, 3, 4), n_coarse=20, kappa=50.0)


# q1_ov3: three hops of overlap around 2 x 2 blocks reach blocks that share no row, so an overlap-based
# block graph differs from the row-based one there
CASES = {"q1_ov1": lambda: _q1_case(4, 1), "q1_ov3": lambda: _q1_case(2, 3), "fd_k0": _fd_k0_case}


def _block_pattern_of_P(level):
    """Structural pattern of P_l: row j spans the columns col0[a] .. col0[a+1]-1 of a = agg(j)."""
    rows, cols = [], []
    for j in range(level.n):
        a = int(level.agg[j])
        c = np.arange(level.col0[a], level.col0[a + 1])
        rows.append(np.full(c.shape[0], j))
        cols.append(c)
    r = np.concatenate(rows)
    return sp.csr_matrix((np.ones(r.shape[0], dtype=np.int64), (r, np.concatenate(cols))),
                         shape=(level.n, int(level.col0[-1])))


def check_coarse_structure(h, p):
    """Rebuild every coarse level's structure from the literal pattern of G_l; return the levels checked."""
    _, pat0 = _brute.dense_G(p)
    pat = sp.csr_matrix(pat0.astype(np.int64))
    checked = 0
    for lvl in range(1, len(h.levels)):
        prev, cur = h.levels[lvl - 1], h.levels[lvl]
        pat = (pat @ _block_pattern_of_P(prev)).tocsr()
        pat.data[:] = 1
        pat = pat[np.diff(pat.indptr) > 0]  # rows touching only k_i = 0 aggregates vanish
        pat.sort_indices()
        # row supports of G_l and the pattern of A_l
        sups = {tuple(pat.indices[pat.indptr[r]:pat.indptr[r + 1]].tolist()) for r in range(pat.shape[0])}
        assert sups == {tuple(int(v) for v in s) for s in cur.sups}, lvl
        A_pat = (pat.T @ pat).tocsr()
        A_pat.sort_indices()
        Ao = cur.A.tocsr()
        Ao.sort_indices()
        assert np.array_equal(A_pat.indptr, Ao.indptr) and np.array_equal(A_pat.indices, Ao.indices), lvl
        if lvl == len(h.levels) - 1:
            break  # the coarsest level is not aggregated
        # coarse blocks: the previous level's aggregates with k > 0, ascending
        live = np.flatnonzero(prev.k > 0)
        block_of_col = np.repeat(np.arange(live.shape[0]), prev.k[live])
        nb = live.shape[0]
        B = np.zeros((nb, nb), dtype=bool)
        for r in range(pat.shape[0]):
            blocks = np.unique(block_of_col[pat.indices[pat.indptr[r]:pat.indptr[r + 1]]])
            B[np.ix_(blocks, blocks)] = True
        np.fill_diagonal(B, False)
        bagg, nagg = vanek_aggregation(sp.csr_matrix(B.astype(np.int8)))
        assert cur.nagg == nagg, lvl
        assert np.array_equal(np.asarray(cur.agg), bagg[block_of_col]), lvl
        checked += 1
    return checked


@pytest.mark.parametrize("name", sorted(CASES))
def test_coarse_aggregates_follow_the_literal_block_graph(name):
    p, kw = CASES[name]()
    h = oracle.setup(p.rowptr, p.col, p.val, p.n, p.D1, p.agg, **kw)
    assert len(h.levels) >= 3
    if name == "fd_k0":
        assert any(np.any(L.k == 0) for L in h.levels[:-2]), "the case must drop blocks with k_i = 0"
    assert check_coarse_structure(h, p) >= 1


def _omega_edges(prev):
    """Planted mistake: blocks adjacent when Omega_a meets omega_b (overlap, not a shared row)."""
    live = np.flatnonzero(prev.k > 0)
    new_id = -np.ones(prev.nagg, dtype=np.int64)
    new_id[live] = np.arange(live.shape[0])
    nb = live.shape[0]
    B = np.zeros((nb, nb), dtype=bool)
    for a in live:
        for b in np.unique(prev.agg[prev.Omega[a]]):
            if new_id[b] >= 0:
                B[new_id[a], new_id[b]] = B[new_id[b], new_id[a]] = True
    np.fill_diagonal(B, False)
    bagg, nagg = vanek_aggregation(sp.csr_matrix(B.astype(np.int8)))
    return np.repeat(bagg, prev.k[live]), nagg


def _dead_blocks_kept(prev):
    """Planted mistake: blocks with k_i = 0 stay vertices of the block graph."""
    r, c = [], []
    for t in prev.touched:
        if t.shape[0] > 1:
            r.append(np.repeat(t, t.shape[0]))
            c.append(np.tile(t, t.shape[0]))
    B = sp.csr_matrix((np.ones(sum(x.shape[0] for x in r), dtype=np.int8), (np.concatenate(r), np.concatenate(c))),
                      shape=(prev.nagg, prev.nagg))
    B.setdiag(0)
    B.eliminate_zeros()
    bagg, nagg = vanek_aggregation(B)
    return np.repeat(bagg, prev.k), nagg


@pytest.mark.parametrize("mutant,name", [(_omega_edges, "q1_ov3"), (_dead_blocks_kept, "fd_k0")])
def test_planted_block_graph_mistakes_are_caught(monkeypatch, mutant, name):
    p, kw = CASES[name]()
    monkeypatch.setattr(oconstruct, "_block_aggregation", mutant)
    try:
        h = oracle.setup(p.rowptr, p.col, p.val, p.n, p.D1, p.agg, **kw)
    except Exception:
        return  # the mistake broke the construction outright
    with pytest.raises(AssertionError):
        check_coarse_structure(h, p)


# ---------------------------------------------------------------- metrics ---

def check_operator_complexity(metrics_fn):
    N, bs = 16, 4
    p = q1_2d(N, rotated_sqrtK(math.pi / 6, 1e-2), agg=block_aggregates_2d(N, bs))
    h = oracle.setup(p.rowptr, p.col, p.val, p.n, p.D1, p.agg, overlap=1, c_min=(2,), n_coarse=200, L_max=2)
    assert len(h.levels) == 2
    n_side = N - 1
    nnz0 = (3 * n_side - 2) ** 2  # 9-point pattern: per axis n + 2(n - 1) index pairs
    nbs = -(-n_side // bs)
    k = np.asarray(h.levels[0].k).reshape(nbs, nbs)  # aggregate id = I + nbs J: row J, column I
    nnz1 = 0
    for J in range(nbs):
        for I in range(nbs):
            for J2 in range(max(J - 1, 0), min(J + 2, nbs)):
                for I2 in range(max(I - 1, 0), min(I + 2, nbs)):
                    nnz1 += int(k[J, I]) * int(k[J2, I2])
    m = metrics_fn(h)
    assert m["nnz"] == [nnz0, nnz1]
    assert abs(m["op_complexity"] - (nnz0 + nnz1) / nnz0) <= 1e-15 * (nnz0 + nnz1) / nnz0


def _one_level():
    """A stand-in hierarchy with one 1 x 1 level, for hand-made residual histories."""
    lvl = type("L", (), {"A": sp.identity(1, format="csr"), "n": 1})()
    return type("H", (), {"levels": [lvl]})()


def check_convergence_factor(metrics_fn):
    m = metrics_fn(_one_level(), dict(iters=4, relres=1e-4))
    assert abs(m["rho"] - 0.1) <= 1e-14 and abs(m["iters_per_digit"] - 1.0) <= 1e-12
    p = q1_2d(12, rotated_sqrtK(math.pi / 6, 1e-2), agg=block_aggregates_2d(12, 3))
    h = oracle.setup(p.rowptr, p.col, p.val, p.n, p.D1, p.agg, overlap=1, c_min=(3,), n_coarse=30)
    b = seeded_rhs(p.n, 1, 2)[:, 0]
    G, _ = _brute.dense_G(p)
    A = G.T @ G
    for k in (2, 3, 5):
        x, info = oracle.pcg(h, b, tol=1e-30, maxit=k)
        assert info["iters"] == k
        rho = (np.linalg.norm(b - A @ x) / np.linalg.norm(b)) ** (1.0 / k)
        m = metrics_fn(h, info)
        assert abs(m["rho"] - rho) <= 1e-8 * rho, k
        assert abs(m["iters_per_digit"] - math.log(0.1) / math.log(rho)) <= 1e-6, k


def test_operator_complexity_matches_a_hand_count():
    check_operator_complexity(ocycle.metrics)


def test_convergence_factor_matches_recomputed_residuals():
    check_convergence_factor(ocycle.metrics)


def test_planted_metric_mistakes_are_caught():
    def oc_over_coarsest(h, info=None):
        m = ocycle.metrics(h, info)
        m["op_complexity"] = sum(m["nnz"]) / m["nnz"][-1]
        return m

    def rho_not_averaged(h, info=None):
        m = ocycle.metrics(h, info)
        if "rho" in m:
            m["rho"] = info["relres"] ** info["iters"]
        return m

    with pytest.raises(AssertionError):
        check_operator_complexity(oc_over_coarsest)
    with pytest.raises(AssertionError):
        check_convergence_factor(rho_not_averaged)
