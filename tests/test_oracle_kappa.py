"""Pins of the kappa-derived eigenvalue threshold (Section 3.4).

* the colouring is proper (subdomains coupled by A differ) and greedy (a subdomain of colour c has, for
  every c' < c, an earlier coupled subdomain of colour c'), against a brute-force coupling test on the
  dense A;
* the 2D finite-difference workload with 4x4 aggregates: the subdomain graph is the king's graph of the
  blocks (the stencil's (i+1, j)-(i, j+1) coupling reaches the diagonal blocks, two blocks apart nothing
  couples), which needs 4 colours; a row of G spans 3 nodes that can sit in 3 blocks, so n_multiplicity = 3
  and thresh = (50 - 4) / (4 * 3);
* one aggregate: n_color = n_multiplicity = 1, thresh = kappa - 1;
* the 0.1 floor binds when kappa <= n_color;
* with kappa, setup keeps exactly the eigenpairs with lambda > thresh (below the cap).
"""
import math

import numpy as np
import pytest

import oracle
from oracle.structure import kappa_threshold, structural_adjacency, subdomain_colouring
from oracle.construct import row_groups_from_csr
from oracle.structure import cleanup_aggregates, overlapping_subdomains
from inputs import fd_2d, fd_block_aggregates, q1_2d, rotated_sqrtK, block_aggregates_2d


def _subdomains(p, overlap=1):
    sups, _ = row_groups_from_csr(p.rowptr, p.col, p.val, p.n, p.D1)
    adj = structural_adjacency(sups, p.n)
    agg, nagg = cleanup_aggregates(p.agg, adj)
    _, _, Om = overlapping_subdomains(agg, nagg, adj, overlap)
    return Om, adj


def _dense_coupled(p, Om):
    Gs = np.zeros((p.m, p.n), dtype=bool)  # structural: every listed entry counts
    for r in range(p.m):
        Gs[r, p.col[p.rowptr[r]:p.rowptr[r + 1]]] = True
    Ad = (Gs.T.astype(int) @ Gs.astype(int) + np.eye(p.n, dtype=int)) > 0
    k = len(Om)
    C = np.zeros((k, k), dtype=bool)
    for i in range(k):
        for j in range(k):
            C[i, j] = Ad[np.ix_(Om[i], Om[j])].any()
    return C


@pytest.mark.parametrize("make", [lambda: fd_2d(13, 0.5, 1e-3, agg=fd_block_aggregates(13, 3)),
                                  # 2x2 blocks: many subdomain pairs are coupled by A without sharing a node
                                  # (9 colours; a colouring by shared nodes alone needs 4)
                                  lambda: fd_2d(13, 0.5, 1e-3, agg=fd_block_aggregates(13, 2)),
                                  lambda: q1_2d(12, rotated_sqrtK(0.4, 1e-3), agg=block_aggregates_2d(12, 3))])
def test_colouring_is_proper_and_greedy(make):
    p = make()
    Om, adj = _subdomains(p)
    col, nc = subdomain_colouring(Om, adj, p.n)
    C = _dense_coupled(p, Om)
    assert nc == col.max() + 1
    for i in range(len(Om)):
        for j in range(len(Om)):
            if i != j and C[i, j]:
                assert col[i] != col[j]
        for c in range(col[i]):
            assert any(C[i, j] and col[j] == c for j in range(i))


def test_fd_blocks_need_four_colours_and_multiplicity_three():
    N = 16
    p = fd_2d(N, math.pi / 6, 1e-4, agg=fd_block_aggregates(N, 4))
    h = oracle.setup(p.rowptr, p.col, p.val, p.n, p.D1, p.agg, overlap=1, c_min=(2,), n_coarse=1, L_max=2,
                     kappa=50.0)
    L0 = h.levels[0]
    assert (L0.n_color, L0.n_mult) == (4, 3)
    assert L0.thresh == (50.0 - 4) / 12


def test_single_aggregate():
    # (setup itself stops there: with one subdomain S~ = A_ww, every lambda = 1 < 19 and k = 0)
    from oracle.structure import multiplicity_and_nz

    N = 6
    p = fd_2d(N, 0.3, 1e-2, agg=fd_block_aggregates(N, N))
    Om, adj = _subdomains(p)
    _, nc = subdomain_colouring(Om, adj, p.n)
    sups, _ = row_groups_from_csr(p.rowptr, p.col, p.val, p.n, p.D1)
    M, _, _ = multiplicity_and_nz(sups, p.agg.astype(np.int64), 1)
    assert (nc, int(M.max()), kappa_threshold(20.0, nc, int(M.max()))) == (1, 1, 19.0)


def test_floor():
    assert kappa_threshold(3.0, 4, 3) == 0.1
    assert kappa_threshold(4.0, 4, 3) == 0.1
    assert kappa_threshold(50.0, 5, 9) == 1.0


def test_selection_follows_derived_threshold():
    N = 16
    p = fd_2d(N, math.pi / 6, 1e-4, agg=fd_block_aggregates(N, 4))
    h = oracle.setup(p.rowptr, p.col, p.val, p.n, p.D1, p.agg, overlap=1, c_min=(2,), n_coarse=1, L_max=2,
                     kappa=50.0)
    L0 = h.levels[0]
    for i in range(L0.nagg):
        mu = L0.mu[i]
        lam = np.where(mu > 0, 1.0 / np.where(mu > 0, mu, 1.0), np.inf)
        want = min(int(np.sum(lam > L0.thresh)), max(1, L0.omega[i].shape[0] // 2))
        assert L0.Z[i].shape[1] == want


def test_aggregates_without_coarse_vectors():
    """Isotropic 16 x 16 with kappa = 50: some aggregates keep k_i = 0 (no lambda above the threshold).
    They add no coarse dofs, rows touching only them vanish from G_{l+1}, they are left out of the block
    graph, and A_{l+1} is still P_l^T A_l P_l."""
    from oracle.structure import standard_aggregation
    from inputs import seeded_rhs

    p = fd_2d(16, math.pi / 6, 1.0)
    sups, _ = row_groups_from_csr(p.rowptr, p.col, p.val, p.n, p.D1)
    agg, _ = standard_aggregation(sups, p.n, 1)
    h = oracle.setup(p.rowptr, p.col, p.val, p.n, p.D1, agg, overlap=1, c_min=(2, 3, 4), n_coarse=20, kappa=50.0)
    assert any(np.any(L.k == 0) for L in h.levels[:-1])
    for lvl in range(len(h.levels) - 1):
        L, Ln = h.levels[lvl], h.levels[lvl + 1]
        assert Ln.n == int(L.k.sum()) == L.P.shape[1]
        ref = (L.P.T @ L.A @ L.P).toarray()
        assert np.abs(Ln.A.toarray() - ref).max() <= 1e-13 * np.abs(ref).max()
        for i in np.flatnonzero(L.k == 0):
            assert L.P[L.omega[i]].nnz == 0
    x, info = oracle.pcg(h, seeded_rhs(p.n, 1, 1)[:, 0], tol=1e-8)
    assert info["status"] == 0 and info["relres_true"] <= 1e-8


def test_empty_coarse_space_is_an_error():
    from oracle.structure import standard_aggregation

    p = fd_2d(20, math.pi / 6, 1.0)
    sups, _ = row_groups_from_csr(p.rowptr, p.col, p.val, p.n, p.D1)
    agg, _ = standard_aggregation(sups, p.n, 1)
    with pytest.raises(ValueError, match="empty coarse space"):
        oracle.setup(p.rowptr, p.col, p.val, p.n, p.D1, agg, overlap=1, c_min=(2, 3, 4), n_coarse=20, kappa=50.0)


def test_two_level_with_threshold_selection_is_size_independent():
    """With every local eigenvector above the kappa threshold kept (cap |omega_i|, c_min = 1), the two-level
    method's PCG count does not grow with the grid (the GenEO-type bound behind Section 3.4's formula depends
    on n_color, n_multiplicity and thresh only): 48^2, 64^2 and 96^2 all take 12 iterations to 1e-8."""
    from oracle.structure import standard_aggregation
    from inputs import seeded_rhs

    its = []
    for N in (48, 64, 96):
        p = fd_2d(N, math.pi / 6, 1e-5)
        sups, _ = row_groups_from_csr(p.rowptr, p.col, p.val, p.n, p.D1)
        agg, _ = standard_aggregation(sups, p.n, 1)
        h = oracle.setup(p.rowptr, p.col, p.val, p.n, p.D1, agg, overlap=1, c_min=(1,), L_max=2, n_coarse=1,
                         kappa=50.0)
        _, info = oracle.pcg(h, seeded_rhs(p.n, 1, 6)[:, 0], tol=1e-8)
        its.append(info["iters"])
    assert max(its) - min(its) <= 1 and max(its) <= 14, its


def test_two_level_with_threshold_selection_is_angle_robust():
    """The same two-level method across the anisotropy angle (theta = 0, pi/6, pi/4 on 48^2 at eps = 1e-5): the
    bound does not see theta, and the PCG counts stay within 10-18 (12-15 here; a Schur complement that ignores
    the Gamma rows takes 320-1000)."""
    from oracle.structure import standard_aggregation
    from inputs import seeded_rhs

    for theta in (0.0, math.pi / 6, math.pi / 4):
        p = fd_2d(48, theta, 1e-5)
        sups, _ = row_groups_from_csr(p.rowptr, p.col, p.val, p.n, p.D1)
        agg, _ = standard_aggregation(sups, p.n, 1)
        h = oracle.setup(p.rowptr, p.col, p.val, p.n, p.D1, agg, overlap=1, c_min=(1,), L_max=2, n_coarse=1,
                         kappa=50.0)
        _, info = oracle.pcg(h, seeded_rhs(p.n, 1, 6)[:, 0], tol=1e-8)
        assert 10 <= info["iters"] <= 18, (theta, info["iters"])
