"""Pins of the row form of the Schur complement (Eq. gevp-S) and of G_{l+1} = G_l P_l carried as rows.

* the rows carried to level 1 reproduce that level's Grams, and the stacked weighted rows of a subdomain
  reproduce the Gram-route splitting A~_i (the Lemma), to rounding;
* on a Q1 workload, where the pseudo-inverse has a clean gap, the row route builds the same hierarchy as the
  Gram route: equal k_i, local eigenvalues within 1e-10, A_l within 1e-12;
* on the finite-difference workload the first coarse level has singular values of W^(1/2) G_Gamma near 4e-7
  (eigenvalues near 1.5e-13 of A~_GG): the row route's spectrum there does not move when its cut moves over six
  orders (1e-8 .. 1e-14), while the Gram route's spectrum changes at the first decimal between cuts of 1e-12 and
  1e-13.
"""
import math

import numpy as np

import oracle
from oracle.construct import local_splitting, local_splitting_rows
from inputs import block_aggregates_2d, fd_2d, fd_block_aggregates, q1_2d, rotated_sqrtK


def _fd48(**kw):
    p = fd_2d(48, math.pi / 6, 1e-4, agg=fd_block_aggregates(48, 4))
    return oracle.setup(p.rowptr, p.col, p.val, p.n, p.D1, p.agg, overlap=1, c_min=(2, 3, 4), n_coarse=100,
                        keep_local=True, kappa=50.0, L_max=3, **kw)


def test_rows_reproduce_grams_and_splitting():
    h = _fd48(schur="rows")
    for L in h.levels[:2]:
        for R, H in zip(L.rows, L.grams):
            assert np.abs(R.T @ R - H).max() <= 1e-13 * max(np.abs(H).max(), 1e-300)
    L = h.levels[1]
    for i in range(0, L.nagg, 3):
        Y = local_splitting_rows(L.Omega[i], L.nz[i], L.sups, L.rows, L.M)
        At = local_splitting(L.Omega[i], L.nz[i], L.sups, L.grams, L.M)
        assert np.abs(Y.T @ Y - At).max() <= 1e-13 * np.abs(At).max()


def test_rows_match_gram_route_on_clean_gap():
    p = q1_2d(23, rotated_sqrtK(0.4, 1e-2), agg=block_aggregates_2d(23, 4))
    kw = dict(overlap=1, c_min=(2, 3), n_coarse=40)
    hg = oracle.setup(p.rowptr, p.col, p.val, p.n, p.D1, p.agg, schur="gram", **kw)
    hr = oracle.setup(p.rowptr, p.col, p.val, p.n, p.D1, p.agg, schur="rows", **kw)
    assert [L.n for L in hg.levels] == [L.n for L in hr.levels]
    for Lg, Lr in zip(hg.levels, hr.levels):
        A = Lg.A.toarray()
        assert np.abs(Lr.A.toarray() - A).max() <= 1e-12 * np.abs(A).max()
        if Lg.k is None:
            continue
        assert np.array_equal(Lg.k, Lr.k)
        for mg, mr in zip(Lg.mu, Lr.mu):
            assert np.abs(mg - mr).max() <= 1e-10


def test_rows_route_is_stable_where_gram_route_is_not():
    base = _fd48(schur="rows", sv_rtol=1e-10).levels[1].mu[0]
    for sv in (1e-8, 1e-12, 1e-14):
        assert np.abs(_fd48(schur="rows", sv_rtol=sv).levels[1].mu[0] - base).max() <= 1e-9
    g12 = _fd48(schur="gram", schur_rtol=1e-12).levels[1].mu[0]
    g13 = _fd48(schur="gram", schur_rtol=1e-13).levels[1].mu[0]
    assert np.abs(g12 - g13).max() > 1e-2
    assert np.abs(g13 - base).max() <= 1e-4  # the Gram route's finer cut lands near the row answer


def test_schur_is_the_least_squares_minimum():
    """u^T S~ u = min_v ||X u + Y_G v||^2 (the shorted operator of A~_i onto omega_i), by a least-squares
    solve per random u: no projector, no Gram, no pseudo-inverse."""
    from oracle.construct import local_splitting_rows

    h = _fd48(schur="rows")
    rng = np.random.default_rng(7)
    for lvl in (0, 1):
        L = h.levels[lvl]
        for i in range(0, L.nagg, 5):
            no = L.omega[i].shape[0]
            Y = local_splitting_rows(L.Omega[i], L.nz[i], L.sups, L.rows, L.M)
            X, YG = Y[:, :no], Y[:, no:]
            for _ in range(2):
                u = rng.standard_normal(no)
                if YG.shape[1]:
                    v = np.linalg.lstsq(YG, -X @ u, rcond=None)[0]
                    best = float(np.sum((X @ u + YG @ v) ** 2))
                else:
                    best = float(np.sum((X @ u) ** 2))
                got = float(u @ L.S[i] @ u)
                assert abs(got - best) <= 1e-9 * float(np.sum((X @ u) ** 2)), (lvl, i, got, best)
