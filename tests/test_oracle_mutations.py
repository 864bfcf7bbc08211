"""Planted mistakes in the oracle (CPU only): each must break one pin.

A pin set that still passes after a dropped term, a wrong sign, a wrong
index or a transposed operand would not be worth much; these tests plant
such mistakes with monkeypatch and check that the corresponding invariant
fails.
"""
import math

import numpy as np
import scipy.linalg as sla

import oracle
import oracle.construct as osetup
import oracle.cycle as osolve
import oracle.structure as ostruct
from inputs import block_aggregates_2d, q1_2d, rotated_sqrtK
from tests import _brute


def _prob(N=9, bs=3):
    return q1_2d(N, rotated_sqrtK(math.pi / 6, 1e-2), agg=block_aggregates_2d(N, bs))


def _h(p, **kw):
    kw.setdefault("n_coarse", 10)
    kw.setdefault("L_max", 2)
    return oracle.setup(p.rowptr, p.col, p.val, p.n, p.D1, p.agg, overlap=1, keep_local=True, **kw)


def _lemma_error(h):
    L = h.levels[0]
    A = L.A.toarray()
    S = np.zeros_like(A)
    for i in range(L.nagg):
        S[np.ix_(L.Omega[i], L.Omega[i])] += L.Atil[i]
    return np.abs(S - A).max() / np.abs(A).max()


def test_dropped_multiplicity_breaks_lemma(monkeypatch):
    p = _prob()
    assert _lemma_error(_h(p)) <= 1e-14
    orig = osetup.local_splitting_rows
    monkeypatch.setattr(osetup, "local_splitting_rows",
                        lambda Om, nz, sups, rows, M: orig(Om, nz, sups, rows, np.ones_like(M)))
    assert _lemma_error(_h(p)) > 1e-3


def test_dropped_multiplicity_breaks_lemma_gram_route(monkeypatch):
    p = _prob()
    assert _lemma_error(_h(p, schur="gram")) <= 1e-14
    orig = osetup.local_splitting
    monkeypatch.setattr(osetup, "local_splitting",
                        lambda Om, nz, sups, grams, M: orig(Om, nz, sups, grams, np.ones_like(M)))
    assert _lemma_error(_h(p, schur="gram")) > 1e-3


def test_schur_sign_error_breaks_svd_pin(monkeypatch):
    p = _prob()

    def bad(Y, no, sv_rtol=None):  # the projected part added instead of removed
        X, YG = Y[:, :no], Y[:, no:]
        if YG.shape[1] == 0:
            return X.T @ X
        U, sv, _ = np.linalg.svd(YG, full_matrices=False)
        Uk = U[:, sv > 1e-12 * sv.max()]
        T = Uk.T @ X
        return X.T @ X + T.T @ T

    monkeypatch.setattr(osetup, "schur_complement_rows", bad)
    h = _h(p)
    L = h.levels[0]
    G, P = _brute.dense_G(p)
    worst = max(np.abs(L.S[i] - _brute.svd_schur(G, P, L.agg, i, L.omega[i], L.gamma[i])).max()
                / np.abs(L.Ai[i]).max() for i in range(L.nagg))
    assert worst > 1e-3


def test_swapped_gep_operands_break_mu_range(monkeypatch):
    p = _prob()
    orig = osetup.sla.eigh

    def swapped(a, b=None, **kw):
        return orig(b, a + 1e-12 * np.eye(a.shape[0]), **kw) if b is not None else orig(a, **kw)

    monkeypatch.setattr(osetup.sla, "eigh", swapped)
    h = _h(p)
    L = h.levels[0]
    assert max(m.max() for m in L.mu) > 1 + 1e-6


def test_ras_t_with_pou_on_wrong_side_breaks_adjointness(monkeypatch):
    p = _prob()
    h = _h(p)
    L = h.levels[0]
    rng = np.random.default_rng(0)
    x, y = rng.standard_normal(p.n), rng.standard_normal(p.n)
    assert abs(osolve.ras(L, x) @ y - x @ osolve.rast(L, y)) <= 1e-11
    monkeypatch.setattr(osolve, "rast", osolve.ras)
    assert abs(osolve.ras(L, x) @ y - x @ osolve.rast(L, y)) > 1e-6


def test_missing_overlap_hop_breaks_bfs_pin():
    p = _prob()
    sups, grams = ostruct.row_groups_from_csr(p.rowptr, p.col, p.val, p.n, p.D1)
    adj = ostruct.structural_adjacency(sups, p.n)
    agg, nagg = ostruct.cleanup_aggregates(p.agg, adj)
    _, ga0, _ = ostruct.overlapping_subdomains(agg, nagg, adj, 0)
    G, P = _brute.dense_G(p)
    ref = _brute.omega_sets(P, agg, 1)
    assert any(not np.array_equal(ga0[i], ref[i][1]) for i in range(nagg))


def test_permuted_coarse_columns_break_galerkin(monkeypatch):
    p = q1_2d(12, rotated_sqrtK(0.4, 0.05), agg=block_aggregates_2d(12, 3))
    for route, name in (("rows", "_next_groups_rows"), ("gram", "_next_groups")):
        orig = getattr(osetup, name)

        def permuted(level, orig=orig):
            # wrong index: coarse columns of every block reversed while propagating G
            good = level.Z
            level.Z = [Z[:, ::-1] for Z in good]
            try:
                return orig(level)
            finally:
                level.Z = good

        monkeypatch.setattr(osetup, name, permuted)
        h = oracle.setup(p.rowptr, p.col, p.val, p.n, p.D1, p.agg, overlap=1, c_min=(3,), n_coarse=5, L_max=2,
                         schur=route)
        P = h.levels[0].P.toarray()
        gal = P.T @ h.levels[0].A.toarray() @ P
        assert np.abs(h.levels[1].A.toarray() - gal).max() > 1e-6 * np.abs(gal).max(), route


def test_transposed_local_factor_breaks_exact_single_block(monkeypatch):
    p = q1_2d(7, rotated_sqrtK(0.3, 0.1), agg=np.zeros(36, dtype=np.int32))
    h = oracle.setup(p.rowptr, p.col, p.val, p.n, p.D1, p.agg, n_coarse=1, L_max=2)
    L = h.levels[0]
    r = np.random.default_rng(1).standard_normal(p.n)
    ref = np.linalg.solve(L.A.toarray(), r)
    monkeypatch.setattr(osolve, "_local_solve", lambda Lf, v: sla.cho_solve((Lf.T, True), v))
    assert np.abs(osolve.ras(L, r) - ref).max() > 1e-6 * np.abs(ref).max()
