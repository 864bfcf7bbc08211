"""Pins of the oracle's numeric setup.

* Lemma (Section 3.1): sum_i R_i^T A~_i R_i = A, every A~_i SPSD, and A~_i
  equal to the literal row-by-row W-weighted Gram of the rows in nz_i;
* Eq. gevp-S: S~ equal to X^T (I - Pi_Y) X computed from the literal rows
  with an SVD projector (an independent route to the Schur complement),
  S~ SPSD, S~ 1 = 0 on interior aggregates when D1 = 0;
* local GEP: mu in [0, 1] (S~ <= A~_ww <= A_ww since W <= I, so every
  lambda >= 1 and thresh = 0.1 never binds), Z^T A_ww Z = I, eigen-residual,
  the local constant in range(Z) on interior aggregates;
* Eq. mg-p: columns of P have disjoint supports, one block per row;
* multilevel propagation: A_1 built from the grouped rows equals the literal
  (G_0 P_0)^T (G_0 P_0) and the Galerkin product P_0^T A_0 P_0.
"""
import math

import numpy as np
import pytest

import oracle
from inputs import block_aggregates_2d, q1_2d, rotated_sqrtK
from oracle.construct import local_gep
from tests import _brute


def _prob(N=9, bs=3, d1=None, theta=math.pi / 6, eps=1e-2):
    D1 = None if d1 is None else np.full((N - 1) ** 2, d1)
    return q1_2d(N, rotated_sqrtK(theta, eps), D1=D1, agg=block_aggregates_2d(N, bs))


def _setup(p, overlap=1, **kw):
    kw.setdefault("n_coarse", 10)
    kw.setdefault("L_max", 2)
    return oracle.setup(p.rowptr, p.col, p.val, p.n, p.D1, p.agg, overlap=overlap, keep_local=True, **kw)


CASES = [dict(), dict(d1=0.2), dict(theta=0.0, eps=1.0), dict(theta=math.pi / 4, eps=1e-6)]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("overlap", [1, 2])
def test_lemma_splitting(case, overlap):
    p = _prob(**case)
    h = _setup(p, overlap)
    L = h.levels[0]
    A = L.A.toarray()
    S = np.zeros_like(A)
    G, P = _brute.dense_G(p)
    for i in range(L.nagg):
        Om = L.Omega[i]
        S[np.ix_(Om, Om)] += L.Atil[i]
        At = L.Atil[i]
        w = np.linalg.eigvalsh(At)
        assert w.min() >= -1e-14 * max(w.max(), 1e-300)
        ref = _brute.literal_splitting(G, P, L.agg, i, Om)
        assert np.abs(At - ref).max() <= 1e-14 * np.abs(ref).max()
    assert np.abs(S - A).max() <= 1e-14 * np.abs(A).max()
    assert np.abs(A - G.T @ G).max() <= 1e-14 * np.abs(A).max()


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("overlap", [1, 2])
def test_schur_against_svd_projection(case, overlap):
    p = _prob(**case)
    h = _setup(p, overlap)
    L = h.levels[0]
    G, P = _brute.dense_G(p)
    for i in range(L.nagg):
        Sref = _brute.svd_schur(G, P, L.agg, i, L.omega[i], L.gamma[i])
        S = L.S[i]
        scale = np.abs(L.Ai[i]).max()
        assert np.abs(S - Sref).max() <= 1e-11 * scale, i
        w = np.linalg.eigvalsh(S)
        assert w.min() >= -1e-12 * scale


def test_schur_annihilates_constants_on_interior_aggregates():
    p = _prob(N=13, bs=3)
    h = _setup(p)
    L = h.levels[0]
    N = 13
    for i in range(L.nagg):
        om = L.omega[i]
        jm1, im1 = np.divmod(om, N - 1)
        if im1.min() == 0 or jm1.min() == 0 or im1.max() == N - 2 or jm1.max() == N - 2:
            continue  # touches the Dirichlet boundary: constants are not local null vectors
        # interior aggregate whose overlap is interior too
        Om = L.Omega[i]
        jo, io = np.divmod(Om, N - 1)
        if io.min() == 0 or jo.min() == 0 or io.max() == N - 2 or jo.max() == N - 2:
            continue
        one = np.ones(om.shape[0])
        assert np.abs(L.S[i] @ one).max() <= 1e-12 * np.abs(L.S[i]).max()
        # the constant is the mu = 0 mode and lies in range(Z)
        Z = L.Z[i]
        Aww = L.Ai[i][:om.shape[0], :om.shape[0]]
        coef = Z.T @ (Aww @ one)
        assert np.linalg.norm(one - Z @ coef) <= 1e-10 * np.linalg.norm(one)


@pytest.mark.parametrize("case", CASES)
def test_gep_properties(case):
    p = _prob(**case)
    h = _setup(p)
    L = h.levels[0]
    for i in range(L.nagg):
        no = L.omega[i].shape[0]
        Aww = L.Ai[i][:no, :no]
        mu, Z = L.mu[i], L.Z[i]
        assert mu.min() >= -1e-12 and mu.max() <= 1 + 1e-12
        assert np.all(np.diff(mu) >= 0)
        k = Z.shape[1]
        assert k == max(1, no // 2)  # thresh 0.1 < 1 <= lambda: the cap decides
        assert np.abs(Z.T @ Aww @ Z - np.eye(k)).max() <= 1e-12
        res = L.S[i] @ Z - Aww @ Z @ np.diag(mu[:k])
        assert np.abs(res).max() <= 1e-12 * np.abs(Aww).max()
        for c in range(k):
            a = np.abs(Z[:, c])
            j = np.nonzero(a >= (1 - 1e-6) * a.max())[0][0]
            assert Z[j, c] > 0


def test_selection_counts_lambda_above_threshold():
    S = np.diag([0.0, 0.3, 0.6, 0.9])
    A = np.eye(4)
    # lambda = 1/mu = inf, 3.33, 1.67, 1.11: thresh 2 keeps two, thresh 1.5 three
    assert local_gep(S, A, 4, 2.0)[1].shape[1] == 2
    assert local_gep(S, A, 4, 1.5)[1].shape[1] == 3
    assert local_gep(S, A, 1, 1.5)[1].shape[1] == 1  # cap binds


def test_interpolation_block_diagonal_and_galerkin():
    p = _prob(N=12, bs=3, d1=0.05)
    h = oracle.setup(p.rowptr, p.col, p.val, p.n, p.D1, p.agg, overlap=1, c_min=(3,), n_coarse=5, L_max=3)
    L0, L1 = h.levels[0], h.levels[1]
    P = L0.P.toarray()
    # disjoint column supports per aggregate; each row hits one block only
    for i in range(L0.nagg):
        cols = np.arange(L0.col0[i], L0.col0[i + 1])
        rows = np.nonzero(np.any(P[:, cols] != 0, axis=1))[0]
        assert set(rows.tolist()) <= set(L0.omega[i].tolist())
    blocks_per_row = [len({int(np.searchsorted(L0.col0, c, side="right") - 1) for c in np.nonzero(P[r])[0]})
                      for r in range(P.shape[0])]
    assert max(blocks_per_row) == 1
    G, _ = _brute.dense_G(p)
    G1 = G @ P
    A1 = L1.A.toarray()
    ref = G1.T @ G1
    assert np.abs(A1 - ref).max() <= 1e-13 * np.abs(ref).max()
    gal = P.T @ L0.A.toarray() @ P
    assert np.abs(A1 - gal).max() <= 1e-13 * np.abs(ref).max()
    # level-1 groups: the literal rows of G_1 with one support sum to that group's Gram
    key = {tuple(s.tolist()): g for g, s in enumerate(L1.sups)}
    acc = [np.zeros_like(H) for H in L1.grams]
    for l in range(G.shape[0]):
        touched = np.unique(L0.agg[np.nonzero(G[l])[0]]) if np.any(G[l]) else None
        if touched is None:
            continue
        cs = np.concatenate([np.arange(L0.col0[a], L0.col0[a + 1]) for a in touched])
        g = key[tuple(cs.tolist())]
        acc[g] += np.outer(G1[l, cs], G1[l, cs])
    for g in range(len(acc)):
        assert np.abs(acc[g] - L1.grams[g]).max() <= 1e-13 * max(np.abs(L1.grams[g]).max(), 1e-300)
