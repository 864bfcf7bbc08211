"""Pins of the oracle's additive two-level method (Section 3.1, after Eq.
cgc): M_2^{-1} = P (P^T A P)^{-1} P^T + M_1^{-1}, with M_1^{-1} additive
Schwarz (Eq. ras without the partition of unity).

* one aggregate covering every node: M_1^{-1} is the exact A^{-1};
* M_1^{-1} and M_2^{-1} are symmetric (dense, from unit vectors);
* M_1^{-1} equals the sum of the local inverses placed on Omega_i, written
  out as dense matrices (an independent assembly);
* the spectral bound the paper quotes: with every eigenvector of the local
  eigenproblem above tau kept (no cap, c_min = 1), the eigenvalues of
  M_2^{-1} A lie in [(2 + (2 k_c + 1) tau)^{-1}, k_c + 1], k_c the number of
  colours of a colouring of the subdomains in which overlapping subdomains
  differ (a greedy colouring gives a valid, possibly larger, k_c);
* with tau below 1 every local eigenvector is kept (lambda >= 1 always),
  P is square and M_2^{-1} A has no eigenvalue below 1 (the coarse part is
  the exact inverse);
* PCG with M_2 converges and reaches the Cholesky solution.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from inputs import block_aggregates_2d, q1_2d, rotated_sqrtK, seeded_rhs
from oracle.cycle import additive_schwarz, two_level_additive


def _two_level(N=12, bs=3, tau=2.0, theta=math.pi / 6, eps=1e-2, overlap=1):
    p = q1_2d(N, rotated_sqrtK(theta, eps), agg=block_aggregates_2d(N, bs))
    h = oracle.setup(p.rowptr, p.col, p.val, p.n, p.D1, p.agg, overlap=overlap, c_min=(1,),
                     n_coarse=1, L_max=2, thresh=tau)
    assert len(h.levels) == 2
    return p, h


def _dense(op, n):
    return np.column_stack([op(e) for e in np.eye(n)])


def _colours(L):
    """Greedy colouring of the subdomains: i ~ j when Omega_i and Omega_j meet."""
    owner = {}
    for i, Om in enumerate(L.Omega):
        for v in Om:
            owner.setdefault(int(v), []).append(i)
    nbr = [set() for _ in range(L.nagg)]
    for lst in owner.values():
        for a in lst:
            nbr[a].update(b for b in lst if b != a)
    col = [-1] * L.nagg
    for i in range(L.nagg):
        used = {col[j] for j in nbr[i] if col[j] >= 0}
        c = 0
        while c in used:
            c += 1
        col[i] = c
    return max(col) + 1


def test_single_aggregate_additive_schwarz_is_exact():
    p = q1_2d(7, rotated_sqrtK(0.3, 0.1), agg=np.zeros(36, dtype=np.int32))
    h = oracle.setup(p.rowptr, p.col, p.val, p.n, p.D1, p.agg, n_coarse=1, L_max=2)
    L = h.levels[0]
    r = np.random.default_rng(1).standard_normal(p.n)
    x = additive_schwarz(L, r)
    ref = np.linalg.solve(L.A.toarray(), r)
    assert np.abs(x - ref).max() <= 1e-12 * np.abs(ref).max()


def test_additive_schwarz_equals_sum_of_local_inverses():
    p, h = _two_level()
    L = h.levels[0]
    A = L.A.toarray()
    ref = np.zeros((p.n, p.n))
    for Om in L.Omega:
        ref[np.ix_(Om, Om)] += np.linalg.inv(A[np.ix_(Om, Om)])
    M1 = _dense(lambda v: additive_schwarz(L, v), p.n)
    assert np.abs(M1 - ref).max() <= 1e-11 * np.abs(ref).max()
    assert np.abs(M1 - M1.T).max() <= 1e-12 * np.abs(M1).max()


@pytest.mark.parametrize("tau", [2.0, 4.0, 8.0])
def test_spectral_bound_of_the_additive_two_level_method(tau):
    p, h = _two_level(tau=tau)
    L = h.levels[0]
    n = p.n
    M2 = _dense(lambda v: two_level_additive(h, v), n)
    assert np.abs(M2 - M2.T).max() <= 1e-11 * np.abs(M2).max()
    A = L.A.toarray()
    # eigenvalues of M_2^{-1} A = those of the symmetric pencil (A, M_2)
    lam = np.sort(sla.eigh(A, np.linalg.inv(0.5 * (M2 + M2.T)), eigvals_only=True))
    kc = _colours(L)
    lo, hi = 1.0 / (2.0 + (2 * kc + 1) * tau), kc + 1.0
    assert lam[0] >= lo * (1 - 1e-10), (lam[0], lo, kc)
    assert lam[-1] <= hi * (1 + 1e-10), (lam[-1], hi, kc)
    # the coarse space is a proper subspace here (a meaningful bound)
    assert L.P.shape[1] < n


def test_full_coarse_space_makes_the_coarse_part_exact():
    p, h = _two_level(tau=0.5)
    L = h.levels[0]
    assert L.P.shape[1] == p.n  # lambda >= 1 > tau: every local eigenvector is kept
    M2 = _dense(lambda v: two_level_additive(h, v), p.n)
    A = L.A.toarray()
    lam = np.sort(sla.eigh(A, np.linalg.inv(0.5 * (M2 + M2.T)), eigvals_only=True))
    assert lam[0] >= 1.0 - 1e-10  # M_2^{-1} = A^{-1} + M_1^{-1} with M_1^{-1} SPD


def test_pcg_with_the_additive_two_level_method():
    p, h = _two_level(N=16, bs=4, tau=4.0)
    b = seeded_rhs(p.n, 1, 3)[:, 0]
    x, info = oracle.pcg(h, b, tol=1e-10, precond=two_level_additive)
    assert info["status"] == 0 and info["relres_true"] <= 1e-9
    A = h.levels[0].A.toarray()
    ref = sla.cho_solve(sla.cho_factor(A), b)
    assert np.abs(x - ref).max() <= 1e-8 * np.abs(ref).max() * np.linalg.cond(A) ** 0.5
