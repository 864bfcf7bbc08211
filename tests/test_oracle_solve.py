"""Pins of the oracle's solve phase on tiny grids (dense checks).

* Eq. ras-t: M_RAS-T^{-1} = M_RAS^{-T} (adjointness on random vectors);
* one aggregate covering every node: RAS is the exact solve A^{-1};
* the V-cycle preconditioner B (applied from x = 0) is symmetric and its
  error propagator E = I - BA has spectrum in [0, 1) (E is A-self-adjoint
  and A-PSD for a symmetric V-cycle with an exact coarsest solve; Section 3.1
  states the cycle is SPD);
* the stationary iteration x <- x + B(b - Ax) contracts at the rate rho(E)
  from a dense eigensolve;
* c_min = 1 on a two-level hierarchy makes P square and invertible, so the
  cycle is an exact solve and PCG stops after one iteration;
* PCG reaches the Cholesky solution (scipy.linalg.cho_solve) within the
  bound tol * cond(A).
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from inputs import block_aggregates_2d, q1_2d, rotated_sqrtK, seeded_rhs
from oracle.cycle import ras, rast, vcycle


def _prob(N=12, bs=2, d1=None, theta=math.pi / 6, eps=1e-2):
    D1 = None if d1 is None else np.full((N - 1) ** 2, d1)
    return q1_2d(N, rotated_sqrtK(theta, eps), D1=D1, agg=block_aggregates_2d(N, bs))


def _h(p, **kw):
    kw.setdefault("overlap", 1)
    kw.setdefault("c_min", (2,))
    kw.setdefault("n_coarse", 12)
    kw.setdefault("L_max", 6)
    return oracle.setup(p.rowptr, p.col, p.val, p.n, p.D1, p.agg, **kw)


def _dense_B(h):
    n = h.levels[0].n
    return np.column_stack([vcycle(h, e) for e in np.eye(n)])


@pytest.mark.parametrize("overlap", [1, 2])
def test_ras_rast_adjoint(overlap):
    p = _prob()
    h = _h(p, overlap=overlap)
    L = h.levels[0]
    rng = np.random.default_rng(0)
    for _ in range(3):
        x, y = rng.standard_normal(p.n), rng.standard_normal(p.n)
        assert abs(ras(L, x) @ y - x @ rast(L, y)) <= 1e-12 * np.linalg.norm(x) * np.linalg.norm(y) * 10


def test_single_aggregate_ras_is_exact():
    p = q1_2d(7, rotated_sqrtK(0.3, 0.1), agg=np.zeros(36, dtype=np.int32))
    h = oracle.setup(p.rowptr, p.col, p.val, p.n, p.D1, p.agg, n_coarse=1, L_max=2)
    L = h.levels[0]
    r = np.random.default_rng(1).standard_normal(p.n)
    x = ras(L, r)
    ref = np.linalg.solve(L.A.toarray(), r)
    assert np.abs(x - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("case", [dict(), dict(d1=0.3), dict(theta=0.0, eps=1.0), dict(theta=1.1, eps=1e-5)])
def test_vcycle_symmetric_and_contracting(case):
    p = _prob(**case)
    h = _h(p)
    assert len(h.levels) >= 3  # recursion is exercised
    A = h.levels[0].A.toarray()
    B = _dense_B(h)
    assert np.abs(B - B.T).max() <= 1e-13 * np.abs(B).max()
    ev = np.linalg.eigvals(B @ A).real
    assert ev.max() <= 1 + 1e-12
    assert ev.min() > 0  # SPD preconditioner (Section 3.1)


def test_stationary_rate_matches_spectral_radius():
    p = _prob(theta=0.5, eps=1e-3)
    h = _h(p, c_min=(4,))
    A = h.levels[0].A.toarray()
    B = _dense_B(h)
    E = np.eye(p.n) - B @ A
    rho = max(abs(np.linalg.eigvals(E)))
    assert 0.05 < rho < 1
    e = np.random.default_rng(3).standard_normal(p.n)
    norms = []
    for _ in range(60):
        e = E @ e
        norms.append(np.linalg.norm(e))
    obs = (norms[-1] / norms[-11]) ** 0.1
    assert abs(obs - rho) <= 0.02 * rho


def test_cmin_one_is_exact_two_level():
    p = _prob(N=10, bs=3)
    h = oracle.setup(p.rowptr, p.col, p.val, p.n, p.D1, p.agg, overlap=1, c_min=(1,), thresh=0.0,
                     n_coarse=1, L_max=2)
    assert h.levels[1].n == p.n
    b = seeded_rhs(p.n, 1, 5)[:, 0]
    x, info = oracle.pcg(h, b, tol=1e-8)
    assert info["iters"] == 1 and info["relres_true"] <= 1e-12


@pytest.mark.parametrize("flexible", [False, True])
def test_pcg_matches_cholesky(flexible):
    p = _prob(N=16, bs=4, theta=math.pi / 6, eps=1e-3)
    h = _h(p, c_min=(2, 3), n_coarse=30)
    A = h.levels[0].A.toarray()
    b = seeded_rhs(p.n, 1, 1)[:, 0]
    x, info = oracle.pcg(h, b, tol=1e-10, flexible=flexible)
    ref = sla.cho_solve(sla.cho_factor(A), b)
    kappa = np.linalg.cond(A)
    assert info["status"] == 0 and info["relres_true"] <= 1e-9
    assert np.linalg.norm(x - ref) <= 1e-10 * kappa * np.linalg.norm(ref)


def test_metrics():
    p = _prob()
    h = _h(p)
    b = seeded_rhs(p.n, 1, 1)[:, 0]
    x, info = oracle.pcg(h, b)
    m = oracle.metrics(h, info)
    assert m["op_complexity"] >= 1 and 0 < m["rho"] < 1
    assert m["n"][0] == p.n and m["levels"] == len(h.levels)
