"""Solve phase of the oracle (test infrastructure).

* RAS, Eq. ras:    x = sum_i R_i^T D_i A_i^{-1} R_i r
  (every node of omega_i takes the omega part of the local solve; Gamma
  entries of the local solution are discarded by the Boolean PoU D_i);
* RAS-T, Eq. ras-t: x = sum_i R_i^T A_i^{-1} D_i R_i r
  (the local right-hand side keeps only its omega entries; the whole local
  solution is added back on Omega_i, so overlapping contributions sum);
* V-cycle (Section 2.1 coarse-grid correction; Section 3.1: one RAS pre-,
  one RAS-T post-smoothing, recursion to an exact coarsest solve), started
  from x = 0 so that it applies a fixed linear preconditioner B;
* the additive two-level method M_2^{-1} = P (P^T A P)^{-1} P^T + M_1^{-1}
  with additive Schwarz M_1^{-1} = sum_i R_i^T A_i^{-1} R_i (Section 3.1,
  after Eq. cgc), on two-level hierarchies;
* preconditioned CG (Hestenes-Stiefel, x_0 = 0), stopped when the
  recursively updated residual satisfies ||r_k|| <= tol ||b||, plus the
  flexible variant beta = r_{k+1}^T (z_{k+1} - z_k) / (r_k^T z_k);
* metrics of Section 4: average convergence factor rho = (||r_k||/||r_0||)^{1/k},
  iterations per 10x reduction ln(0.1)/ln(rho), operator complexity.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla


def apply_A(level, x):
    return level.A @ x


def _local_solve(L, v):
    return sla.cho_solve((L, True), v)


def ras(level, r):
    """x = M_RAS^{-1} r (Eq. ras) applied to x = 0."""
    x = np.zeros(level.n)
    for i in range(level.nagg):
        Om = level.Omega[i]
        no = level.omega[i].shape[0]
        y = _local_solve(level.chol[i], r[Om])
        x[Om[:no]] = y[:no]
    return x


def rast(level, s):
    """x = M_RAS-T^{-1} s (Eq. ras-t)."""
    x = np.zeros(level.n)
    for i in range(level.nagg):
        Om = level.Omega[i]
        no = level.omega[i].shape[0]
        v = s[Om].copy()
        v[no:] = 0.0
        y = _local_solve(level.chol[i], v)
        x[Om] += y
    return x


def vcycle(h, r, lvl=0):
    """z = B_l r: RAS pre-smoothing, coarse-grid correction, RAS-T post."""
    levels = h.levels
    if lvl == len(levels) - 1:
        return sla.cho_solve((h.coarse_chol, True), r)
    L = levels[lvl]
    x = ras(L, r)
    s = r - apply_A(L, x)
    rc = L.P.T @ s
    xc = vcycle(h, rc, lvl + 1)
    x = x + L.P @ xc
    s = r - apply_A(L, x)
    x = x + rast(L, s)
    return x


def additive_schwarz(level, r):
    """x = M_1^{-1} r = sum_i R_i^T A_i^{-1} R_i r: the Schwarz smoother of
    Eq. ras without the partition of unity (additive Schwarz); every local
    solution is added back on all of Omega_i."""
    x = np.zeros(level.n)
    for i in range(level.nagg):
        Om = level.Omega[i]
        x[Om] += _local_solve(level.chol[i], r[Om])
    return x


def two_level_additive(h, r):
    """z = M_2^{-1} r = P (P^T A P)^{-1} P^T r + M_1^{-1} r, the additive
    two-level method the paper sets beside the multiplicative cycle (Section
    3.1), with M_1 additive Schwarz and an exact solve of the level-1
    operator P^T A P.  Defined on two-level hierarchies."""
    if len(h.levels) != 2:
        raise ValueError("the additive two-level method needs a two-level hierarchy")
    L = h.levels[0]
    xc = sla.cho_solve((h.coarse_chol, True), L.P.T @ r)
    return additive_schwarz(L, r) + L.P @ xc


def pcg(h, b, tol=1e-8, maxit=1000, flexible=False, precond=None):
    """Preconditioned CG with the V-cycle (or `precond(h, r)`, e.g. the
    additive two-level method); one right-hand side.

    Returns (x, info) with info = dict(iters, relres (recursive), relres_true,
    history (recursive relative residuals), status) where status is 0 on
    convergence, 1 when maxit was reached, 2 on breakdown (p^T A p <= 0).
    """
    A0 = h.levels[0]
    b = np.asarray(b, dtype=np.float64)
    bn = float(np.linalg.norm(b))
    x = np.zeros_like(b)
    if bn == 0.0:
        return x, dict(iters=0, relres=0.0, relres_true=0.0, history=[0.0], status=0)
    apply_B = vcycle if precond is None else precond
    r = b.copy()
    z = apply_B(h, r)
    p = z.copy()
    rz = float(r @ z)
    hist = [1.0]
    status = 1
    it = 0
    for it in range(1, maxit + 1):
        q = apply_A(A0, p)
        pq = float(p @ q)
        if not pq > 0.0:
            status = 2
            it -= 1
            break
        alpha = rz / pq
        x += alpha * p
        r -= alpha * q
        rel = float(np.linalg.norm(r)) / bn
        hist.append(rel)
        if rel <= tol:
            status = 0
            break
        zn = apply_B(h, r)
        if flexible:
            rzn = float(r @ zn)
            beta = float(r @ (zn - z)) / rz
        else:
            rzn = float(r @ zn)
            beta = rzn / rz
        p = zn + beta * p
        z = zn
        rz = rzn
    true = float(np.linalg.norm(b - apply_A(A0, x))) / bn
    return x, dict(iters=it, relres=hist[-1], relres_true=true, history=hist, status=status)


def metrics(h, info=None):
    """Level sizes, operator and grid complexity, convergence factor."""
    nnz = [int(L.A.nnz) for L in h.levels]
    ns = [int(L.n) for L in h.levels]
    out = dict(levels=len(h.levels), n=ns, nnz=nnz, op_complexity=sum(nnz) / nnz[0],
               grid_complexity=sum(ns) / ns[0])
    if info is not None and info["iters"] > 0 and info["relres"] > 0:
        rho = info["relres"] ** (1.0 / info["iters"])
        out["rho"] = rho
        out["iters_per_digit"] = math.log(0.1) / math.log(rho) if rho < 1 else float("inf")
    return out
