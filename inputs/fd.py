"""Finite-difference least-squares factor G of rotated anisotropic diffusion.

This is the discretization the paper uses for its own rotated-anisotropy study (Section 4.1). On a uniform
grid with spacing h:

    (D_x^+ u)_{i,j} = (u_{i+1,j} - u_{i,j}) / h,   (D_y^+ u)_{i,j} = (u_{i,j+1} - u_{i,j}) / h,
    grad^+ u = (D_x^+ u ; D_y^+ u),   K = Q D Q^T = B B^T,   B = Q sqrt(D),   D = diag(eps, 1),
    G = B^T grad^+,   so that   G^T G u = -div^-(K grad^+ u)

with Q(theta) the rotation by theta.  At theta = 0 and eps = 1, G^T G is the 5-point Laplacian.

Reading of the boundary (the paper does not state one): homogeneous Dirichlet.  The N x N interior nodes
(i, j), 0 <= i, j < N, are the unknowns, h = 1 / (N + 1), and u = 0 outside.  The differences are taken at
the (N + 1) x (N + 1) points (i, j), -1 <= i, j < N, which gives every interior node its four neighbour
differences.  Each point contributes two rows, (B^T grad^+ u)_d for d = 0, 1; rows whose support holds no
unknown are dropped.

Layout (fixed, relied on by the tests):
  * node (i, j) is unknown j N + i (x fastest);
  * rows follow the points (i, j) with j outer and i inner, then d;
  * within a row, columns ascend; all three stencil nodes that are unknowns are structural entries (a
    coefficient that happens to be 0, e.g. at theta = 0, stays in the pattern).
"""
from __future__ import annotations

import math

import numpy as np

from .q1 import Q1Problem


def fd_2d(N: int, theta: float, eps: float, D1: np.ndarray | None = None, agg: np.ndarray | None = None,
          desc: dict | None = None) -> Q1Problem:
    """G = B^T grad^+ for an N x N grid of unknowns (2 rows per difference point).  With agg = None the
    problem carries no level-0 aggregates: the solver chooses them."""
    if N < 2:
        raise ValueError("need at least 2 unknowns per axis")
    h = 1.0 / (N + 1)
    c, s = math.cos(theta), math.sin(theta)
    Q = np.array([[c, -s], [s, c]])
    B = Q @ np.diag([math.sqrt(eps), 1.0])
    Bt = B.T  # row d of B^T weighs (D_x^+, D_y^+)
    rows_ptr = [0]
    cols, vals = [], []
    n = N * N
    for j in range(-1, N):
        for i in range(-1, N):
            # (node, dx coefficient, dy coefficient) of the three stencil nodes
            terms = {}
            for (a, b, cx, cy) in ((i, j, -1.0, -1.0), (i + 1, j, 1.0, 0.0), (i, j + 1, 0.0, 1.0)):
                if 0 <= a < N and 0 <= b < N:
                    terms[b * N + a] = (cx / h, cy / h)
            if not terms:
                continue
            keys = sorted(terms)
            for d in range(2):
                for k in keys:
                    gx, gy = terms[k]
                    cols.append(k)
                    vals.append(Bt[d, 0] * gx + Bt[d, 1] * gy)
                rows_ptr.append(len(cols))
    rowptr = np.asarray(rows_ptr, dtype=np.int64)
    return Q1Problem(N=N, n=n, m=len(rowptr) - 1, rowptr=rowptr, col=np.asarray(cols, dtype=np.int32),
                     val=np.asarray(vals, dtype=np.float64),
                     D1=None if D1 is None else np.ascontiguousarray(D1, dtype=np.float64),
                     agg=None if agg is None else np.ascontiguousarray(agg, dtype=np.int32),
                     desc=dict(desc or {}))


def fd_block_aggregates(N: int, bs: int) -> np.ndarray:
    """Level-0 aggregates: bs x bs blocks of the N x N unknowns (the last block per axis narrower)."""
    k = np.arange(N * N)
    j, i = np.divmod(k, N)
    nb = -(-N // bs)
    return (i // bs + nb * (j // bs)).astype(np.int32)
