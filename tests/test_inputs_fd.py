"""Pins of the finite-difference least-squares factor G = B^T grad^+ (Section 4.1).

* theta = 0, eps = 1: G^T G is the 5-point Laplacian (4 / h^2 on the diagonal, -1 / h^2 to the four
  neighbours, Dirichlet boundary), as the paper states;
* G^T G equals -div^-(K grad^+) assembled another way: the difference matrices D_x^+, D_y^+ built as sparse
  matrices and combined as grad^T (K kron I) grad, with no per-row loop;
* sizes: 2 ((N+1)^2 - 1) rows of at most three entries.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from inputs import fd_2d, fd_block_aggregates
from inputs.q1 import config_problem


def _dplus(N, h):
    """Forward differences on the (N+1) x (N+1) points -1..N-1 of each axis, unknowns 0..N-1."""
    P = (N + 1) ** 2
    Dx = sp.lil_matrix((P, N * N))
    Dy = sp.lil_matrix((P, N * N))
    for j in range(-1, N):
        for i in range(-1, N):
            r = (j + 1) * (N + 1) + (i + 1)
            for (a, b, M, cf) in ((i, j, Dx, -1.0), (i + 1, j, Dx, 1.0), (i, j, Dy, -1.0), (i, j + 1, Dy, 1.0)):
                if 0 <= a < N and 0 <= b < N:
                    M[r, b * N + a] += cf / h
    return Dx.tocsr(), Dy.tocsr()


def test_five_point_laplacian_at_theta_0_eps_1():
    N = 7
    h = 1.0 / (N + 1)
    p = fd_2d(N, 0.0, 1.0)
    A = (p.G_scipy().T @ p.G_scipy()).toarray() * h * h
    for j in range(N):
        for i in range(N):
            r = j * N + i
            assert abs(A[r, r] - 4.0) <= 1e-12
            for (a, b) in ((i + 1, j), (i - 1, j), (i, j + 1), (i, j - 1)):
                if 0 <= a < N and 0 <= b < N:
                    assert abs(A[r, b * N + a] + 1.0) <= 1e-12
            assert abs(np.abs(A[r]).sum() - 4.0 - sum(
                1 for (a, b) in ((i + 1, j), (i - 1, j), (i, j + 1), (i, j - 1)) if 0 <= a < N and 0 <= b < N)) <= 1e-12


@pytest.mark.parametrize("theta,eps", [(math.pi / 6, 1e-3), (0.4, 0.2), (math.pi / 4, 1e-6)])
def test_gtg_is_minus_div_k_grad(theta, eps):
    N = 6
    h = 1.0 / (N + 1)
    p = fd_2d(N, theta, eps)
    c, s = math.cos(theta), math.sin(theta)
    Q = np.array([[c, -s], [s, c]])
    K = Q @ np.diag([eps, 1.0]) @ Q.T
    Dx, Dy = _dplus(N, h)
    ref = (K[0, 0] * Dx.T @ Dx + K[0, 1] * Dx.T @ Dy + K[1, 0] * Dy.T @ Dx + K[1, 1] * Dy.T @ Dy).toarray()
    A = (p.G_scipy().T @ p.G_scipy()).toarray()
    assert np.abs(A - ref).max() <= 1e-12 * np.abs(ref).max()


def test_sizes_and_pattern():
    N = 9
    p = fd_2d(N, 0.3, 1e-2)
    assert p.n == N * N and p.m == 2 * ((N + 1) ** 2 - 1)
    lens = np.diff(p.rowptr)
    assert lens.min() >= 1 and lens.max() <= 3
    for r in range(p.m):
        cols = p.col[p.rowptr[r]:p.rowptr[r + 1]]
        assert np.all(np.diff(cols) > 0)
    agg = fd_block_aggregates(N, 4)
    assert agg.max() + 1 == 9 and np.bincount(agg).min() == 1  # 3 x 3 blocks, the corner one 1 x 1


def test_fd_workload_config():
    p, cfg = config_problem("fd_64_rot")
    assert p.n == 64 * 64 and cfg["kappa"] == 50.0 and p.agg.max() + 1 == 16 * 16
