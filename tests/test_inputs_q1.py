"""Pins of the Q1 least-squares factor G (the problem of Eq. 1, A = G^T G).

G is checked against an independently integrated Q1 stiffness matrix (exact
1D integrals combined by tensor products, no quadrature and no K^{1/2}),
against the textbook 9-point Laplace stencil stored in tests/golden, and
against closed-form sizes.
"""
import math

import numpy as np
import pytest

from inputs import block_aggregates_2d, circular_sqrtK, q1_2d, rotated_sqrtK, seeded_rhs
from inputs.q1 import config_problem


def _exact_q1_stiffness(N, K):
    """Q1 stiffness of -div(K grad u), constant K, from exact 1D integrals."""
    h = 1.0 / N
    K1 = np.array([[1.0, -1.0], [-1.0, 1.0]]) / h  # int l_a' l_c'
    M1 = np.array([[2.0, 1.0], [1.0, 2.0]]) * h / 6  # int l_a l_c
    C1 = np.array([[-0.5, -0.5], [0.5, 0.5]])  # C1[a, c] = int l_a' l_c
    E = np.zeros((2, 2, 2, 2))  # E[a, b, c, d] for corners (a,b), (c,d)
    for a in range(2):
        for b in range(2):
            for c in range(2):
                for d in range(2):
                    E[a, b, c, d] = (K[0, 0] * K1[a, c] * M1[b, d] + K[0, 1] * C1[a, c] * C1[d, b]
                                     + K[1, 0] * C1[c, a] * C1[b, d] + K[1, 1] * M1[a, c] * K1[b, d])
    n = (N - 1) ** 2
    A = np.zeros((n, n))
    for cj in range(N):
        for ci in range(N):
            for a in range(2):
                for b in range(2):
                    i1, j1 = ci + a, cj + b
                    if not (1 <= i1 <= N - 1 and 1 <= j1 <= N - 1):
                        continue
                    r = (j1 - 1) * (N - 1) + (i1 - 1)
                    for c in range(2):
                        for d in range(2):
                            i2, j2 = ci + c, cj + d
                            if not (1 <= i2 <= N - 1 and 1 <= j2 <= N - 1):
                                continue
                            s = (j2 - 1) * (N - 1) + (i2 - 1)
                            A[r, s] += E[a, b, c, d]
    return A


@pytest.mark.parametrize("theta,eps", [(0.0, 1.0), (math.pi / 6, 1e-3), (math.pi / 4, 1e-6), (1.0, 0.3)])
def test_GtG_equals_exact_stiffness(theta, eps):
    N = 7
    p = q1_2d(N, rotated_sqrtK(theta, eps))
    G = p.G_scipy().toarray()
    c, s = math.cos(theta), math.sin(theta)
    R = np.array([[c, -s], [s, c]])
    K = R @ np.diag([1.0, eps]) @ R.T
    Aref = _exact_q1_stiffness(N, K)
    assert np.abs(G.T @ G - Aref).max() <= 1e-14 * np.abs(Aref).max()


def test_laplace_stencil_golden():
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", "q1_laplace_stencil.txt")
    st = np.loadtxt(path)
    N = 9
    p = q1_2d(N, rotated_sqrtK(0.0, 1.0))
    A = (p.G_scipy().T @ p.G_scipy()).toarray()
    nint = N - 1
    for (i, j) in [(4, 4), (2, 5), (6, 3)]:
        r = (j - 1) * nint + (i - 1)
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                s = (j + dy - 1) * nint + (i + dx - 1)
                assert abs(A[r, s] - st[dy + 1, dx + 1]) <= 1e-14
        assert abs(A[r].sum()) <= 1e-13  # interior rows of a pure-Neumann-free stencil sum to 0


def test_sizes_and_layout():
    for N in (4, 9, 64):
        p = q1_2d(N, rotated_sqrtK(0.3, 0.1))
        assert p.n == (N - 1) ** 2
        assert p.m == 8 * N * N
        assert p.nnz == 32 * (N - 1) ** 2  # each interior node is a corner of 4 cells x 8 rows
        # columns ascend within each row
        for r in range(0, p.m, 37):
            c = p.col[p.rowptr[r]:p.rowptr[r + 1]]
            assert np.all(np.diff(c) > 0)
    p = q1_2d(64, rotated_sqrtK(0.0, 1.0))
    assert (p.n, p.m, p.nnz) == (3969, 32768, 127008)


def test_structural_entries_kept_when_zero():
    # theta = 0, eps = 1: no value cancels, but the pattern must not depend on values
    p0 = q1_2d(6, rotated_sqrtK(0.0, 1.0))
    p1 = q1_2d(6, rotated_sqrtK(0.7, 1e-8))
    assert np.array_equal(p0.rowptr, p1.rowptr) and np.array_equal(p0.col, p1.col)


def test_circular_field_sqrtK():
    f = circular_sqrtK(1e-4)
    x = np.array([0.1, 0.9, 0.3, 0.72])
    y = np.array([0.2, 0.4, 0.85, 0.6])
    S = f(x, y)
    for t in range(4):
        K = S[t] @ S[t]
        rad = np.array([x[t] - 0.5, y[t] - 0.5])
        rad /= np.linalg.norm(rad)
        tan = np.array([-rad[1], rad[0]])
        assert np.allclose(K @ tan, tan, atol=1e-14)  # strong direction: along circles
        assert np.allclose(K @ rad, 1e-4 * rad, atol=1e-14)
        assert np.allclose(S[t], S[t].T)


def test_block_aggregates():
    agg = block_aggregates_2d(64, 4)
    assert agg.max() + 1 == 256
    counts = np.bincount(agg)
    assert counts.max() == 16 and counts.min() == 9  # last block per axis is 3 wide
    agg8 = block_aggregates_2d(2048, 8)
    assert agg8.max() + 1 == 65536


def test_seeded_rhs_reproducible():
    b1 = seeded_rhs(100, 3, 7)
    b2 = seeded_rhs(100, 3, 7)
    assert np.array_equal(b1, b2) and b1.flags.f_contiguous
    assert np.array_equal(seeded_rhs(100, 1, 7)[:, 0], np.random.default_rng(7).standard_normal(100))


def test_config_d1():
    p, cfg = config_problem("q1_64_rot", d1=1e-8)
    assert p.D1 is not None and np.allclose(p.D1, 1e-8 / 64 ** 2)
