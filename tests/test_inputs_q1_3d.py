"""Pins of the 3D Q1 generator and of the greedy strength-graph aggregation.

* At K = I, G^T G equals the trilinear Laplacian stencil in closed form:
  centre 8h/3, face neighbours 0, edge neighbours -h/6, corner neighbours
  -h/12, and rows of nodes away from the boundary sum to zero.
* The coefficient root squares to K = eps I + (1 - eps) b b^T with |b| = 1.
* Greedy aggregation on hand-worked graphs, and on the 3D workload every
  node belongs to one aggregate connected through strong edges.
"""
import numpy as np

from inputs.q1_3d import field_sqrtK, fourier_direction, greedy_aggregates, q1_3d, strength_graph


def _identity(x, y, z):
    out = np.zeros(np.shape(x) + (3, 3))
    out[..., 0, 0] = out[..., 1, 1] = out[..., 2, 2] = 1.0
    return out


def test_laplace_stencil_closed_form():
    N = 6
    h = 1.0 / N
    p = q1_3d(N, _identity)
    A = (p.G_scipy().T @ p.G_scipy()).toarray()
    ni = N - 1

    def idx(i, j, k):
        return (k - 1) * ni * ni + (j - 1) * ni + (i - 1)

    c = idx(3, 3, 3)
    assert np.isclose(A[c, c], 8 * h / 3, rtol=1e-13)
    for d in [(1, 0, 0), (0, 1, 0), (0, 0, 1)]:
        assert abs(A[c, idx(3 + d[0], 3 + d[1], 3 + d[2])]) < 1e-15
    assert np.isclose(A[c, idx(4, 4, 3)], -h / 6, rtol=1e-13)
    assert np.isclose(A[c, idx(4, 4, 4)], -h / 12, rtol=1e-13)
    assert abs(A[c].sum()) < 1e-14
    assert p.m == 24 * N ** 3 and p.n == ni ** 3


def test_coefficient_root_squares_to_K():
    eps = 1e-4
    f = field_sqrtK(eps, 7)
    b = fourier_direction(7)
    x = np.random.default_rng(0).random((50, 3))
    S = f(x[:, 0], x[:, 1], x[:, 2])
    bb = b(x[:, 0], x[:, 1], x[:, 2])
    assert np.allclose(np.linalg.norm(bb, axis=1), 1.0)
    K = eps * np.eye(3) + (1 - eps) * bb[:, :, None] * bb[:, None, :]
    assert np.allclose(S @ S, K, atol=1e-14)


def test_greedy_aggregation_hand_worked():
    # path 0-1-2-3-4-5-6: pass 1 roots 0 {0,1}, 3 {2,3,4}; 6 {5,6}
    edges = [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 6)]
    import scipy.sparse as sp

    n = 7
    r = [a for a, b in edges] + [b for a, b in edges]
    c = [b for a, b in edges] + [a for a, b in edges]
    S = sp.csr_matrix((np.ones(len(r)), (r, c)), shape=(n, n))
    S.sort_indices()
    agg = greedy_aggregates(S.indptr, S.indices, n)
    assert agg.tolist() == [0, 0, 1, 1, 1, 2, 2]
    # a star whose centre comes last: pass 1 takes leaf 0 with the centre,
    # pass 2 attaches the other leaves to it
    r = [0, 1, 2, 3, 4, 4, 4, 4]
    c = [4, 4, 4, 4, 0, 1, 2, 3]
    S = sp.csr_matrix((np.ones(8), (r, c)), shape=(5, 5))
    S.sort_indices()
    assert greedy_aggregates(S.indptr, S.indices, 5).tolist() == [0, 0, 0, 0, 0]
    # an isolated node becomes its own aggregate in pass 3
    S = sp.csr_matrix((3, 3))
    assert greedy_aggregates(S.indptr, S.indices, 3).tolist() == [0, 1, 2]


def test_workload_aggregates_cover_and_connect():
    p = q1_3d(8, field_sqrtK(1e-4, 44))
    ip, ix = strength_graph(p)
    agg = greedy_aggregates(ip, ix, p.n)
    assert agg.min() == 0 and np.all(agg >= 0)
    assert np.array_equal(np.unique(agg), np.arange(agg.max() + 1))
    for a in range(agg.max() + 1):
        nodes = np.nonzero(agg == a)[0]
        seen = {nodes[0]}
        stack = [nodes[0]]
        member = set(nodes.tolist())
        while stack:
            v = stack.pop()
            for w in ix[ip[v]:ip[v + 1]]:
                if w in member and w not in seen:
                    seen.add(w)
                    stack.append(w)
        assert len(seen) == len(nodes)
