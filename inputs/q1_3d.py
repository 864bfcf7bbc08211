"""Trilinear (Q1) least-squares factor G of anisotropic diffusion on the unit
cube, and greedy strength-graph aggregates for it.

    row (c, q, d)[a] = sqrt(w_q) * (K(x_q)^{1/2} grad phi_a(x_q))_d

for every interior corner node a of hexahedral cell c, Gauss point q of the
2x2x2 rule (w_q = h^3 / 8) and direction d, so that G^T G is the Q1
stiffness matrix of -div(K grad u) with homogeneous Dirichlet data.  The
coefficient is K = eps I + (1 - eps) b b^T with b(x) a smooth unit vector
field: the normalised sum of four seeded random Fourier modes.

Layout (fixed, relied on by the tests):
  * nodes (i, j, k), 1 <= i, j, k <= N-1, are numbered
    (k-1)(N-1)^2 + (j-1)(N-1) + (i-1);
  * cells (ci, cj, ck) are numbered ci + N*cj + N^2*ck;
  * rows are cell-major, then Gauss point q = qx + 2*qy + 4*qz, then d;
  * within a row, columns ascend; every interior corner is a structural
    entry.

The level-0 aggregates of this workload are irregular: standard greedy
aggregation (root passes, then attachment, then leftovers) on the strength
graph |a_ij| >= theta sqrt(a_ii a_jj) of A = G^T G.  On trilinear stencils
every off-diagonal is at most 1/16 of the diagonal when K = I, so the
customary theta = 0.25 leaves singletons; the workload takes theta = 0.03,
which gives aggregates of about 5-40 nodes and one-hop subdomains of about
30-200.  The aggregates are an input of the method, built here and passed to
setup like the 2D block aggregates.
"""
from __future__ import annotations

import math

import numpy as np

from .q1 import Q1Problem

_G0 = 0.5 - 0.5 / math.sqrt(3.0)
_G1 = 0.5 + 0.5 / math.sqrt(3.0)
_QX = np.array([_G0, _G1, _G0, _G1, _G0, _G1, _G0, _G1])
_QY = np.array([_G0, _G0, _G1, _G1, _G0, _G0, _G1, _G1])
_QZ = np.array([_G0, _G0, _G0, _G0, _G1, _G1, _G1, _G1])
# corner offsets in ascending global-index order (x fastest)
_DX = np.array([0, 1, 0, 1, 0, 1, 0, 1])
_DY = np.array([0, 0, 1, 1, 0, 0, 1, 1])
_DZ = np.array([0, 0, 0, 0, 1, 1, 1, 1])


def fourier_direction(seed: int, modes: int = 4):
    """b(x) = v(x) / |v(x)|, v = sum_j a_j cos(2 pi k_j . x + phi_j) with
    a_j ~ N(0, I_3), k_j uniform in {-2..2}^3 minus 0, phi_j ~ U[0, 2 pi)
    (e_x where |v| < 1e-12)."""
    rng = np.random.default_rng(seed)
    amp = rng.standard_normal((modes, 3))
    ks = []
    while len(ks) < modes:
        k = rng.integers(-2, 3, size=3)
        if np.any(k != 0):
            ks.append(k)
    ks = np.array(ks, dtype=np.float64)
    ph = rng.uniform(0.0, 2.0 * math.pi, size=modes)

    def b(x, y, z):
        v = np.zeros(np.shape(x) + (3,))
        for j in range(modes):
            arg = 2.0 * math.pi * (ks[j, 0] * x + ks[j, 1] * y + ks[j, 2] * z) + ph[j]
            v += np.cos(arg)[..., None] * amp[j]
        nv = np.linalg.norm(v, axis=-1, keepdims=True)
        ex = np.zeros_like(v)
        ex[..., 0] = 1.0
        return np.where(nv < 1e-12, ex, v / np.maximum(nv, 1e-300))

    return b


def field_sqrtK(eps: float, seed: int):
    """K^{1/2} = sqrt(eps) I + (1 - sqrt(eps)) b b^T for K = eps I + (1 - eps) b b^T."""
    b = fourier_direction(seed)
    se = math.sqrt(eps)

    def f(x, y, z):
        bb = b(x, y, z)
        out = (1.0 - se) * bb[..., :, None] * bb[..., None, :]
        out[..., 0, 0] += se
        out[..., 1, 1] += se
        out[..., 2, 2] += se
        return out

    return f


def q1_3d(N: int, sqrtK, D1: np.ndarray | None = None, agg: np.ndarray | None = None,
          desc: dict | None = None) -> Q1Problem:
    """Assemble G (24 rows per cell) for an N x N x N cell grid on [0,1]^3."""
    if N < 3:
        raise ValueError("need at least 3 cells per axis")
    h = 1.0 / N
    nint = N - 1
    C = N ** 3
    cells = np.arange(C)
    ck, rem = np.divmod(cells, N * N)
    cj, ci = np.divmod(rem, N)
    ni = ci[:, None] + _DX[None, :]
    nj = cj[:, None] + _DY[None, :]
    nk = ck[:, None] + _DZ[None, :]
    interior = (ni >= 1) & (ni <= nint) & (nj >= 1) & (nj <= nint) & (nk >= 1) & (nk <= nint)
    node = (nk - 1) * nint * nint + (nj - 1) * nint + (ni - 1)
    # gradients of the eight trilinear shape functions at the eight points
    fx = np.where(_DX[None, :] == 1, _QX[:, None], 1 - _QX[:, None])
    fy = np.where(_DY[None, :] == 1, _QY[:, None], 1 - _QY[:, None])
    fz = np.where(_DZ[None, :] == 1, _QZ[:, None], 1 - _QZ[:, None])
    sx = (2 * _DX[None, :] - 1).astype(np.float64)
    sy = (2 * _DY[None, :] - 1).astype(np.float64)
    sz = (2 * _DZ[None, :] - 1).astype(np.float64)
    grad = np.stack([sx * fy * fz, fx * sy * fz, fx * fy * sz], axis=-1) / h  # (q, a, 3)
    xq = (ci[:, None] + _QX[None, :]) * h
    yq = (cj[:, None] + _QY[None, :]) * h
    zq = (ck[:, None] + _QZ[None, :]) * h
    S = sqrtK(xq, yq, zq)  # (C, 8, 3, 3)
    sw = math.sqrt(h ** 3 / 8.0)
    vals = sw * np.einsum("cqde,qae->cqda", S, grad)  # (C, 8, 3, 8)
    mask = np.broadcast_to(interior[:, None, None, :], vals.shape)
    col = np.broadcast_to(node[:, None, None, :], vals.shape)[mask].astype(np.int32)
    val = np.ascontiguousarray(vals[mask], dtype=np.float64)
    cnt = np.repeat(interior.sum(axis=1), 24)
    rowptr = np.zeros(24 * C + 1, dtype=np.int64)
    np.cumsum(cnt, out=rowptr[1:])
    n = nint ** 3
    if agg is None:
        agg = np.zeros(n, dtype=np.int32)
    return Q1Problem(N=N, n=n, m=24 * C, rowptr=rowptr, col=col, val=val,
                     D1=None if D1 is None else np.ascontiguousarray(D1, dtype=np.float64),
                     agg=np.ascontiguousarray(agg, dtype=np.int32), desc=dict(desc or {}))


def strength_graph(prob: Q1Problem, theta: float = 0.25):
    """CSR (indptr, indices) of |a_ij| >= theta sqrt(|a_ii a_jj|), i != j, for A = G^T G."""
    G = prob.G_scipy()
    A = (G.T @ G).tocsr()
    d = np.abs(A.diagonal())
    A = A.tocoo()
    keep = (A.row != A.col) & (np.abs(A.data) >= theta * np.sqrt(d[A.row] * d[A.col]))
    import scipy.sparse as sp

    S = sp.csr_matrix((np.ones(int(keep.sum())), (A.row[keep], A.col[keep])), shape=(prob.n, prob.n))
    S.sort_indices()
    return S.indptr, S.indices


def greedy_aggregates(indptr: np.ndarray, indices: np.ndarray, n: int) -> np.ndarray:
    """Standard greedy aggregation on a symmetric strength graph.

    Pass 1 (ascending nodes): a node whose strong neighbours are all free
    becomes a root and takes them.  Pass 2: each free node joins the
    aggregate of its lowest-numbered strong neighbour aggregated in pass 1.
    Pass 3 (ascending): a node still free starts an aggregate with its free
    strong neighbours."""
    agg = np.full(n, -1, dtype=np.int64)
    nagg = 0
    for i in range(n):
        if agg[i] >= 0:
            continue
        nb = indices[indptr[i]:indptr[i + 1]]
        if np.all(agg[nb] < 0):
            agg[i] = nagg
            agg[nb] = nagg
            nagg += 1
    snap = agg.copy()
    for i in np.nonzero(snap < 0)[0]:
        nb = indices[indptr[i]:indptr[i + 1]]
        hit = nb[snap[nb] >= 0]
        if hit.size:
            agg[i] = snap[hit.min()]
    for i in range(n):
        if agg[i] >= 0:
            continue
        nb = indices[indptr[i]:indptr[i + 1]]
        free = nb[agg[nb] < 0]
        agg[i] = nagg
        agg[free] = nagg
        nagg += 1
    return agg.astype(np.int32)
