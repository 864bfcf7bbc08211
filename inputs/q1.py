"""Q1 least-squares factor G of anisotropic diffusion on the unit square.

The operator is A = D1 + G^T G with G sparse (the least-squares form of the
paper's Eq. 1, Section 1).  Here G is the bilinear (Q1) finite-element
gradient sampled at the 2x2 Gauss points of every cell:

    row (c, q, d)[a] = sqrt(w_q) * (K(x_q)^{1/2} grad phi_a(x_q))_d

for every interior corner node a of cell c, Gauss point q and direction d,
so that G^T G is the Q1 stiffness matrix of -div(K grad u) with homogeneous
Dirichlet data (boundary nodes eliminated).  This is the synthetic stand-in
for the paper's rotated-anisotropy workload (Section 4.1), with K = R(theta)
diag(1, eps) R(theta)^T, and for its closed-field-line workload (Section 4.2),
with theta following circles about the centre of the square.

Layout (fixed, relied on by the tests):
  * nodes (i, j), 1 <= i, j <= N-1, are numbered (j-1)(N-1) + (i-1);
  * cells (ci, cj), 0 <= ci, cj < N, are numbered ci + N*cj;
  * rows are cell-major, then Gauss point q = qx + 2*qy, then direction d;
  * within a row, columns ascend; every interior corner is a structural
    entry, even when its value happens to be zero.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# 2-point Gauss-Legendre abscissae on [0, 1]; exact for the bilinear products
# that make up the Q1 stiffness matrix.
_G0 = 0.5 - 0.5 / math.sqrt(3.0)
_G1 = 0.5 + 0.5 / math.sqrt(3.0)
_XI = np.array([_G0, _G1, _G0, _G1])
_ETA = np.array([_G0, _G0, _G1, _G1])
# corner offsets in ascending global-index order
_DX = np.array([0, 1, 0, 1])
_DY = np.array([0, 0, 1, 1])


@dataclass
class Q1Problem:
    """One synthetic least-squares problem in CSR form (host arrays)."""

    N: int
    n: int
    m: int
    rowptr: np.ndarray  # int64, m+1
    col: np.ndarray  # int32, nnz
    val: np.ndarray  # float64, nnz
    D1: np.ndarray | None  # float64, n, or None for D1 = 0
    agg: np.ndarray | None  # int32, n, level-0 aggregate ids; None: the solver aggregates
    desc: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def G_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.m, self.n))


def rotated_sqrtK(theta: float, eps: float):
    """K^{1/2} = R diag(1, sqrt(eps)) R^T for a constant rotation angle."""
    c, s = math.cos(theta), math.sin(theta)
    R = np.array([[c, -s], [s, c]])
    S = R @ np.diag([1.0, math.sqrt(eps)]) @ R.T

    def f(x, y):
        out = np.empty(np.shape(x) + (2, 2))
        out[...] = S
        return out

    return f


def circular_sqrtK(eps: float):
    """K^{1/2} with the strong direction tangent to circles about (1/2, 1/2).

    theta(x, y) = atan2(y - 1/2, x - 1/2) + pi/2; at the centre itself the
    angle is undefined and theta = 0 is used (Gauss points never land there
    for an even number of cells).
    """
    se = math.sqrt(eps)

    def f(x, y):
        dx, dy = x - 0.5, y - 0.5
        th = np.arctan2(dy, dx) + 0.5 * math.pi
        th = np.where(np.hypot(dx, dy) < 1e-300, 0.0, th)
        c, s = np.cos(th), np.sin(th)
        # R diag(1, se) R^T = I*se + (1 - se) * t t^T with t = (c, s)
        out = np.empty(np.shape(x) + (2, 2))
        out[..., 0, 0] = se + (1 - se) * c * c
        out[..., 0, 1] = (1 - se) * c * s
        out[..., 1, 0] = (1 - se) * c * s
        out[..., 1, 1] = se + (1 - se) * s * s
        return out

    return f


def q1_2d(N: int, sqrtK, D1: np.ndarray | None = None, agg: np.ndarray | None = None,
          desc: dict | None = None) -> Q1Problem:
    """Assemble G (8 rows per cell) for an N x N cell grid on [0,1]^2."""
    if N < 3:
        raise ValueError("need at least 3 cells per axis")
    h = 1.0 / N
    nint = N - 1
    C = N * N
    cells = np.arange(C)
    cj, ci = np.divmod(cells, N)
    ni = ci[:, None] + _DX[None, :]
    nj = cj[:, None] + _DY[None, :]
    interior = (ni >= 1) & (ni <= nint) & (nj >= 1) & (nj <= nint)
    node = (nj - 1) * nint + (ni - 1)

    # reference gradients of the four bilinear shape functions at the 4 points
    # dphi[q, a] on the physical cell (factor 1/h from the affine map)
    dphidx = ((2 * _DX[None, :] - 1) * ((1 - _DY[None, :]) * (1 - _ETA[:, None]) + _DY[None, :] * _ETA[:, None])) / h
    dphidy = (((1 - _DX[None, :]) * (1 - _XI[:, None]) + _DX[None, :] * _XI[:, None]) * (2 * _DY[None, :] - 1)) / h

    xq = (ci[:, None] + _XI[None, :]) * h
    yq = (cj[:, None] + _ETA[None, :]) * h
    S = sqrtK(xq, yq)  # (C, 4, 2, 2)
    sw = math.sqrt(h * h / 4.0)
    # vals[c, q, d, a]
    vals = sw * (S[:, :, :, 0, None] * dphidx[None, :, None, :] + S[:, :, :, 1, None] * dphidy[None, :, None, :])
    mask = np.broadcast_to(interior[:, None, None, :], vals.shape)
    col = np.broadcast_to(node[:, None, None, :], vals.shape)[mask].astype(np.int32)
    val = np.ascontiguousarray(vals[mask], dtype=np.float64)
    cnt = np.repeat(interior.sum(axis=1), 8)
    rowptr = np.zeros(8 * C + 1, dtype=np.int64)
    np.cumsum(cnt, out=rowptr[1:])
    n = nint * nint
    if agg is None:
        agg = np.zeros(n, dtype=np.int32)
    return Q1Problem(N=N, n=n, m=8 * C, rowptr=rowptr, col=col, val=val,
                     D1=None if D1 is None else np.ascontiguousarray(D1, dtype=np.float64),
                     agg=np.ascontiguousarray(agg, dtype=np.int32), desc=dict(desc or {}))


def block_aggregates_2d(N: int, bs: int) -> np.ndarray:
    """Level-0 aggregates: bs x bs blocks of interior nodes (last block narrower)."""
    nint = N - 1
    k = np.arange(nint * nint)
    jm1, im1 = np.divmod(k, nint)
    nb = -(-nint // bs)
    return (im1 // bs + nb * (jm1 // bs)).astype(np.int32)


def seeded_rhs(n: int, nrhs: int, seed: int) -> np.ndarray:
    """b ~ N(0, 1), n x nrhs, column-major (Fortran order)."""
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal((n, nrhs)))


# Workloads.  Each entry fixes the problem (grid, coefficient field, D1,
# level-0 aggregates, overlap, seed) and the recommended method parameters
# (per-level minimum coarsening ratio c, coarse size, threshold).
CONFIGS = {
    # 64 x 64 cells, theta = pi/6, eps = 1e-3, 4x4 aggregates, overlap 1
    "q1_64_rot": dict(N=64, field="rot", theta=math.pi / 6, eps=1e-3, d1=0.0, bs=4, overlap=1, seed=1,
                      c_min=(2, 3, 4), n_coarse=2000, thresh=0.1, nrhs=1),
    # 512 x 512 cells, one point of the (eps, theta) sweep
    "q1_512_rot": dict(N=512, field="rot", theta=math.pi / 6, eps=1e-4, d1=0.0, bs=4, overlap=1, seed=2,
                       c_min=(2, 3, 4), n_coarse=2000, thresh=0.1, nrhs=1),
    # the same with the kappa-derived threshold of Section 3.4 (kappa = 50)
    # and no cap on the kept eigenvectors
    "q1_512_rot_kappa": dict(N=512, field="rot", theta=math.pi / 6, eps=1e-4, d1=0.0, bs=4, overlap=1, seed=2,
                             c_min=(1,), n_coarse=2000, thresh=0.1, kappa=50.0, nrhs=1),
    # 2048 x 2048 cells, closed circular field lines, D1 = 1e-8 h^2; two
    # layers of overlap on level 0, one on coarse levels
    "q1_2048_circ": dict(N=2048, field="circ", theta=0.0, eps=1e-6, d1=1e-8, bs=8, overlap=2, coarse_overlap=1,
                         seed=3, c_min=(4, 5), n_coarse=2000, thresh=0.1, nrhs=1),
    # the same structure on 512 x 512 cells
    "q1_512_circ": dict(N=512, field="circ", theta=0.0, eps=1e-6, d1=1e-8, bs=8, overlap=2, coarse_overlap=1,
                        seed=3, c_min=(4, 5), n_coarse=2000, thresh=0.1, nrhs=1),
    # the closed-field-line workload with two layers of overlap on every level
    # (one layer above level 0 loses convergence as the grid grows)
    "q1_2048_circ_ov2": dict(N=2048, field="circ", theta=0.0, eps=1e-6, d1=1e-8, bs=8, overlap=2, coarse_overlap=2,
                             seed=3, c_min=(4, 5), n_coarse=2000, thresh=0.1, nrhs=1),
    "q1_512_circ_ov2": dict(N=512, field="circ", theta=0.0, eps=1e-6, d1=1e-8, bs=8, overlap=2, coarse_overlap=2,
                            seed=3, c_min=(4, 5), n_coarse=2000, thresh=0.1, nrhs=1),
    # the closed-field-line workload with the kappa-derived threshold of
    # Section 3.4 (kappa = 50) and no cap on the kept eigenvectors
    "q1_2048_circ_kappa": dict(N=2048, field="circ", theta=0.0, eps=1e-6, d1=1e-8, bs=8, overlap=2,
                               coarse_overlap=1, seed=3, c_min=(1,), n_coarse=2000, thresh=0.1, kappa=50.0, nrhs=1),
    # the paper's own finite-difference discretization (Section 4.1): 500 x 500
    # unknowns, theta = pi/6, 4x4 aggregates, the threshold from kappa = 50
    # (level-0 aggregates from one pass of standard aggregation, chosen by each solver itself)
    "fd_500_rot": dict(N=500, field="fd", theta=math.pi / 6, eps=1e-4, d1=0.0, bs=0, agg_passes=1, overlap=1,
                       seed=6, c_min=(2, 3, 4), n_coarse=2000, thresh=0.1, kappa=50.0, nrhs=1),
    "fd_500_blk": dict(N=500, field="fd", theta=math.pi / 6, eps=1e-4, d1=0.0, bs=4, overlap=1, seed=6,
                       c_min=(2, 3, 4), n_coarse=2000, thresh=0.1, kappa=50.0, nrhs=1),
    "fd_64_rot": dict(N=64, field="fd", theta=math.pi / 6, eps=1e-4, d1=0.0, bs=4, overlap=1, seed=6,
                      c_min=(2, 3, 4), n_coarse=2000, thresh=0.1, kappa=50.0, nrhs=1),
    # 3D: 128^3 hexahedral cells, K = eps I + (1 - eps) b b^T with b a smooth
    # seeded unit field, greedy strength-graph aggregates, 8 right-hand sides
    "q1_3d_128": dict(N=128, dim=3, field="fourier", theta=0.0, eps=1e-4, d1=0.0, bs=0, overlap=1, seed=4,
                      field_seed=44, soc=0.03, c_min=(3, 4), n_coarse=2000, thresh=0.1, nrhs=8),
    # the same on 32^3 cells (29,791 unknowns)
    "q1_3d_32": dict(N=32, dim=3, field="fourier", theta=0.0, eps=1e-4, d1=0.0, bs=0, overlap=1, seed=4,
                     field_seed=44, soc=0.03, c_min=(3, 4), n_coarse=2000, thresh=0.1, nrhs=8),
}

SWEEP_EPS = (1.0, 1e-2, 1e-4, 1e-6)
SWEEP_THETA = (0.0, math.pi / 8, math.pi / 6, math.pi / 4)


def config_problem(name: str | None = None, **over) -> tuple[Q1Problem, dict]:
    """Build the problem of a named workload (keyword overrides allowed).

    Returns (problem, params) where params carries overlap, c_min, n_coarse,
    thresh, seed and nrhs.
    """
    cfg = dict(CONFIGS[name]) if name is not None else {}
    cfg.update(over)
    N = int(cfg["N"])
    if cfg.get("dim", 2) == 3:
        from .q1_3d import field_sqrtK, greedy_aggregates, q1_3d, strength_graph

        prob = q1_3d(N, field_sqrtK(float(cfg["eps"]), int(cfg["field_seed"])),
                     desc=dict(name=name, dim=3, field="fourier", eps=cfg["eps"]))
        ip, ix = strength_graph(prob, float(cfg.get("soc", 0.03)))
        prob.agg = greedy_aggregates(ip, ix, prob.n)
        return prob, cfg
    if cfg["field"] == "fd":
        from .fd import fd_2d, fd_block_aggregates

        prob = fd_2d(N, float(cfg["theta"]), float(cfg["eps"]),
                     agg=fd_block_aggregates(N, int(cfg["bs"])) if cfg["bs"] else None,
                     desc=dict(name=name, field="fd", theta=cfg["theta"], eps=cfg["eps"], bs=cfg["bs"]))
        return prob, cfg
    if cfg["field"] == "rot":
        sk = rotated_sqrtK(float(cfg["theta"]), float(cfg["eps"]))
    elif cfg["field"] == "circ":
        sk = circular_sqrtK(float(cfg["eps"]))
    else:
        raise ValueError(cfg["field"])
    n = (N - 1) ** 2
    D1 = None
    if cfg.get("d1", 0.0):
        h = 1.0 / N
        D1 = np.full(n, float(cfg["d1"]) * h * h)
    agg = block_aggregates_2d(N, int(cfg["bs"]))
    prob = q1_2d(N, sk, D1=D1, agg=agg, desc=dict(name=name, **{k: cfg[k] for k in ("field", "theta", "eps", "d1", "bs")}))
    return prob, cfg
