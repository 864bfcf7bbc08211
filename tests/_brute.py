"""Literal, row-by-row constructions used to pin the oracle on tiny grids.

Everything here works on the dense m x n matrix G (rows sqrt(D1_jj) e_j^T
appended), row by row, with no grouping of rows, and takes the Schur
complement through an SVD projector onto range(Y) instead of a
pseudo-inverse of a Gram matrix.  It shares no code with oracle/.
"""
import numpy as np


def dense_G(p):
    G = p.G_scipy().toarray()
    pat = p.G_scipy().copy()
    pat.data[:] = 1.0
    P = pat.toarray() != 0
    if p.D1 is not None:
        G = np.vstack([G, np.diag(np.sqrt(p.D1))])
        P = np.vstack([P, np.eye(p.n, dtype=bool)])
    return G, P


def omega_sets(P, agg, overlap):
    """Omega_i by breadth-first hops on the structural graph of G^T G."""
    n = P.shape[1]
    adj = (P.T.astype(int) @ P.astype(int)) > 0
    out = []
    for i in range(agg.max() + 1):
        om = np.nonzero(agg == i)[0]
        cur = np.zeros(n, dtype=bool)
        cur[om] = True
        for _ in range(overlap):
            cur = cur | adj[cur].any(axis=0)
        ga = np.array(sorted(set(np.nonzero(cur)[0]) - set(om)), dtype=np.int64)
        out.append((om, ga))
    return out


def row_multiplicity(P, agg):
    return np.array([len(set(agg[np.nonzero(P[l])[0]])) for l in range(P.shape[0])])


def nz_rows(P, agg, i):
    return np.array([l for l in range(P.shape[0]) if np.any(agg[np.nonzero(P[l])[0]] == i)], dtype=np.int64)


def literal_splitting(G, P, agg, i, Om):
    M = row_multiplicity(P, agg)
    rows = nz_rows(P, agg, i)
    X = G[np.ix_(rows, Om)]
    return X.T @ np.diag(1.0 / M[rows]) @ X


def svd_schur(G, P, agg, i, om, ga, rtol=1e-12):
    """X^T (I - Pi_Y) X with X, Y the W^{1/2}-weighted rows of nz_i."""
    M = row_multiplicity(P, agg)
    rows = nz_rows(P, agg, i)
    w = 1.0 / np.sqrt(M[rows])
    X = w[:, None] * G[np.ix_(rows, om)]
    if ga.size == 0:
        return X.T @ X
    Y = w[:, None] * G[np.ix_(rows, ga)]
    U, s, _ = np.linalg.svd(Y, full_matrices=False)
    r = int(np.sum(s > np.sqrt(rtol) * s.max())) if s.size and s.max() > 0 else 0
    Ur = U[:, :r]
    R = X - Ur @ (Ur.T @ X)
    return R.T @ R
