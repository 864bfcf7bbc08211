"""Numeric setup of the oracle: Algorithm 1 step by step (test infrastructure).

For each level l (Algorithm 1), while l < L_max - 1 and n_l > n_coarse:

  1. aggregation: the level-0 aggregates are an input; on coarse levels the
     block graph (one node per previous-level aggregate, an edge where a row
     of G touches both) is aggregated with standard passes and every coarse
     dof of a block follows its block (the paper leaves the coarse rule
     open; this reading keeps the cycle independent of the basis chosen
     inside each block);
  2. overlapping subdomains and Boolean PoU (Section 2.2, Eq. pou2);
  3. smoother blocks A_i = A_l(Omega_i, Omega_i) and their Cholesky factors
     (Section 2.2; the factors are applied by triangular solves);
  4. SPSD splitting A~_i = sum_{rows in nz_i} g^T g / M (Lemma), kept as its
     rows Y = [X Y_G] (the rows of nz_i scaled by 1/sqrt(M)), A~_i = Y^T Y;
  5. reduced generalized eigenproblem on omega_i (Eq. gevp-S):
     A_ww u = lambda S~ u with S~ the Schur complement of A~_i onto omega_i,
     X^T (I - Pi) X with Pi the projector onto the Gamma rows (the
     pseudo-inverse reading); solved as S~ u = mu A_ww u, mu = 1/lambda
     ascending, so the largest lambda come first;
  6. selection: all lambda > thresh, at most max(1, floor(|omega_i|/c_l))
     (Section 3.4), thresh fixed or derived per level from kappa; an
     aggregate may keep none (k_i = 0); Z_i normalised so Z_i^T A_ww Z_i = I and the first entry
     within (1 - 1e-6) of the column's largest magnitude is positive;
  7. P_l = [R_{omega_1}^T Z_1 ... ] (Eq. mg-p), columns ordered by aggregate
     then by ascending mu;
  8. G_{l+1} = G_l P_l (its rows carried group by group), A_{l+1} =
     G_{l+1}^T G_{l+1} (Section 3.1, "Multilevel method").

The coarsest level is factored densely (Cholesky).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .structure import (
    cleanup_aggregates,
    multiplicity_and_nz,
    subdomain_colouring,
    kappa_threshold,
    overlapping_subdomains,
    row_groups_from_csr,
    structural_adjacency,
    vanek_aggregation,
)


@dataclass
class Level:
    n: int
    sups: list  # row-group supports of G_l
    grams: list  # row-group outer-product sums of G_l
    A: sp.csr_matrix  # A_l = G_l^T G_l (structural pattern kept)
    agg: np.ndarray | None = None
    nagg: int = 0
    omega: list = field(default_factory=list)
    gamma: list = field(default_factory=list)
    Omega: list = field(default_factory=list)
    M: np.ndarray | None = None
    nz: list = field(default_factory=list)
    touched: list = field(default_factory=list)
    chol: list = field(default_factory=list)  # lower Cholesky factor of each A_i
    mu: list = field(default_factory=list)  # all local eigenvalues mu (ascending)
    Z: list = field(default_factory=list)  # selected, A_ww-orthonormal
    k: np.ndarray | None = None
    col0: np.ndarray | None = None  # first coarse column of each aggregate
    P: sp.csr_matrix | None = None
    Atil: list = field(default_factory=list)  # kept only when keep_local
    S: list = field(default_factory=list)  # kept only when keep_local
    Ai: list = field(default_factory=list)  # kept only when keep_local
    rows: list | None = None  # schur="rows": per group its rows R_g (R_g^T R_g = grams[g])
    thresh: float = 0.1  # eigenvalue threshold used on this level
    n_color: int = 0  # with kappa: colours of the subdomain colouring
    n_mult: int = 0  # with kappa: largest row multiplicity M(j)


@dataclass
class Hierarchy:
    levels: list
    coarse_chol: np.ndarray  # lower Cholesky factor of the coarsest A_L
    params: dict


def assemble_A(sups, grams, n):
    """A = sum_g embed(H_g): the structural pattern of G^T G is kept."""
    rows, cols, vals = [], [], []
    for s, H in zip(sups, grams):
        rows.append(np.repeat(s, s.shape[0]))
        cols.append(np.tile(s, s.shape[0]))
        vals.append(H.ravel())
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    A = A.tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


def local_splitting(Omega_i, nz_i, sups, grams, M):
    """A~_i of the Lemma: sum over rows in nz_i of g^T W g, embedded in Omega_i."""
    m = Omega_i.shape[0]
    order = np.argsort(Omega_i)
    At = np.zeros((m, m))
    for g in nz_i:
        p = order[np.searchsorted(Omega_i, sups[g], sorter=order)]
        At[np.ix_(p, p)] += grams[g] / M[g]
    return At


def schur_complement(Atil, no, rtol):
    """S~ of Eq. gevp-S: A~_ww - A~_wG (A~_GG)^+ A~_Gw.

    Where A~_GG is singular (a Gamma node or direction that no row of nz_i
    sees) the inverse is read as the pseudo-inverse, eigenvalues at or below
    rtol * (largest eigenvalue) being treated as zero.
    """
    Aww = Atil[:no, :no]
    if Atil.shape[0] == no:
        S = Aww.copy()
    else:
        Awg = Atil[:no, no:]
        Agg = Atil[no:, no:]
        w, U = np.linalg.eigh(Agg)
        keep = w > rtol * max(w.max(), 0.0) if w.size else w > 0
        if not np.any(keep):
            S = Aww.copy()
        else:
            Uk = U[:, keep]
            T = Awg @ Uk
            S = Aww - (T / w[keep]) @ T.T
    return 0.5 * (S + S.T)


def local_splitting_rows(Omega_i, nz_i, sups, rows, M):
    """The rows behind A~_i of the Lemma: the rows of every group in nz_i,
    scaled by 1/sqrt(M) and embedded in Omega_i, so that Y^T Y = A~_i."""
    m = Omega_i.shape[0]
    order = np.argsort(Omega_i)
    blocks = []
    for g in nz_i:
        p = order[np.searchsorted(Omega_i, sups[g], sorter=order)]
        Yg = np.zeros((rows[g].shape[0], m))
        Yg[:, p] = rows[g] / np.sqrt(M[g])
        blocks.append(Yg)
    return np.vstack(blocks) if blocks else np.zeros((0, m))


def schur_complement_rows(Y, no, sv_rtol=None):
    """S~ of Eq. gevp-S from the rows Y = [X Y_G] (X on omega_i, Y_G on Gamma_i):
    A~_ww - A~_wG (A~_GG)^+ A~_Gw = X^T (I - Pi) X with Pi the orthogonal
    projector onto range(Y_G).  Pi comes from the SVD of Y_G, singular values
    at or below the rank tolerance being treated as zero: max(shape) * eps *
    (largest) by default (the numerical rank of Y_G), sv_rtol * (largest) when
    given; S~ = Xp^T Xp with Xp = (I - Pi) X, never a difference of Grams."""
    X = Y[:, :no]
    YG = Y[:, no:]
    if YG.shape[1] == 0 or YG.shape[0] == 0:
        S = X.T @ X
    else:
        U, sv, _ = np.linalg.svd(YG, full_matrices=False)
        rt = max(YG.shape) * np.finfo(np.float64).eps if sv_rtol is None else sv_rtol
        keep = sv > rt * sv.max() if sv.size and sv.max() > 0 else np.zeros(sv.shape, dtype=bool)
        Uk = U[:, keep]
        Xp = X - Uk @ (Uk.T @ X)
        S = Xp.T @ Xp
    return 0.5 * (S + S.T)


def local_gep(S, Aww, cap, thresh):
    """Reduced GEP (Eq. gevp-S) and the eigenvector selection of Section 3.4.

    Solves S~ u = mu A_ww u (mu = 1/lambda, ascending).  Keeps the first
    k = min(#{lambda > thresh}, cap) columns; mu <= 0 counts as lambda = inf.
    Returns (mu_all, Z) with Z^T A_ww Z = I.  Sign (the paper fixes none):
    the first entry whose magnitude is within a factor (1 - 1e-6) of the
    column's largest is made positive, so that entries equal in magnitude in
    exact arithmetic (symmetric or antisymmetric modes of symmetric
    aggregates) cannot trade places under rounding.
    """
    mu, V = sla.eigh(S, Aww)
    if thresh > 0:
        count = int(np.sum((mu <= 0) | (mu < 1.0 / thresh)))
    else:
        count = mu.shape[0]
    k = min(count, cap)
    Z = V[:, :k].copy()
    for c in range(k):
        a = np.abs(Z[:, c])
        j = int(np.nonzero(a >= (1.0 - 1e-6) * a.max())[0][0])
        if Z[j, c] < 0:
            Z[:, c] = -Z[:, c]
    return mu, Z


def _block_aggregation(prev):
    """Coarse aggregates on the block graph of the previous level.

    One vertex per previous-level aggregate that kept coarse dofs (k_i > 0;
    one with k_i = 0 has none on the next level and is left out), in
    ascending order; an edge where a row of G touches both."""
    live = np.flatnonzero(prev.k > 0)
    nb = live.shape[0]
    new_id = -np.ones(prev.nagg, dtype=np.int64)
    new_id[live] = np.arange(nb)
    r, c = [], []
    for t in prev.touched:
        t = new_id[t]
        t = t[t >= 0]
        if t.shape[0] > 1:
            r.append(np.repeat(t, t.shape[0]))
            c.append(np.tile(t, t.shape[0]))
    if r:
        B = sp.csr_matrix((np.ones(sum(x.shape[0] for x in r), dtype=np.int8),
                           (np.concatenate(r), np.concatenate(c))), shape=(nb, nb))
        B.setdiag(0)
        B.eliminate_zeros()
    else:
        B = sp.csr_matrix((nb, nb), dtype=np.int8)
    B.sort_indices()
    bagg, nagg = vanek_aggregation(B)
    agg = np.repeat(bagg, prev.k[live])
    return agg, nagg


def _next_groups(level):
    """Row groups of G_{l+1} = G_l P_l, merged by identical support.

    A row g of G_l becomes g P_l; its support is the coarse columns of every
    aggregate the row touches, and g^T g becomes P^T (g^T g) P restricted to
    those columns.  A row whose touched aggregates all kept k = 0 columns
    becomes zero and is dropped.
    """
    # row j of P is Z_a(position of j in omega_a, :) in the columns of a
    pos = np.zeros(level.n, dtype=np.int64)
    for i in range(level.nagg):
        pos[level.omega[i]] = np.arange(level.omega[i].shape[0])
    merged = {}
    for s, H, t in zip(level.sups, level.grams, level.touched):
        if not np.any(level.k[t] > 0):
            continue
        cs = np.concatenate([np.arange(level.col0[a], level.col0[a] + level.k[a]) for a in t])
        Pg = np.zeros((s.shape[0], cs.shape[0]))  # P(S_g, S'_g)
        off = np.concatenate([[0], np.cumsum([level.k[a] for a in t])])
        for r, j in enumerate(s):
            a = int(level.agg[j])
            c = int(np.searchsorted(t, a))
            Pg[r, off[c]:off[c + 1]] = level.Z[a][pos[j]]
        Hn = Pg.T @ H @ Pg
        key = tuple(int(a) for a in t)
        if key in merged:
            merged[key][1][...] += Hn
        else:
            merged[key] = (cs.astype(np.int64), Hn)
    keys = sorted(merged)
    return [merged[k][0] for k in keys], [merged[k][1] for k in keys]


def _next_groups_rows(level):
    """Row groups of G_{l+1} = G_l P_l carried as rows: each group's rows R_g
    become R_g P(S_g, S'_g); groups with one touched-aggregate set are stacked
    and compressed to the R factor of their QR decomposition (an orthogonal
    change of rows that keeps R^T R).  Same groups, supports and order as
    `_next_groups`."""
    pos = np.zeros(level.n, dtype=np.int64)
    for i in range(level.nagg):
        pos[level.omega[i]] = np.arange(level.omega[i].shape[0])
    merged = {}
    for s, R, t in zip(level.sups, level.rows, level.touched):
        if not np.any(level.k[t] > 0):
            continue
        cs = np.concatenate([np.arange(level.col0[a], level.col0[a] + level.k[a]) for a in t])
        Pg = np.zeros((s.shape[0], cs.shape[0]))
        off = np.concatenate([[0], np.cumsum([level.k[a] for a in t])])
        for r, j in enumerate(s):
            a = int(level.agg[j])
            c = int(np.searchsorted(t, a))
            Pg[r, off[c]:off[c + 1]] = level.Z[a][pos[j]]
        key = tuple(int(a) for a in t)
        merged.setdefault(key, (cs.astype(np.int64), []))[1].append(R @ Pg)
    keys = sorted(merged)
    sups, rows, grams = [], [], []
    for k in keys:
        cs, parts = merged[k]
        Rn = np.linalg.qr(np.vstack(parts), mode="r")
        sups.append(cs)
        rows.append(Rn)
        grams.append(Rn.T @ Rn)
    return sups, rows, grams


def setup(rowptr, col, val, n, D1, agg, overlap=1, c_min=(2, 3, 4), n_coarse=2000, L_max=10,
          thresh=0.1, schur_rtol=1e-12, keep_local=False, coarse_overlap=0, kappa=None, schur="rows",
          sv_rtol=None):
    """Build the multilevel hierarchy {A_l, G_l, P_l} of Algorithm 1.

    schur = "rows" (default) carries the rows of every G_l and forms S~ by an
    orthogonal projector on the Gamma rows, cut at their numerical rank
    (max(shape) eps of the largest singular value, or `sv_rtol` of it);
    "gram" forms S~ from the Gram A~_i with an eigenvalue-thresholded
    pseudo-inverse (`schur_rtol`).  The two agree in exact arithmetic; the
    row form resolves the small singular directions the Gram squares away.

    With `kappa` given, each level's eigenvalue threshold is derived from it
    (Section 3.4): max{0.1, (kappa - n_color) / (n_color n_multiplicity)}, with
    n_color the colours of `subdomain_colouring` and n_multiplicity the largest
    row multiplicity M(j) of the level's G; otherwise `thresh` holds on every
    level.

    `overlap` hops of neighbours form Omega_i on level 0; coarse levels use
    `coarse_overlap` hops (0: the same as level 0).  Algorithm 1 itself adds
    one layer of neighbours in A_l on every level."""
    if schur not in ("gram", "rows"):
        raise ValueError("schur must be 'gram' or 'rows'")
    sups, grams, rows = row_groups_from_csr(rowptr, col, val, n, D1, with_rows=True)
    A = assemble_A(sups, grams, n)
    levels = []
    cur = Level(n=n, sups=sups, grams=grams, A=A, rows=rows if schur == "rows" else None)
    lvl = 0
    agg0 = np.asarray(agg)
    while lvl < L_max - 1 and cur.n > n_coarse:
        adj = structural_adjacency(cur.sups, cur.n)
        if lvl == 0:
            cur.agg, cur.nagg = cleanup_aggregates(agg0, adj)
        else:
            cur.agg, cur.nagg = _block_aggregation(levels[-1])
        ov = overlap if lvl == 0 or coarse_overlap <= 0 else coarse_overlap
        cur.omega, cur.gamma, cur.Omega = overlapping_subdomains(cur.agg, cur.nagg, adj, ov)
        cur.M, cur.nz, cur.touched = multiplicity_and_nz(cur.sups, cur.agg, cur.nagg)
        if kappa is not None:
            _, cur.n_color = subdomain_colouring(cur.Omega, adj, cur.n)
            cur.n_mult = int(cur.M.max()) if cur.M.shape[0] else 1
            cur.thresh = kappa_threshold(float(kappa), cur.n_color, cur.n_mult)
        else:
            cur.thresh = thresh
        c = c_min[min(lvl, len(c_min) - 1)]
        ks = np.zeros(cur.nagg, dtype=np.int64)
        Acsr = cur.A
        for i in range(cur.nagg):
            om, Om = cur.omega[i], cur.Omega[i]
            no = om.shape[0]
            Ai = Acsr[Om][:, Om].toarray()
            L = np.linalg.cholesky(Ai)  # raises LinAlgError when A_i is not SPD
            cur.chol.append(L)
            if schur == "rows":
                Y = local_splitting_rows(Om, cur.nz[i], cur.sups, cur.rows, cur.M)
                At = Y.T @ Y
                S = schur_complement_rows(Y, no, sv_rtol)
            else:
                At = local_splitting(Om, cur.nz[i], cur.sups, cur.grams, cur.M)
                S = schur_complement(At, no, schur_rtol)
            mu, Z = local_gep(S, Ai[:no, :no], max(1, no // c), cur.thresh)
            cur.mu.append(mu)
            cur.Z.append(Z)
            ks[i] = Z.shape[1]
            if keep_local:
                cur.Atil.append(At)
                cur.S.append(S)
                cur.Ai.append(Ai)
        cur.k = ks
        cur.col0 = np.zeros(cur.nagg + 1, dtype=np.int64)
        np.cumsum(ks, out=cur.col0[1:])
        nc = int(cur.col0[-1])
        if nc == 0:  # no lambda above any level's threshold: nothing to coarsen to
            raise ValueError(f"level {lvl} produced an empty coarse space")
        r, cc, v = [], [], []
        for i in range(cur.nagg):
            Z = cur.Z[i]
            r.append(np.repeat(cur.omega[i], Z.shape[1]))
            cc.append(np.tile(np.arange(cur.col0[i], cur.col0[i + 1]), Z.shape[0]))
            v.append(Z.ravel())
        cur.P = sp.csr_matrix((np.concatenate(v), (np.concatenate(r), np.concatenate(cc))), shape=(cur.n, nc))
        cur.P.sort_indices()
        levels.append(cur)
        if schur == "rows":
            nsups, nrows, ngrams = _next_groups_rows(cur)
        else:
            nsups, ngrams = _next_groups(cur)
            nrows = None
        cur = Level(n=nc, sups=nsups, grams=ngrams, A=assemble_A(nsups, ngrams, nc), rows=nrows)
        lvl += 1
    levels.append(cur)
    AL = cur.A.toarray()
    coarse = np.linalg.cholesky(AL)
    params = dict(overlap=overlap, coarse_overlap=coarse_overlap, c_min=tuple(c_min), n_coarse=n_coarse, L_max=L_max,
                  thresh=thresh, kappa=kappa,
                  schur_rtol=schur_rtol, schur=schur, sv_rtol=sv_rtol)
    return Hierarchy(levels=levels, coarse_chol=coarse, params=params)
