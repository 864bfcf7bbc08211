"""GPU parity of the kappa-derived threshold on the finite-difference workload (Sections 3.4, 4.1).

The library colours the overlapping subdomains and takes the largest row multiplicity on every level on the
host, derives thresh_l = max{0.1, (kappa - n_color) / (n_color n_multiplicity)} and selects the local
eigenpairs with it.

What is unique is compared exactly or to the Q1 parity tolerances; what is not is checked for validity.
Both sides form the Schur complement of Eq. gevp-S from rows (a projector onto the Gamma rows cut at their
numerical rank).  On the finite-difference G some coarse levels have Gamma rows whose singular values run
evenly from 1e-14 to 1e-6 of the largest, across the rank cut: there the rank, and with it the coarse
spectra, is not fixed by FP64 data.  Up to the first such level (found in the oracle, first_ill_posed_level):
structure, n_color, n_multiplicity and thresh_l exactly, spectra and operators to the parity bars scaled by
the rows' conditioning (level_bar).  From it on: the library's own hierarchy is valid (mu in [0, 1], k_i
within its cap) and its PCG converges to the tolerance in a comparable number of iterations.
"""
import math

import numpy as np
import pytest

import oracle
from inputs import fd_2d, fd_block_aggregates, seeded_rhs
from oracle.construct import row_groups_from_csr
from test_gpu_parity import (_apply, _check_patterns, _check_spectra, _degenerate_cut, _rel, _x_at_iters,
                             first_ill_posed_level, level_bar)

pytestmark = pytest.mark.gpu

CASES = {
    # 48 x 48 unknowns, theta = pi/6, eps = 1e-4, 4x4 aggregates: three levels
    "fd_48": dict(N=48, theta=math.pi / 6, eps=1e-4, bs=4, c_min=(2, 3, 4), n_coarse=100, kappa=50.0),
    # ragged blocks (30 = 7 x 4 + 2 per axis), kappa small enough that the 0.1 floor binds on coarse levels
    "fd_30_floor": dict(N=30, theta=0.9, eps=1e-3, bs=4, c_min=(2, 3), n_coarse=60, kappa=6.0),
    # isotropic, standard aggregation chosen by each side: aggregates with k_i = 0 on levels 0 and 1 (no
    # lambda above the threshold), left out of the next level's dofs, rows and block graph
    "fd_16_iso": dict(N=16, theta=math.pi / 6, eps=1.0, bs=0, c_min=(2, 3, 4), n_coarse=20, kappa=50.0),
    # two levels at the diagonal angle, every eigenvector above the threshold kept (c_min = 1): level 0 is well
    # posed and the coarsest level is solved exactly, so the whole hierarchy and the solve have full parity
    "fd_48_2lvl": dict(N=48, theta=math.pi / 4, eps=1e-5, bs=0, c_min=(1,), n_coarse=1, kappa=50.0, L_max=2),
}


@pytest.fixture(scope="module")
def amg():
    from paper_2601_04112_gb300 import build

    build.build()
    import paper_2601_04112_gb300 as amg

    amg.load_library()
    return amg


def check_structure_upto(amg, H, ho, g):
    """Aggregates, Omega lists and the G_l / A_l patterns on levels <= g, k_i and the P_l pattern on levels < g,
    exactly."""
    for lvl in range(min(g, len(ho.levels) - 2) + 1):
        Lo = ho.levels[lvl]
        d = H.describe(lvl)
        assert d["n"] == Lo.n and d["nagg"] == Lo.nagg, lvl
        assert np.array_equal(H.export(lvl, amg.ARR_AGG), Lo.agg.astype(np.int32))
        ptr = H.export(lvl, amg.ARR_OMEGA_PTR)
        idx = H.export(lvl, amg.ARR_OMEGA_IDX)
        for i in range(Lo.nagg):
            assert np.array_equal(idx[ptr[i]:ptr[i + 1]], Lo.Omega[i].astype(np.int32)), (lvl, i)
        if lvl < g:
            assert np.array_equal(H.export(lvl, amg.ARR_K), np.array([Z.shape[1] for Z in Lo.Z], dtype=np.int32))
        # G_l and A_l patterns follow from the k_i above this level; P_l's from this level's k_i
        _check_patterns(amg, H, Lo, lvl, coarsest=lvl >= g)


def check_valid_from(amg, H, c_min, g):
    """The library's own levels >= g: mu in [0, 1] (S~ <= A_ww), 0 <= k_i <= max(1, |omega_i| / c_l)."""
    nl = H.num_levels
    for lvl in range(g, nl - 1):
        mu = H.export(lvl, amg.ARR_MU)
        assert mu.min() >= -1e-10 and mu.max() <= 1 + 1e-10, lvl
        k = H.export(lvl, amg.ARR_K)
        nom = H.export(lvl, amg.ARR_NOMEGA)
        cap = np.maximum(1, nom // c_min[min(lvl, len(c_min) - 1)])
        assert np.all(k >= 0) and np.all(k <= cap), lvl


def check_level0_operators(amg, H, ho):
    """A, RAS, RAS-T and P P^T on level 0 (the V-cycle reaches the coarse levels)."""
    rng = np.random.default_rng(11)
    Lo = ho.levels[0]
    x = rng.standard_normal(Lo.n)
    assert _rel(_apply(amg, H, amg.OP_A, 0, x, Lo.n), Lo.A @ x) <= 1e-13
    assert _rel(_apply(amg, H, amg.OP_RAS, 0, x, Lo.n), oracle.ras(Lo, x)) <= 1e-12
    assert _rel(_apply(amg, H, amg.OP_RAST, 0, x, Lo.n), oracle.rast(Lo, x)) <= 1e-12
    nn = ho.levels[1].n
    y = _apply(amg, H, amg.OP_PROLONG, 0, _apply(amg, H, amg.OP_RESTRICT, 0, x, nn), Lo.n)
    yo = Lo.P @ (Lo.P.T @ x)
    for i in range(Lo.nagg):
        if _degenerate_cut(Lo.mu[i], Lo.Z[i].shape[1], Lo.omega[i].shape[0]):
            continue
        om = Lo.omega[i]
        assert np.abs(y[om] - yo[om]).max() <= 1e-10 * np.abs(yo).max(), i


def check_solve(amg, H, ho, b):
    """FP64 and mixed PCG reach 1e-8; FP64 iterations within the oracle's +- 1 when the whole hierarchy is
    well posed, else at most 1.5 x the oracle's + 3."""
    xo, io = oracle.pcg(ho, b, tol=1e-8)
    H.set_precision(amg.FP64)
    xg, ig = H.solve(b, tol=1e-8)
    assert ig[0]["status"] == 0 and ig[0]["relres_true"] <= 1e-8
    if first_ill_posed_level(ho) == len(ho.levels) - 1:
        assert abs(ig[0]["iters"] - io["iters"]) <= 1
        assert _rel(_x_at_iters(H, b, io["iters"]), xo) <= level_bar(ho, len(ho.levels), 1e-10)
    else:
        assert ig[0]["iters"] <= 1.5 * io["iters"] + 3, (ig[0]["iters"], io["iters"])
    H.set_precision(amg.MIXED32)
    _, i32 = H.solve(b, tol=1e-8)
    assert i32[0]["status"] == 0 and i32[0]["relres_true"] <= 1e-8
    H.set_precision(amg.FP64)


def _both(amg, c):
    p = fd_2d(c["N"], c["theta"], c["eps"], agg=fd_block_aggregates(c["N"], c["bs"]) if c["bs"] else None)
    agg = p.agg
    if agg is None:
        sups, _ = row_groups_from_csr(p.rowptr, p.col, p.val, p.n, p.D1)
        agg, _ = oracle.standard_aggregation(sups, p.n, 1)
    L_max = c.get("L_max", 10)
    ho = oracle.setup(p.rowptr, p.col, p.val, p.n, p.D1, agg, overlap=1, c_min=c["c_min"],
                      n_coarse=c["n_coarse"], keep_local=True, kappa=c["kappa"], L_max=L_max)
    H = amg.Hierarchy.from_problem(p, overlap=1, c_min=c["c_min"], n_coarse=c["n_coarse"], kappa=c["kappa"],
                                   precision=amg.FP64, L_max=L_max)
    return p, ho, H


@pytest.mark.parametrize("name", list(CASES))
def test_kappa_threshold_per_level(amg, name):
    c = CASES[name]
    p, ho, H = _both(amg, c)
    st = H.stats()
    g = first_ill_posed_level(ho)
    lv = ho.levels[:g + 1]
    upto = min(g + 1, len(ho.levels) - 1)
    assert st["n_color"][:upto] == [L.n_color for L in lv][:upto]
    assert st["n_mult"][:upto] == [L.n_mult for L in lv][:upto]
    assert st["thresh"][:upto] == [L.thresh for L in lv][:upto]
    if name == "fd_30_floor":
        assert st["thresh"][1] == 0.1  # (6 - 5) / (5 * 3) < 0.1
    check_structure_upto(amg, H, ho, g)
    for lvl in range(g):
        _check_spectra(amg, H, ho, lvl)
    check_valid_from(amg, H, c["c_min"], g)


@pytest.mark.parametrize("name", list(CASES))
def test_kappa_operators_and_solve(amg, name):
    c = CASES[name]
    p, ho, H = _both(amg, c)
    check_level0_operators(amg, H, ho)
    check_solve(amg, H, ho, seeded_rhs(p.n, 1, 3)[:, 0])


def test_kappa_zero_keeps_fixed_threshold(amg):
    N = 24
    p = fd_2d(N, 0.5, 1e-3, agg=fd_block_aggregates(N, 4))
    H = amg.Hierarchy.from_problem(p, overlap=1, c_min=(2,), n_coarse=50, thresh=0.25)
    st = H.stats()
    assert all(t == 0.25 for t in st["thresh"]) and all(v == 0 for v in st["n_color"])


def test_empty_coarse_space_rejected(amg):
    """Isotropic 20 x 20: every aggregate of a coarse level keeps k_i = 0; setup fails cleanly (the oracle
    raises on the same level)."""
    p = fd_2d(20, math.pi / 6, 1.0)
    with pytest.raises(Exception, match="empty coarse space"):
        amg.Hierarchy.from_problem(p, overlap=1, c_min=(2, 3, 4), n_coarse=20, kappa=50.0)


def test_negative_kappa_rejected(amg):
    p = fd_2d(8, 0.5, 1e-3, agg=fd_block_aggregates(8, 4))
    with pytest.raises(Exception):
        amg.Hierarchy.from_problem(p, overlap=1, kappa=-1.0)
