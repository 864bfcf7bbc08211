"""Batched right-hand sides (amgdd_solve with nrhs > 1) against single solves
and the FP64 oracle.

A batch of K in {2, 4, 8, 16, 32} columns runs K independent CGs that share
every V-cycle and A-apply launch (gather-GEMVs whose staged input would not
fit shared memory at K columns run over column tiles).  Each column follows the single right-hand-side
recurrence, so in FP64 it must reach the oracle's iterate (same iteration
count, 1e-9 relative; the batched kernels only sum in another order), and in
mixed precision it must reach the 1e-8 relative residual.  Columns that
converge early keep their iterate while the others continue.
"""
import numpy as np
import pytest

import oracle
from inputs import seeded_rhs

from tests.test_gpu_parity import CASES, _gpu, _oracle, _problem, _rel, _torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amg():
    from paper_2601_04112_gb300 import build

    build.build()
    import paper_2601_04112_gb300 as amg

    amg.load_library()
    return amg


def _cols(x):
    return x if x.ndim == 2 else x[:, None]


@pytest.mark.parametrize("name", list(CASES))
def test_batched_fp64_matches_single_and_oracle(amg, name):
    c = CASES[name]
    p = _problem(c)
    H = _gpu(amg, p, c["overlap"], c["c_min"], c["n_coarse"], coarse_overlap=c.get("coarse_overlap", 0))
    ho = _oracle(p, c["overlap"], c["c_min"], c["n_coarse"], coarse_overlap=c.get("coarse_overlap", 0))
    B = seeded_rhs(p.n, 5, 11)  # a batch of 8 with three padding columns
    B[:, 3] *= 1e-3  # scale does not change the iteration (relative test)
    X, infos = H.solve(B, tol=1e-8)
    X = _cols(np.asarray(X))
    assert len(infos) == 5
    for j in range(5):
        assert infos[j]["status"] == 0 and infos[j]["relres_true"] <= 1e-8
        xs, isg = H.solve(np.ascontiguousarray(B[:, j]), tol=1e-8)
        assert abs(infos[j]["iters"] - isg[0]["iters"]) <= 1
        assert _rel(X[:, j], _cols(xs)[:, 0]) <= 1e-9
        xo, io = oracle.pcg(ho, B[:, j], tol=1e-8)
        # the batch's column j after exactly the oracle's iteration count (tol = 0 runs every column to the
        # limit), not only at stop
        H.set_max_iter(io["iters"])
        Xk, ik = H.solve(B, tol=0.0)
        H.set_max_iter(1000)
        assert ik[j]["iters"] == io["iters"]
        assert _rel(_cols(np.asarray(Xk))[:, j], xo) <= 1e-9


@pytest.mark.parametrize("name", ["q1_64", "overlap2_d1"])
def test_batched_mixed_reaches_tolerance(amg, name):
    c = CASES[name]
    p = _problem(c)
    H = _gpu(amg, p, c["overlap"], c["c_min"], c["n_coarse"], coarse_overlap=c.get("coarse_overlap", 0))
    B = seeded_rhs(p.n, 8, 12)
    _, i64 = H.solve(B, tol=1e-8)
    H.set_precision(amg.MIXED32)
    X, i32 = H.solve(B, tol=1e-8)
    for j in range(8):
        assert i32[j]["status"] == 0 and i32[j]["relres_true"] <= 1e-8
        assert i32[j]["iters"] <= i64[j]["iters"] + 5


def test_batched_groups_zero_and_early_columns(amg):
    """nrhs = 10 runs as a batch of 8 and a batch of 2.  A zero column stops
    at once and keeps x = 0 while the other columns of its batch iterate;
    every other column matches its single solve."""
    t = _torch()
    c = CASES["ragged_3lvl"]
    p = _problem(c)
    H = _gpu(amg, p, c["overlap"], c["c_min"], c["n_coarse"], coarse_overlap=c.get("coarse_overlap", 0))
    B = seeded_rhs(p.n, 10, 13)
    B[:, 2] = 0.0
    Bd = t.from_numpy(B).cuda()  # (n, nrhs) tensor; the binding passes it column-major
    Xd, infos = H.solve(Bd, tol=1e-8)
    X = Xd.cpu().numpy()
    assert infos[2]["iters"] == 0 and np.all(X[:, 2] == 0.0)
    for j in range(10):
        if j == 2:
            continue
        assert infos[j]["status"] == 0 and infos[j]["relres_true"] <= 1e-8
        xs, isg = H.solve(np.ascontiguousarray(B[:, j]), tol=1e-8)
        assert abs(infos[j]["iters"] - isg[0]["iters"]) <= 1
        assert _rel(X[:, j], _cols(xs)[:, 0]) <= 1e-9


@pytest.mark.parametrize("name", ["q1_64", "circ_ov2", "q1_3d_12"])
def test_wide_batches_match_single_and_oracle(amg, name):
    """With batch_cols = 32, 20 columns run as one batch of 32 (the column
    tiles of the wide launches included); each column matches its single
    solve and, after the oracle's iteration count, the oracle's iterate.  A
    narrower batch before and after the wide one (the workspace grows and
    the batched graphs are captured again) gives the same columns as
    before."""
    c = CASES[name]
    p = _problem(c)
    H = amg.Hierarchy.from_problem(p, overlap=c["overlap"], c_min=c["c_min"], n_coarse=c["n_coarse"],
                                   coarse_overlap=c.get("coarse_overlap", 0), batch_cols=32)
    ho = _oracle(p, c["overlap"], c["c_min"], c["n_coarse"], coarse_overlap=c.get("coarse_overlap", 0))
    B = seeded_rhs(p.n, 20, 17)
    X3, i3 = H.solve(np.ascontiguousarray(B[:, :3]), tol=1e-8)
    X, infos = H.solve(B, tol=1e-8)
    X = _cols(np.asarray(X))
    X3b, i3b = H.solve(np.ascontiguousarray(B[:, :3]), tol=1e-8)
    for j in range(3):
        assert abs(i3b[j]["iters"] - i3[j]["iters"]) <= 1  # atomic sums reorder between runs
        assert _rel(_cols(np.asarray(X3b))[:, j], _cols(np.asarray(X3))[:, j]) <= 1e-9
    for j in range(20):
        assert infos[j]["status"] == 0 and infos[j]["relres_true"] <= 1e-8
    for j in (0, 7, 19):
        xs, isg = H.solve(np.ascontiguousarray(B[:, j]), tol=1e-8)
        assert abs(infos[j]["iters"] - isg[0]["iters"]) <= 1
        assert _rel(X[:, j], _cols(xs)[:, 0]) <= 1e-9
        xo, io = oracle.pcg(ho, B[:, j], tol=1e-8)
        H.set_max_iter(io["iters"])
        Xk, ik = H.solve(B, tol=0.0)
        H.set_max_iter(1000)
        assert ik[j]["iters"] == io["iters"]
        assert _rel(_cols(np.asarray(Xk))[:, j], xo) <= 1e-9


def test_sixty_four_columns_mixed(amg):
    """64 columns in mixed precision, in two batches of 32 and in four of 16,
    reach the tolerance with at most a few iterations more than FP64."""
    c = CASES["q1_64"]
    p = _problem(c)
    H = amg.Hierarchy.from_problem(p, overlap=c["overlap"], c_min=c["c_min"], n_coarse=c["n_coarse"], batch_cols=32)
    H16 = amg.Hierarchy.from_problem(p, overlap=c["overlap"], c_min=c["c_min"], n_coarse=c["n_coarse"], batch_cols=16,
                                     precision=amg.MIXED32)
    _, i16 = H16.solve(seeded_rhs(p.n, 64, 18), tol=1e-8)
    assert all(i["status"] == 0 and i["relres_true"] <= 1e-8 for i in i16)
    B = seeded_rhs(p.n, 64, 18)
    _, i64 = H.solve(B, tol=1e-8)
    H.set_precision(amg.MIXED32)
    X, i32 = H.solve(B, tol=1e-8)
    assert len(i32) == 64
    A = _oracle(p, c["overlap"], c["c_min"], c["n_coarse"]).levels[0].A
    X = np.asarray(X)
    for j in range(64):
        assert i32[j]["status"] == 0 and i32[j]["relres_true"] <= 1e-8
        assert i32[j]["iters"] <= i64[j]["iters"] + 5
    for j in (0, 31, 32, 63):
        assert np.linalg.norm(B[:, j] - A @ X[:, j]) <= 1.01e-8 * np.linalg.norm(B[:, j])
