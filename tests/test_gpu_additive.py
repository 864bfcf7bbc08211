"""GPU parity of the additive two-level method (cycle = 1): M_2^{-1} =
P (P^T A P)^{-1} P^T + sum_i R_i^T A_i^{-1} R_i on a two-level hierarchy,
against the oracle's two_level_additive, and PCG with it against the
oracle's PCG with the same preconditioner."""
import math

import numpy as np
import pytest

import oracle
from inputs import block_aggregates_2d, q1_2d, rotated_sqrtK, seeded_rhs
from oracle.cycle import two_level_additive

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amg():
    from paper_2601_04112_gb300 import build

    build.build()
    import paper_2601_04112_gb300 as amg

    amg.load_library()
    return amg


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("tau,N,bs", [(4.0, 12, 3), (2.0, 16, 4), (0.1, 20, 4)])
def test_additive_two_level_matches_oracle(amg, tau, N, bs):
    import torch

    p = q1_2d(N, rotated_sqrtK(math.pi / 6, 1e-2), agg=block_aggregates_2d(N, bs))
    kw = dict(overlap=1, c_min=(1,), n_coarse=1, L_max=2, thresh=tau)
    ho = oracle.setup(p.rowptr, p.col, p.val, p.n, p.D1, p.agg, **kw)
    H = amg.Hierarchy.from_problem(p, cycle=1, **kw)
    assert H.num_levels == 2
    rng = np.random.default_rng(5)
    for _ in range(3):
        x = rng.standard_normal(p.n)
        y = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        H.apply(amg.OP_M2, 0, torch.from_numpy(x).cuda(), y)
        torch.cuda.synchronize()
        assert _rel(y.cpu().numpy(), two_level_additive(ho, x)) <= 1e-11
    b = seeded_rhs(p.n, 1, 3)[:, 0]
    xo, io = oracle.pcg(ho, b, tol=1e-8, precond=two_level_additive)
    xg, ig = H.solve(b, tol=1e-8)
    assert ig[0]["status"] == 0 and ig[0]["relres_true"] <= 1e-8
    assert abs(ig[0]["iters"] - io["iters"]) <= 1
    H.set_max_iter(io["iters"])  # the iterate at the oracle's count, not only at stop
    xk, ik = H.solve(b, tol=0.0)
    H.set_max_iter(1000)
    assert ik[0]["iters"] == io["iters"]
    assert _rel(np.asarray(xk).ravel(), xo) <= 1e-10
    # several right-hand sides (solved column by column) agree with single solves
    B = seeded_rhs(p.n, 3, 4)
    X, infos = H.solve(B, tol=1e-8)
    for j in range(3):
        xj, _ = H.solve(B[:, j], tol=1e-8)
        assert infos[j]["status"] == 0
        assert _rel(np.asarray(X)[:, j], np.asarray(xj).ravel()) <= 1e-12


def test_additive_two_level_refuses_what_it_does_not_define(amg):
    p = q1_2d(16, rotated_sqrtK(0.3, 1e-2), agg=block_aggregates_2d(16, 4))
    with pytest.raises(amg.AmgddError):  # three levels: no exact level-1 solve
        amg.Hierarchy.from_problem(p, overlap=1, c_min=(2,), n_coarse=20, L_max=6, cycle=1)
    with pytest.raises(amg.AmgddError):  # FP64 only
        amg.Hierarchy.from_problem(p, overlap=1, c_min=(1,), n_coarse=1, L_max=2, cycle=1, precision=amg.MIXED32)
    H = amg.Hierarchy.from_problem(p, overlap=1, c_min=(1,), n_coarse=1, L_max=2, cycle=1)
    with pytest.raises(amg.AmgddError):
        H.set_precision(amg.MIXED32)
    Hm = amg.Hierarchy.from_problem(p, overlap=1, c_min=(1,), n_coarse=1, L_max=2)
    import torch

    x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    with pytest.raises(amg.AmgddError):  # M2 needs a cycle = 1 hierarchy
        Hm.apply(amg.OP_M2, 0, x, torch.zeros_like(x))
