"""Level-0 aggregation through the C ABI (amgdd_aggregate, and amgdd_setup with agg = NULL) against the
oracle's standard aggregation with repeated passes (Section 3.3).

The library runs the passes on the device in parallel rounds (pass 1's roots as the first maximal
independent set of the distance-2 graph, pass 3's as that of the graph on the leftovers); the oracle
visits the unknowns one by one.  Aggregate ids are integers: bit-exact, on structured grids, on
random patterns with isolated unknowns and many pass-2 joins, and on grids large enough for hundreds
of rounds.  (With every edge strong, pass 3 never has work: an unknown that is not a root had a
neighbour aggregated at its visit, so pass 2 places it.)  The hierarchy built from library-chosen aggregates then matches the
oracle's hierarchy on the same aggregates (structure, spectra, level operators, PCG).
"""
import math

import numpy as np
import pytest

import oracle
from inputs import fd_2d, q1_2d, rotated_sqrtK, seeded_rhs
from inputs.q1 import config_problem
from oracle.construct import row_groups_from_csr
from test_gpu_kappa import check_level0_operators, check_solve, check_structure_upto, check_valid_from
from test_gpu_parity import first_ill_posed_level
from test_gpu_parity import _check_spectra

pytestmark = pytest.mark.gpu

PROBLEMS = {
    "fd_40": lambda: fd_2d(40, math.pi / 6, 1e-4),
    "q1_33": lambda: q1_2d(33, rotated_sqrtK(0.4, 1e-3)),
    "q1_3d_10": lambda: config_problem("q1_3d_32", N=10)[0],
    "q1_129": lambda: q1_2d(129, rotated_sqrtK(0.4, 1e-3)),
    "q1_3d_18": lambda: config_problem("q1_3d_32", N=18)[0],
}


@pytest.fixture(scope="module")
def amg():
    from paper_2601_04112_gb300 import build

    build.build()
    import paper_2601_04112_gb300 as amg

    amg.load_library()
    return amg


def _oracle_agg(p, passes):
    sups, _ = row_groups_from_csr(p.rowptr, p.col, p.val, p.n, p.D1)
    return oracle.standard_aggregation(sups, p.n, passes)


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("passes", [1, 2, 3])
def test_aggregate_matches_oracle(amg, name, passes):
    p = PROBLEMS[name]()
    ao, no = _oracle_agg(p, passes)
    ag, ng = amg.aggregate(p.rowptr, p.col, p.n, passes)
    assert ng == no and np.array_equal(ag, ao.astype(np.int32))


def _random_pattern(seed, n, m):
    """Rows of 1-4 distinct random columns; some columns in no row (isolated unknowns)."""
    rng = np.random.default_rng(seed)
    used = rng.permutation(n)[: int(0.9 * n)]
    rp, cl = [0], []
    for _ in range(m):
        k = int(rng.integers(1, 5))
        cl.extend(sorted(set(rng.choice(used, size=k).tolist())))
        rp.append(len(cl))
    return np.array(rp, dtype=np.int64), np.array(cl, dtype=np.int32)


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("passes", [1, 2])
def test_aggregate_random_patterns_match_oracle(amg, seed, passes):
    n = 3000
    rp, cl = _random_pattern(seed, n, 2200)
    sups, _ = row_groups_from_csr(rp, cl, np.ones(len(cl)), n)
    ao, no = oracle.standard_aggregation(sups, n, passes)
    ag, ng = amg.aggregate(rp, cl, n, passes)
    assert ng == no and np.array_equal(ag, ao.astype(np.int32))


def test_aggregate_path_by_hand(amg):
    n = 27
    rp = np.arange(0, 2 * (n - 1) + 1, 2)
    cl = np.array(sum(([i, i + 1] for i in range(n - 1)), []))
    ag, ng = amg.aggregate(rp, cl, n, 2)
    assert ng == 3 and ag.tolist() == [0] * 5 + [1] * 9 + [2] * 13


def test_aggregate_device_buffers(amg):
    import ctypes

    import torch

    p = PROBLEMS["fd_40"]()
    rp = torch.from_numpy(p.rowptr.astype(np.int64)).cuda()
    cl = torch.from_numpy(p.col.astype(np.int32)).cuda()
    vl = torch.from_numpy(p.val).cuda()
    out = torch.full((p.n,), -5, dtype=torch.int32, device="cuda")
    csr = amg.Csr(m=p.m, n=p.n, nnz=len(p.col), rowptr=rp.data_ptr(), col=cl.data_ptr(), val=vl.data_ptr(),
                  mem=amg.DEVICE)
    na = ctypes.c_int64()
    lib = amg.load_library()
    st = lib.amgdd_aggregate(ctypes.byref(csr), 2, torch.cuda.current_stream().cuda_stream, out.data_ptr(),
                             ctypes.byref(na))
    assert st == 0
    ao, no = _oracle_agg(p, 2)
    assert na.value == no and np.array_equal(out.cpu().numpy(), ao.astype(np.int32))


def test_aggregate_rejects_bad_input(amg):
    with pytest.raises(Exception):
        amg.aggregate(np.array([0, 2]), np.array([1, 0]), 3, 1)  # columns not increasing
    with pytest.raises(Exception):
        amg.aggregate(np.array([0, 1]), np.array([0]), 2, 0)  # passes < 1


@pytest.mark.parametrize("passes", [1, 2])
def test_setup_without_aggregates(amg, passes):
    p = fd_2d(48, math.pi / 6, 1e-4)
    ao, _ = _oracle_agg(p, passes)
    ho = oracle.setup(p.rowptr, p.col, p.val, p.n, p.D1, ao, overlap=1, c_min=(2, 3, 4), n_coarse=100,
                      keep_local=True, kappa=50.0)
    H = amg.Hierarchy(p.rowptr, p.col, p.val, p.n, agg=None, overlap=1, c_min=(2, 3, 4), n_coarse=100,
                      kappa=50.0, agg_passes=passes, precision=amg.FP64)
    # the finite-difference coarse levels are compared as in the kappa tests (exactly up to the first level
    # whose pseudo-inverse is not well posed, for validity and convergence from it on)
    g = first_ill_posed_level(ho)
    check_structure_upto(amg, H, ho, g)
    for lvl in range(g):
        _check_spectra(amg, H, ho, lvl)
    check_valid_from(amg, H, (2, 3, 4), g)
    check_level0_operators(amg, H, ho)
    check_solve(amg, H, ho, seeded_rhs(p.n, 1, 5)[:, 0])
