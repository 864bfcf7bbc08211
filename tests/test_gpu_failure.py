"""Failure detection of the bounded device-side waits, tested without a GPU
fault: a grid barrier that one CTA never reaches and an mbarrier that nothing
completes must each give up after their limit, report AMGDD_ERR_TIMEOUT
through the error word, and leave the context usable."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_bounded_waits_report_timeout_and_context_survives():
    from paper_2601_04112_gb300 import build

    build.build()
    import paper_2601_04112_gb300 as amg
    from inputs import block_aggregates_2d, q1_2d, rotated_sqrtK, seeded_rhs

    amg.load_library()
    bar, mb = amg.selftest_wait_timeouts()
    assert bar == -9 and mb == -9
    # the context still runs a solve
    p = q1_2d(16, rotated_sqrtK(0.3, 1e-2), agg=block_aggregates_2d(16, 4))
    H = amg.Hierarchy.from_problem(p, overlap=1, c_min=(2,), n_coarse=30)
    b = seeded_rhs(p.n, 1, 2)[:, 0]
    x, info = H.solve(b, tol=1e-8)
    assert info[0]["status"] == 0 and info[0]["relres_true"] <= 1e-8
    assert np.isfinite(np.asarray(x)).all()
