"""amgdd_apply_noalloc against amgdd_apply, through the C ABI (GPU).

Some callers may not allocate device memory after setup (for instance a
serving loop that runs under a fixed memory budget owned by another
component).  amgdd_apply_noalloc gives them every operator of amgdd_apply
without any allocation: in MIXED32 its FP32 staging vectors live in one
fixed file-scope device array.  This test checks, for every operator, level
and precision, that two calls in a row agree with amgdd_apply within the
tolerances the parity tests use (1e-12 relative in FP64; the FP32 cycle
reorders atomic additions, so 1e-5 there), the additive two-level operator
M_2 too, that the calls allocate nothing (the library's own count of device
allocations does not move over 100 calls, while one amgdd_apply in MIXED32
moves it, and the device's free memory is unchanged), and that levels larger
than the fixed staging size are refused with an error instead of touching
memory.  The file is named so that pytest collects it last.
"""
import math

import numpy as np
import pytest

from inputs import block_aggregates_2d, q1_2d, rotated_sqrtK

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


def test_noalloc_matches_apply_twice(amg):
    import torch

    p = q1_2d(24, rotated_sqrtK(0.5, 1e-2), agg=block_aggregates_2d(24, 4))
    H = amg.Hierarchy.from_problem(p, overlap=1, c_min=(2, 3), n_coarse=60)
    lib = H._lib
    stream = torch.cuda.current_stream().cuda_stream
    g = torch.Generator(device="cuda").manual_seed(3)
    nl = H.num_levels
    sizes = [H.describe(l)["n"] for l in range(nl)]
    ops = [amg.OP_A, amg.OP_RAS, amg.OP_RAST, amg.OP_RESTRICT, amg.OP_PROLONG, amg.OP_VCYCLE]
    for prec, tol in ((amg.FP64, 1e-12), (amg.MIXED32, 1e-5)):
        H.set_precision(prec)
        for lvl in range(nl - 1):
            for op in ops:
                nin = sizes[lvl + 1] if op == amg.OP_PROLONG else sizes[lvl]
                nout = sizes[lvl + 1] if op == amg.OP_RESTRICT else sizes[lvl]
                x = torch.randn(nin, dtype=torch.float64, device="cuda", generator=g)
                ref = torch.zeros(nout, dtype=torch.float64, device="cuda")
                H.apply(op, lvl, x, ref)
                for _ in range(2):
                    y = torch.full((nout,), float("nan"), dtype=torch.float64, device="cuda")
                    st = lib.amgdd_apply_noalloc(H._h, op, lvl, x.data_ptr(), y.data_ptr(), stream)
                    assert st == 0, lib.amgdd_last_error()
                    assert _rel(y.cpu().numpy(), ref.cpu().numpy()) <= tol, (prec, lvl, op)
        # the coarsest solve
        xc = torch.randn(sizes[-1], dtype=torch.float64, device="cuda", generator=g)
        ref = torch.zeros_like(xc)
        H.apply(amg.OP_COARSE, nl - 1, xc, ref)
        for _ in range(2):
            y = torch.zeros_like(xc)
            assert lib.amgdd_apply_noalloc(H._h, amg.OP_COARSE, nl - 1, xc.data_ptr(), y.data_ptr(), stream) == 0
            assert _rel(y.cpu().numpy(), ref.cpu().numpy()) <= 1e-12


def _allocs(H):
    return int(H.stats()["process_device_allocs"])


def test_noalloc_allocates_nothing(amg):
    import torch

    p = q1_2d(24, rotated_sqrtK(0.5, 1e-2), agg=block_aggregates_2d(24, 4))
    H = amg.Hierarchy.from_problem(p, overlap=1, c_min=(2, 3), n_coarse=60, precision=amg.MIXED32)
    lib = H._lib
    stream = torch.cuda.current_stream().cuda_stream
    x = torch.randn(p.n, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    # control: amgdd_apply stages MIXED32 vectors in buffers it allocates, and the count sees them
    a0 = _allocs(H)
    H.apply(amg.OP_VCYCLE, 0, x, y)
    assert _allocs(H) > a0
    for prec in (amg.MIXED32, amg.FP64):
        H.set_precision(prec)
        ops = (amg.OP_VCYCLE, amg.OP_RAS, amg.OP_RAST, amg.OP_A)
        # one call of each operator first: the first call on the device looks up the staging array's
        # address, and CUDA loads a kernel's module at its first launch (lazy loading), which takes
        # device memory outside the library's own allocations
        a0 = _allocs(H)
        for op in ops:
            assert lib.amgdd_apply_noalloc(H._h, op, 0, x.data_ptr(), y.data_ptr(), stream) == 0
        torch.cuda.synchronize()
        assert _allocs(H) == a0, prec
        free0 = torch.cuda.mem_get_info()[0]
        for i in range(100):
            op = ops[i % 4]
            assert lib.amgdd_apply_noalloc(H._h, op, 0, x.data_ptr(), y.data_ptr(), stream) == 0, \
                lib.amgdd_last_error()
        torch.cuda.synchronize()
        assert _allocs(H) == a0, prec
        assert torch.cuda.mem_get_info()[0] == free0, prec


def test_noalloc_additive_two_level_matches_apply_twice(amg):
    import torch

    p = q1_2d(16, rotated_sqrtK(math.pi / 6, 1e-2), agg=block_aggregates_2d(16, 4))
    H = amg.Hierarchy.from_problem(p, overlap=1, c_min=(1,), n_coarse=1, L_max=2, thresh=2.0, cycle=1)
    lib = H._lib
    stream = torch.cuda.current_stream().cuda_stream
    g = torch.Generator(device="cuda").manual_seed(7)
    x = torch.randn(p.n, dtype=torch.float64, device="cuda", generator=g)
    ref = torch.zeros_like(x)
    H.apply(amg.OP_M2, 0, x, ref)
    a0 = _allocs(H)
    for _ in range(2):
        y = torch.full_like(x, float("nan"))
        assert lib.amgdd_apply_noalloc(H._h, amg.OP_M2, 0, x.data_ptr(), y.data_ptr(), stream) == 0, \
            lib.amgdd_last_error()
        assert _rel(y.cpu().numpy(), ref.cpu().numpy()) <= 1e-12
    assert _allocs(H) == a0


def test_noalloc_refuses_levels_above_the_staging_size(amg):
    import torch

    N = 364  # 363^2 = 131,769 unknowns > 131,072 staging entries
    p = q1_2d(N, rotated_sqrtK(0.3, 1e-2), agg=block_aggregates_2d(N, 4))
    H = amg.Hierarchy.from_problem(p, overlap=1, c_min=(4,), n_coarse=2000, precision=amg.MIXED32)
    x = torch.ones(p.n, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    st = H._lib.amgdd_apply_noalloc(H._h, amg.OP_RAS, 0, x.data_ptr(), y.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
    assert st == -1
    assert b"staging" in H._lib.amgdd_last_error()
    assert float(y.abs().max()) == 0.0
    # FP64 needs no staging: the same level works
    H.set_precision(amg.FP64)
    st = H._lib.amgdd_apply_noalloc(H._h, amg.OP_RAS, 0, x.data_ptr(), y.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
    assert st == 0
    assert math.isfinite(float(y.abs().max()))
