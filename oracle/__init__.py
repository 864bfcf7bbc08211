"""Plain, slow FP64 CPU oracle of the LS-AMG-DD method -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import, call or execute anything
in this package.  The CUDA library never does: the two share no code, no
helpers and no constants; the only common module is ``inputs`` (seeded problem
generators holding none of the method's arithmetic).

What it computes (paper sections / equations):

  structure.py  aggregates, cleanup of unaggregated nodes (Section 3.3),
                overlapping subdomains Omega_i = omega_i u Gamma_i and the
                Boolean partition of unity (Section 2.2, Eq. PoU / pou2),
                row multiplicity M and the rows nz_i (Section 3.1, Lemma),
                coarse-level aggregation of the block graph (reading of
                Algorithm 1's aggregation step on coarse levels).
  construct.py  local principal blocks A_i (Section 2.2), the SPSD splitting
                A~_i (Lemma, Eq. local_splitting), the Schur-complement
                generalized eigenproblem (Eq. gevp-S) and the eigenvector
                selection (Section 3.4), the block-diagonal interpolation
                (Eq. mg-p) and the least-squares propagation G_{l+1} = G_l P_l,
                A_{l+1} = G_{l+1}^T G_{l+1} (Section 3.1, multilevel method;
                Algorithm 1).
  cycle.py      RAS (Eq. ras) and RAS-T (Eq. ras-t) smoothers, the V-cycle
                (one RAS pre-, one RAS-T post-smoothing, exact coarsest
                solve), preconditioned CG, and the convergence metrics of
                Section 4 (average convergence factor, operator complexity).

Representation.  G_l is held as its rows grouped by identical structural
support; each group keeps the sum of its rows' outer products
H_g = sum_{l in g} g_l^T g_l.  Every formula of the method consumes G only
through such sums (A = sum_l g_l^T g_l, A~_i = sum_{l in nz_i} g_l^T g_l / M(l)),
and rows with the same support share M and nz-membership, so grouping is the
associativity of those sums and nothing more.  The tests compare it with a
literal row-by-row construction on small grids.

Pins: every function is pinned by ``tests/test_oracle_*.py`` against closed
forms, invariants stated in the paper, brute-force constructions and library
routines (see the test docstrings).  The paper prints no worked example, so
no function is pinned to printed numbers; the paper's convergence factors
are for a different discretisation and pin nothing.
"""
from .structure import (  # noqa: F401
    row_groups_from_csr,
    structural_adjacency,
    cleanup_aggregates,
    overlapping_subdomains,
    multiplicity_and_nz,
    vanek_aggregation,
    standard_aggregation,
    subdomain_colouring,
    kappa_threshold,
)
from .construct import Hierarchy, Level, setup, local_splitting, schur_complement, local_gep  # noqa: F401
from .cycle import ras, rast, vcycle, pcg, apply_A, metrics, additive_schwarz, two_level_additive  # noqa: F401
