"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package builds the *problem* handed to ``setup``/``solve`` (the sparse
least-squares factor G of a Q1 diffusion discretisation, the diagonal D1, the
level-0 aggregates and the right-hand sides).  It contains none of the
multilevel method's arithmetic: no splitting, no eigenproblem, no smoother,
no coarse space.  Both the CPU oracle and the CUDA library consume what it
produces; neither is imported here.
"""
from .q1 import (  # noqa: F401
    Q1Problem,
    q1_2d,
    block_aggregates_2d,
    seeded_rhs,
    rotated_sqrtK,
    circular_sqrtK,
    config_problem,
)
from .q1_3d import q1_3d, field_sqrtK, strength_graph, greedy_aggregates  # noqa: F401
from .fd import fd_2d, fd_block_aggregates  # noqa: F401
