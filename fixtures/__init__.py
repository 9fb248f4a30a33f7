"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This package generates problem instances only: finite-element meshes, the assembled
sparse SPD stiffness matrix ``A`` (CSR, FP64), integer lattice coordinates of the
unknowns, and right-hand sides.  It holds none of the solver's arithmetic (no
ordering, no factorization, no Krylov method); both the oracle and the CUDA path
consume the identical arrays it returns.
"""
from .meshes import (  # noqa: F401
    Problem,
    q1_square,
    hex_cube,
    hex_elasticity,
    p1_jittered,
    rhs_uniform,
    lognormal_coefficients,
    workload,
    WORKLOADS,
    p1_batch_sizes,
    p1_batch,
    block_diagonal,
)
