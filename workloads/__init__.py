"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package holds only input generation: the rough multiscale coefficient
field, the random right-hand side, the Q1 finite-element stiffness matrix of
-div(a grad u) = g with homogeneous Dirichlet conditions (the problem of
Section 5.1, Eq. for the discrete system), and the level-q lattice cells that
define the nested dyadic measurement hierarchy (Construction 4.2 with H = 1/2).
None of the gamblet method's arithmetic lives here.
"""
from .rough import (  # noqa: F401
    Problem,
    K_REF,
    assemble_q1,
    assemble_q1_mass,
    M_REF,
    cell_corner_dofs,
    example1_coefficient,
    example1_rhs,
    make_example1,
    make_problem,
    make_batch,
    make_batch_problem,
    BATCH_SIDES,
    rough_log_coefficient,
    interior_cells,
)
from .rough3d import (  # noqa: F401
    K_REF3,
    assemble_q1_3d,
    interior_cells3,
    make_problem3,
    rough_log_coefficient3,
)
