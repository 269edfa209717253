"""Oracle: direct solution of the fine system A u = g (Sec. 5.1, the
discrete problem solved by Algorithms 1 and 2).

SuperLU factorisation (minimum-degree ordering on A + A^T, symmetric mode)
followed by classical iterative refinement whose residual g - A u is
accumulated in numpy.longdouble (80-bit extended on x86-64, binary128 on
aarch64), so the returned u is limited by the conditioning of A rather than
by the rounding of one float64 triangular solve.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as sla


def factor(A):
    A = sp.csc_matrix(A)
    return sla.splu(A, permc_spec="MMD_AT_PLUS_A",
                    options=dict(SymmetricMode=True), diag_pivot_thresh=0.0)


def residual_ext(A, u, g):
    """g - A u with products and sums in numpy.longdouble."""
    A = sp.csr_matrix(A)
    ld = np.longdouble
    prod = A.data.astype(ld) * np.asarray(u, dtype=ld)[A.indices]
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    Au = np.zeros(A.shape[0], dtype=ld)
    np.add.at(Au, rows, prod)
    return np.asarray(g, dtype=ld) - Au


def solve(A, g, refine_steps: int = 3, lu=None):
    """u = A^-1 g by SuperLU plus `refine_steps` extended-precision
    refinement steps.  Returns (u, lu)."""
    lu = factor(A) if lu is None else lu
    u = lu.solve(np.asarray(g, dtype=np.float64))
    for _ in range(refine_steps):
        r = residual_ext(A, u, g)
        du = lu.solve(np.asarray(r, dtype=np.float64))
        u = np.asarray(np.asarray(u, dtype=np.longdouble) + du, dtype=np.float64)
    return u, lu
