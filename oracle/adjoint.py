"""Oracle: gradient of J(theta) = 1/2 |u(theta) - u_obs|^2 with respect to
the cell log-coefficients theta_c = log a_c, for the discrete problem of
Sec. 5.1 (Eq. eqhuiuhiuhuiu, Q1 elements, a piecewise constant per cell).

The paper has no adjoint; this is the textbook discrete adjoint of
A(theta) u = g:  A lambda = u - u_obs (A is symmetric) and
dJ/dtheta_c = -lambda^T (dA/dtheta_c) u = -a_c sum_{p,r} lambda_p K_ref[p,r] u_r
over the interior corners p, r of cell c.  Pinned by central finite
differences (tests/test_oracle_adjoint.py).
"""
from __future__ import annotations

import numpy as np

from workloads import cell_corner_dofs

from . import direct


def contract(n, a, lam, u, K_ref):
    """-a_c sum_{p,r} lam_p K_ref[p,r] u_r per cell (boundary corners skip)."""
    cd = cell_corner_dofs(n)
    av = np.asarray(a).ravel()
    lam_c = np.where(cd >= 0, np.asarray(lam)[np.maximum(cd, 0)], 0.0)
    u_c = np.where(cd >= 0, np.asarray(u)[np.maximum(cd, 0)], 0.0)
    return -av * np.einsum("cp,pr,cr->c", lam_c, K_ref, u_c)


def gradient(A, g, u_obs, n, a, K_ref):
    """Returns (J, dJ/dlog a (n*n, row-major cells), u)."""
    u, lu = direct.solve(A, g)
    r = u - u_obs
    lam, _ = direct.solve(A, r, lu=lu)
    J = 0.5 * float(r @ r)
    return J, contract(n, a, lam, u, K_ref), u
