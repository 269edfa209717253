"""Oracle: level-q initialisation by the mass matrix (test infrastructure).

Algorithm 1, lines 1-5 (Sec. 5.2): the level-q gamblets are
psi^(q)_i = sum_j (M^-1)_{ij} phi_j, the elements of the span of the nodal
basis with integral against phi_j equal to delta_ij, so
    A^(q) = M^-1 A M^-1,    g^(q)_i = g_i  (g = sum_i g_i phi_i).
Algorithm 2, lines 2a-5 with Definition deflocinvm (Sec. 5.3): each column
i of M^-1 is replaced by the solution of the mass system restricted to the
nodes of i^{rho_q} with right-hand side e_i (zero elsewhere),
    M[i^rho_q, i^rho_q] y = e_i,   (M^-1,loc)_{j,i} = y_j,
and A^(q),loc = (M^-1,loc)^T A M^-1,loc.  The method then runs on A^(q)
unchanged; the solution u = sum_i U_i psi^(q)_i has nodal coefficients
u_phi = M^-1,loc U.  With the exact inverse, A u_phi = M g: the finite
element system with the load of g interpolated in the nodal space.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .hierarchy import Hierarchy
from .local import gamblet_local_setup, gamblet_local_solve


def localized_mass_inverse(M, cells, q, rho_q, rule: str = "euclid"):
    """M^-1,loc of Definition deflocinvm as a sparse n x n matrix (column i
    supported on i^{rho_q}).  rho_q = inf gives the exact inverse."""
    M = sp.csr_matrix(M, dtype=np.float64)
    n = M.shape[0]
    if not np.isfinite(rho_q):
        return sp.csr_matrix(np.linalg.inv(M.toarray()))
    H = Hierarchy(cells, q)
    nbrs = H.neighbours(q, rho_q, rule)
    rows, cols, vals = [], [], []
    for i in range(n):
        idx = nbrs[i]
        e = (idx == i).astype(np.float64)
        y = sla.cho_solve(sla.cho_factor(M[idx][:, idx].toarray(), lower=True), e)
        rows.append(idx)
        cols.append(np.full(len(idx), i))
        vals.append(y)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


def mass_initialised_operator(A, M, cells, q, rho_q, rule: str = "euclid"):
    """(A^(q),loc, M^-1,loc): Algorithm 2 lines 2a-5 (Algorithm 1 lines
    1-5 for rho_q = inf).  A^(q) is symmetrised as (X + X^T) / 2."""
    Minv = localized_mass_inverse(M, cells, q, rho_q, rule)
    Aq = sp.csr_matrix(Minv.T @ sp.csr_matrix(A) @ Minv)
    return sp.csr_matrix(0.5 * (Aq + Aq.T)), Minv


def gamblet_mass_setup(A, M, cells, q, rho, rho_q, rule: str = "euclid"):
    """Localized setup on the mass-initialised level-q operator."""
    Aq, Minv = mass_initialised_operator(A, M, cells, q, rho_q, rule)
    setup = gamblet_local_setup(Aq, cells, q, rho, rule)
    setup["Minv"] = Minv
    return setup


def gamblet_mass_solve(setup, g):
    """One-pass solve with g^(q) = g (Algorithm 1 line 4); returns the
    nodal coefficients u_phi = M^-1,loc U and U."""
    U = gamblet_local_solve(setup, g)["u"]
    return setup["Minv"] @ U, U
