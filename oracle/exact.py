"""Oracle: Algorithm 1, exact gamblet transform and solve (Sec. 5.2).

Initialisation psi^(q)_i = phi_i (the alternative stated in Sec. 5.2 after
Algorithm 1): A^(q) is the fine stiffness matrix and g^(q) = g.  Then for
k = q..2 (dense float64):

  B^(k)      = W A^(k) W^T                       Eq. (eqjgfytfjhyyyg)
  w^(k)      = B^(k)^-1 W g^(k)                  Eq. (eqsdjoejddi1)
  D^(k,k-1)  = -B^(k)^-1 W A^(k) pibar^(k,k-1)   Eq. (eqdkdjhdkhse)
  R^(k-1,k)  = pibar^(k-1,k) + D^(k-1,k) W       Eq. (eqhuhiddeuv)
  A^(k-1)    = R A^(k) R^T                       Eq. (eqhuhiuv)
  g^(k-1)    = R g^(k)                           Eq. (eqyguugy6t)

and U^(1) = A^(1)^-1 g^(1) (Eq. eqsdjoejddi2).  The level components in
fine coordinates are u^(1) = P_1 U^(1) and u^(k) - u^(k-1) = P_k W^T w^(k)
(Theorem thddwedmgugyug), with P_k = R^(q,q-1) ... R^(k+1,k) because
psi^(k-1) = R psi^(k) (Eq. eq:ftfytftfx); u is their sum (Algorithm 1,
final line; Theorem thmgugyug2).

Pins (tests/test_oracle_pins.py): sum of components = direct solve,
A-orthogonality of components, pi R^T = I, R = A^-1 pi^T (pi A^-1 pi^T)^-1
(Theorem thmhggfees5 with Theorem thm:Gaussian), A^(k) = (Pi_k A^-1
Pi_k^T)^-1, W-independence of A^(k), R and u, brute-force projections.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .hierarchy import Hierarchy


def _dense(M):
    return M.toarray() if sp.issparse(M) else np.asarray(M, dtype=np.float64)


def gamblet_exact(A, g, cells, q, construction: str = "const2"):
    """Run Algorithm 1.  Returns a dict with, per level k:
    A[k] (n_k x n_k), g[k], B[k], W[k], w[k] (k >= 2), R[k] = R^(k-1,k)
    (k >= 2), U1, comps (q x n_q, row k-1 holds u^(k) - u^(k-1), row 0 holds
    u^(1)) and u (their sum)."""
    H = Hierarchy(cells, q)
    out = {"A": {}, "g": {}, "B": {}, "W": {}, "w": {}, "R": {}, "hier": H}
    Ak = _dense(A)
    gk = np.asarray(g, dtype=np.float64).copy()
    out["A"][q] = Ak
    out["g"][q] = gk
    for k in range(q, 1, -1):
        W = H.W(k, construction).toarray()
        pibar = H.pibar(k).toarray()
        B = W @ Ak @ W.T
        cf = sla.cho_factor(B, lower=True)
        w = sla.cho_solve(cf, W @ gk)
        D = -sla.cho_solve(cf, W @ Ak @ pibar.T)          # J^(k) x I^(k-1)
        R = pibar + D.T @ W                               # I^(k-1) x I^(k)
        Akm1 = R @ Ak @ R.T
        Akm1 = 0.5 * (Akm1 + Akm1.T)
        gkm1 = R @ gk
        out["B"][k] = B
        out["W"][k] = W
        out["w"][k] = w
        out["R"][k] = R
        out["A"][k - 1] = Akm1
        out["g"][k - 1] = gkm1
        Ak, gk = Akm1, gkm1
    U1 = sla.cho_solve(sla.cho_factor(Ak, lower=True), gk)
    out["U1"] = U1
    # prolongation matrices P_k (n_q x n_k)
    nq = H.n(q)
    P = {q: np.eye(nq)}
    for k in range(q, 1, -1):
        P[k - 1] = P[k] @ out["R"][k].T
    comps = np.zeros((q, nq))
    comps[0] = P[1] @ U1
    for k in range(2, q + 1):
        comps[k - 1] = P[k] @ (out["W"][k].T @ out["w"][k])
    out["P"] = P
    out["comps"] = comps
    out["u"] = comps.sum(axis=0)
    return out
