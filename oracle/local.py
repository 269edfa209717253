"""Oracle: localized gamblet setup and one-pass solve (Algorithm 2, Sec. 5.3).

Initialisation psi^(q),loc = phi (Sec. 5.2 alternative; Sec. 5.3 notes that
g^(q),loc = g loses no accuracy), so A^(q),loc = A and g^(q) = g.  For
k = q..2 (sparse float64):

  B      = W A^(k),loc W^T                                 (Alg. 2, line 7)
  for each i in I^(k-1) (Definition defb):
      i^rho  = level-(k-1) nodes within distance H_{k-1} rho of tau_i
      i^chi  = rows j of W^(k) whose parent j^(k-1) lies in i^rho
      solve  B[i^chi, i^chi] y = b,  b_j = -(W A^(k),loc pibar^(k,k-1))_{j,i}
      D^loc[i^chi, i] = y, zero elsewhere                  (Alg. 2, line 11)
  R^(k-1,k) = pibar + D^loc^T W                            (Alg. 2, line 12)
  A^(k-1),loc = R A^(k),loc R^T                            (Alg. 2, line 13)
  g^(k-1) = R g^(k)                                        (Alg. 2, line 15)

The one-pass solve takes w^(k) = B^-1 W g^(k) and U^(1) = A^(1)^-1 g^(1)
exactly (sparse direct, Alg. 2 lines 8 and 16) and sums the components
prolongated with the localized R (lines 10, 17, 18).  With rho large enough
that every i^rho is all of I^(k-1) this reduces to Algorithm 1
(tests/test_oracle_local.py pins that, and the decay of the localization
error with rho, Sec. 4.10 Theorem thmerrorpropagation / Sec. 5.4
Theorem tmdiscrete).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .hierarchy import Hierarchy


def gamblet_local_setup(A, cells, q, rho, rule: str = "euclid",
                        construction: str = "const2"):
    """Localized fine-to-coarse setup.  Returns dict with A[k] (sparse
    A^(k),loc), B[k], W[k], R[k] = R^(k-1,k) (sparse) and the hierarchy."""
    H = Hierarchy(cells, q)
    out = {"A": {}, "B": {}, "W": {}, "R": {}, "hier": H,
           "rho": rho, "rule": rule}
    Ak = sp.csr_matrix(A, dtype=np.float64)
    out["A"][q] = Ak
    for k in range(q, 1, -1):
        W = H.W(k, construction)
        pibar = H.pibar(k)
        B = sp.csr_matrix(W @ Ak @ W.T)
        rhs = sp.csc_matrix(-(W @ Ak @ pibar.T))        # J^(k) x I^(k-1)
        jpar = H.j_parent(k)
        nbrs = H.neighbours(k - 1, rho, rule)
        nkm1 = H.n(k - 1)
        in_patch = np.zeros(nkm1, dtype=bool)
        Drows, Dcols, Dvals = [], [], []
        for i in range(nkm1):
            in_patch[:] = False
            in_patch[nbrs[i]] = True
            chi = np.nonzero(in_patch[jpar])[0]
            if len(chi) == 0:
                continue
            Bp = B[chi][:, chi].toarray()
            b = rhs[:, i].toarray().ravel()[chi]
            y = sla.cho_solve(sla.cho_factor(Bp, lower=True), b)
            Drows.append(chi)
            Dcols.append(np.full(len(chi), i))
            Dvals.append(y)
        D = sp.csr_matrix((np.concatenate(Dvals) if Dvals else [],
                           (np.concatenate(Drows) if Drows else [],
                            np.concatenate(Dcols) if Dcols else [])),
                          shape=(W.shape[0], nkm1))
        R = sp.csr_matrix(pibar + D.T @ W)
        Akm1 = sp.csr_matrix(R @ Ak @ R.T)
        Akm1 = sp.csr_matrix(0.5 * (Akm1 + Akm1.T))
        out["B"][k] = B
        out["W"][k] = W
        out["R"][k] = R
        out["A"][k - 1] = Akm1
        Ak = Akm1
    return out


def gamblet_local_solve(setup, g, return_components: bool = False):
    """One-pass localized solve with exact level solves."""
    q = setup["hier"].q
    R, W, B, A = setup["R"], setup["W"], setup["B"], setup["A"]
    gk = {q: np.asarray(g, dtype=np.float64)}
    for k in range(q, 1, -1):
        gk[k - 1] = R[k] @ gk[k]
    w = {}
    for k in range(2, q + 1):
        w[k] = spla.spsolve(sp.csc_matrix(B[k]), W[k] @ gk[k]) \
            if B[k].shape[0] > 0 else np.zeros(0)
    U1 = np.linalg.solve(A[1].toarray(), gk[1])
    v = U1
    for k in range(2, q + 1):
        v = R[k].T @ v + W[k].T @ w[k]
    res = {"u": v, "w": w, "U1": U1, "g": gk}
    if return_components:
        nq = setup["hier"].n(q)
        comps = np.zeros((q, nq))
        for lev in range(1, q + 1):
            c = U1 if lev == 1 else W[lev].T @ w[lev]
            for k in range(lev + 1, q + 1):
                c = R[k].T @ c
            comps[lev - 1] = c
        res["comps"] = comps
    return res
