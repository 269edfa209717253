"""Oracle cross-check by brute force, for tiny grids (no level recursion).

Uses only the definitions of Sec. 4.2 / 4.5, never Algorithm 1's recursion:
the level-k measurement matrix Pi_k (n_k x n_q) sums the fine nodal
coefficients over each level-k cell (nested aggregation of Sec. 5.1 with
phi^(q) = the nodal basis), Theta^(k) = Pi_k A^-1 Pi_k^T (Eq. eq:kldldje34),
psi^(k) = A^-1 Pi_k^T Theta^(k)^-1 (Eq. eq:doehddcasek), A^(k) = Theta^(k)^-1,
R^(k-1,k)_{ij} = (Pi_k psi^(k-1))_{ji} (Theorem eqhjgjhgjgjg), and
u^(k) = psi^(k) Pi_k u, the A-orthogonal projection of u onto V^(k)
(Theorem thmgugyug0).
"""
from __future__ import annotations

import numpy as np


def level_cells(cells, q, k):
    """Sorted distinct level-k cells and the map fine node -> level-k index
    (row-major (y, x) order in 2-D, (z, y, x) in 3-D, matching the oracle
    hierarchy)."""
    c = np.asarray(cells, dtype=np.int64) >> (q - k)
    key = np.zeros(len(c), dtype=np.int64)
    for a in range(c.shape[1] - 1, -1, -1):
        key = key * (1 << k) + c[:, a]
    ukey, inv = np.unique(key, return_inverse=True)
    return ukey, inv


def measurement(cells, q, k):
    """Pi_k: n_k x n_q 0/1 matrix."""
    ukey, inv = level_cells(cells, q, k)
    nq = len(inv)
    P = np.zeros((len(ukey), nq))
    P[inv, np.arange(nq)] = 1.0
    return P


def brute(A, g, cells, q):
    Ad = A.toarray() if hasattr(A, "toarray") else np.asarray(A)
    Ainv = np.linalg.inv(Ad)
    u = Ainv @ g
    out = {"u": u, "Ak": {}, "psi": {}, "uk": {}, "R": {}}
    for k in range(1, q + 1):
        Pk = measurement(cells, q, k)
        Theta = Pk @ Ainv @ Pk.T
        Ak = np.linalg.inv(Theta)
        psi = Ainv @ Pk.T @ Ak                     # n_q x n_k
        out["Ak"][k] = 0.5 * (Ak + Ak.T)
        out["psi"][k] = psi
        out["uk"][k] = psi @ (Pk @ u)
    for k in range(2, q + 1):
        Pk = measurement(cells, q, k)
        out["R"][k] = (Pk @ out["psi"][k - 1]).T   # n_{k-1} x n_k
    comps = [out["uk"][1]] + [out["uk"][k] - out["uk"][k - 1]
                              for k in range(2, q + 1)]
    out["comps"] = np.array(comps)
    return out
