"""Oracle: compression of u in the normalised gamblet basis (test
infrastructure).

Sec. 5.1 (Example 1, after the figure of the coefficients): u has a sparse
representation in the basis formed by psi^(1)_i / ||psi^(1)_i||_a and
chi^(k)_j / ||chi^(k)_j||_a, and can be compressed by setting the smallest
coefficients to zero.  With u = sum_i U_i psi^(1)_i + sum_k sum_j w^(k)_j
chi^(k)_j (Theorem thddwedmgugyug), the normalised coefficients are
    c^(1)_i = U_i ||psi^(1)_i||_a = U_i sqrt(A^(1)_ii),
    c^(k)_j = w^(k)_j ||chi^(k)_j||_a = w^(k)_j sqrt(B^(k)_jj)
(chi^(k)_j = sum_i W_ji psi^(k)_i, so ||chi^(k)_j||_a^2 = (W A^(k) W^T)_jj).
Compression keeps the coefficients with |c| >= eps * max |c| and rebuilds
u from them with the level recursion of the one-pass solve.
"""
from __future__ import annotations

import numpy as np

from .local import gamblet_local_solve


def normalised_coefficients(setup, g):
    """({k: c^(k)}, one-pass solve result); k = 1 holds c^(1)."""
    res = gamblet_local_solve(setup, g)
    c = {1: res["U1"] * np.sqrt(setup["A"][1].diagonal())}
    for k in range(2, setup["hier"].q + 1):
        c[k] = res["w"][k] * np.sqrt(setup["B"][k].diagonal())
    return c, res


def compress(setup, g, eps):
    """(u_c, kept, total): u rebuilt from the coefficients with
    |c| >= eps * max |c|."""
    q = setup["hier"].q
    c, res = normalised_coefficients(setup, g)
    cmax = max(np.abs(v).max() for v in c.values() if v.size)
    keep = {k: np.abs(v) >= eps * cmax for k, v in c.items()}
    U = np.where(keep[1], res["U1"], 0.0)
    v = U
    for k in range(2, q + 1):
        w = np.where(keep[k], res["w"][k], 0.0)
        v = setup["R"][k].T @ v + setup["W"][k].T @ w
    kept = int(sum(m.sum() for m in keep.values()))
    total = int(sum(m.size for m in keep.values()))
    return v, kept, total
