"""Oracle: nested dyadic measurement hierarchy (Sections 4.1 and 4.6).

Index tree (Sec. 4.1, Definition defindextree) and nested partitions
(Construction defmulires) for H = 1/2 (Sec. 5.1, Example ex1 hierarchy):
the level-k subdomain of a fine node is its level-q lattice cell shifted
right by q - k bits.  pi^(k-1,k) is the 0/1 aggregation matrix of
Eq. (eq:eigdeiud3dd), pibar its row-normalised version (Sec. 4.7), and W^(k)
a basis of Ker(pi^(k-1,k)) with one block per parent (Sec. 4.6, Lemma lemwk),
built by Construction const1 (consecutive differences) or Construction
const2 (normalised rows 1..m-1 of U^(m) from Lemma const0).

The construction is the same in every dimension d (the paper's setting
is a domain of R^d; the cells are squares for d = 2 and cubes for d = 3, so
a parent has up to 2^d children).

Ordering conventions (the CUDA path uses the same ones so that
W-dependent quantities can be compared entry by entry):
* level q: the fine dof order given by the caller;
* level k < q: distinct cells sorted row-major by (y, x) in 2-D and by
  (z, y, x) in 3-D (x varies fastest);
* the children of a parent are ordered by the child slot
  sum_a (c_a & 1) 2^a: row-major by (y & 1, x & 1) in 2-D and by
  (z & 1, y & 1, x & 1) in 3-D;
* rows of W^(k) are ordered by parent, then by t = 1..m_s - 1.

Parity pins: tests/test_oracle_pins.py (pi pibar^T = I, W W^T = I for
const2, pi W^T = 0, closed forms of R and A^(k)).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp


def helmert_u(n: int) -> np.ndarray:
    """U^(n) of Sec. 4.6, Lemma const0 (rows orthogonal, last row all ones)."""
    if n == 1:
        return np.ones((1, 1))
    U = np.array([[1.0, -1.0], [1.0, 1.0]])
    for m in range(2, n):
        V = np.zeros((m + 1, m + 1))
        V[:m - 1, :m] = U[:m - 1, :]
        V[m - 1, :m] = 1.0
        V[m - 1, m] = -float(m)
        V[m, :] = 1.0
        U = V
    return U


def helmert_ubar(n: int) -> np.ndarray:
    U = helmert_u(n)
    return U / np.linalg.norm(U, axis=1, keepdims=True)


def cell_key(c: np.ndarray, k: int) -> np.ndarray:
    """Row-major key of level-k lattice cells c (n x d, x first): x varies
    fastest, then y, then z."""
    c = np.asarray(c, dtype=np.int64)
    key = np.zeros(len(c), dtype=np.int64)
    for a in range(c.shape[1] - 1, -1, -1):
        key = key * (1 << k) + c[:, a]
    return key


def key_cells(key: np.ndarray, k: int, d: int) -> np.ndarray:
    """Inverse of cell_key: n x d cells of the keys."""
    key = np.asarray(key, dtype=np.int64)
    return np.stack([(key >> (k * a)) & ((1 << k) - 1) for a in range(d)], axis=1)


@dataclasses.dataclass
class Level:
    cells: np.ndarray          # n_k x d lattice cells (x, y[, z]) at level k
    parent: np.ndarray | None  # n_k -> index in level k-1 (None for k = 1)


class Hierarchy:
    """Levels 1..q built from the fine nodes' level-q cells (n x d,
    d = 2 or 3)."""

    def __init__(self, cells_q: np.ndarray, q: int):
        cells_q = np.asarray(cells_q, dtype=np.int64)
        self.q = q
        self.d = cells_q.shape[1]
        self.levels: dict[int, Level] = {}
        self.levels[q] = Level(cells=cells_q, parent=None)
        for k in range(q - 1, 0, -1):
            child = self.levels[k + 1].cells
            ukey, inv = np.unique(cell_key(child >> 1, k), return_inverse=True)
            self.levels[k] = Level(cells=key_cells(ukey, k, self.d), parent=None)
            self.levels[k + 1].parent = inv.astype(np.int64)

    def n(self, k: int) -> int:
        return len(self.levels[k].cells)

    def children(self, k: int) -> list[np.ndarray]:
        """Children (level-k indices) of each level-(k-1) node, ordered by
        the child slot sum_a (c_a & 1) 2^a."""
        par = self.levels[k].parent
        cells = self.levels[k].cells
        slot = sum((cells[:, a] & 1) << a for a in range(self.d))
        order = np.lexsort((slot, par))
        counts = np.bincount(par, minlength=self.n(k - 1))
        splits = np.cumsum(counts)[:-1]
        return np.split(order, splits)

    def pi(self, k: int) -> sp.csr_matrix:
        """pi^(k-1,k): pi[i, j] = 1 iff j is a child of i (Eq. eq:eigdeiud3dd)."""
        par = self.levels[k].parent
        nk = self.n(k)
        return sp.csr_matrix((np.ones(nk), (par, np.arange(nk))),
                             shape=(self.n(k - 1), nk))

    def pibar(self, k: int) -> sp.csr_matrix:
        """pibar^(k-1,k) = pi / m_i (Section 4.7)."""
        P = self.pi(k)
        m = np.asarray(P.sum(axis=1)).ravel()
        return sp.diags(1.0 / m) @ P

    def W(self, k: int, construction: str = "const2") -> sp.csr_matrix:
        """W^(k) (J^(k) x I^(k)), block-local to each parent (Section 4.6)."""
        rows, cols, vals = [], [], []
        r = 0
        for ch in self.children(k):
            m = len(ch)
            if m < 2:
                continue
            if construction == "const2":
                blk = helmert_ubar(m)[:m - 1, :]
            elif construction == "const1":
                blk = np.zeros((m - 1, m))
                for t in range(m - 1):
                    blk[t, t] = 1.0
                    blk[t, t + 1] = -1.0
            else:
                raise ValueError(construction)
            for t in range(m - 1):
                for tp in range(m):
                    rows.append(r + t)
                    cols.append(ch[tp])
                    vals.append(blk[t, tp])
            r += m - 1
        return sp.csr_matrix((vals, (rows, cols)), shape=(r, self.n(k)))

    def j_parent(self, k: int) -> np.ndarray:
        """Parent (level k-1 index) of every row of W^(k)."""
        out = []
        for s, ch in enumerate(self.children(k)):
            out.extend([s] * max(len(ch) - 1, 0))
        return np.asarray(out, dtype=np.int64)

    def neighbours(self, k: int, rho: float, rule: str = "euclid") -> list[np.ndarray]:
        """i^rho at level k (Sec. 4.10, first paragraph): level-k nodes whose subdomain
        lies within distance H_k * rho of tau_i.  In lattice units the
        distance between closed squares (cubes) whose offsets are
        (d_1, .., d_d) is sqrt(sum_a max(|d_a| - 1, 0)^2).  rule="cheb" uses
        the box max_a |d_a| <= rho instead."""
        c = self.levels[k].cells
        out = []
        for i in range(len(c)):
            dist = np.abs(c - c[i])
            if rule == "euclid":
                e = np.maximum(dist - 1, 0)
                ok = (e * e).sum(axis=1) <= rho * rho
            elif rule == "cheb":
                ok = dist.max(axis=1) <= rho
            else:
                raise ValueError(rule)
            out.append(np.nonzero(ok)[0])
        return out
