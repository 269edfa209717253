"""Synthetic rough-coefficient Poisson problems on the unit cube (d = 3).

The same recipe as the two-dimensional family, one dimension up:

* Mesh: ``n`` x ``n`` x ``n`` cubic cells of side h = 1/n (n a power of
  two), interior nodes (ix, iy, iz) with 1 <= ix, iy, iz <= n-1, numbered
  ``dof = ((iz-1)*(n-1) + (iy-1))*(n-1) + (ix-1)`` (x fastest).
* Coefficient: piecewise constant per cell, log a = sum_{s=1..S} xi_s with
  xi_s constant on the dyadic cubes of side 2^-s and
  xi_s ~ U[-1/2, 1/2] * ln(C) / S.  Draw order: ``default_rng(seed)``; for
  s = 1..S draw 8^s uniforms laid out row-major over (sz, sy, sx).
* Right-hand side: g_i ~ N(0, 1) iid per interior node, drawn after the
  coefficient from the same generator, in dof order.
* Fine operator: Q1 (trilinear) elements.  On a cube of side h the element
  stiffness is a_c * h * K_REF3, corners indexed by
  c = b_x + 2 b_y + 4 b_z for the corner (cx + b_x, cy + b_y, cz + b_z)
  (the child-slot order of the hierarchy).  Boundary rows and columns are
  dropped (homogeneous Dirichlet): a 27-point stencil matrix.
* Hierarchy: the level-q cell of node (ix, iy, iz) is (ix, iy, iz) in a
  2^q x 2^q x 2^q lattice (q = log2 n); its level-k cell is the coordinates
  shifted right by q - k bits.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .rough import Problem


def _k_ref3() -> np.ndarray:
    """Trilinear stiffness on the unit cube.  The 1-D linear element has
    stiffness [[1, -1], [-1, 1]] and mass [[1/3, 1/6], [1/6, 1/3]]; the
    trilinear shape functions are products, so entry (a, b) is
    sum over axes of (1-D stiffness on that axis) x (1-D masses on the other
    two).  By the number of axes on which corners a and b differ: 0 -> 1/3,
    1 -> 0, 2 -> -1/12, 3 -> -1/12."""
    K = np.zeros((8, 8))
    for a in range(8):
        for b in range(8):
            K[a, b] = {0: 1.0 / 3.0, 1: 0.0, 2: -1.0 / 12.0, 3: -1.0 / 12.0}[bin(a ^ b).count("1")]
    return K


# Trilinear element stiffness on the unit cube, corners c = bx + 2 by + 4 bz.
K_REF3 = _k_ref3()


def rough_log_coefficient3(n: int, scales: int, contrast: float,
                           rng: np.random.Generator) -> np.ndarray:
    """log a on an n^3 cell grid ([cz, cy, cx]), sum of `scales` dyadic
    piecewise-constant layers with amplitude ln(contrast)/scales each."""
    q = int(round(np.log2(n)))
    assert 1 << q == n, "n must be a power of two"
    assert scales <= q
    amp = np.log(contrast) / scales
    log_a = np.zeros((n, n, n))
    cz, cy, cx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    for s in range(1, scales + 1):
        u = rng.random(8 ** s).reshape(1 << s, 1 << s, 1 << s)  # [sz, sy, sx]
        xi = (u - 0.5) * amp
        log_a += xi[cz >> (q - s), cy >> (q - s), cx >> (q - s)]
    return log_a


def interior_cells3(n: int) -> np.ndarray:
    """Level-q lattice cells (x, y, z) of the interior nodes, dof order."""
    iz, iy, ix = np.meshgrid(np.arange(1, n), np.arange(1, n), np.arange(1, n), indexing="ij")
    return np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.int32)


def assemble_q1_3d(a: np.ndarray) -> sp.csr_matrix:
    """Q1 stiffness matrix for a cellwise coefficient a[cz, cy, cx] on an
    n^3 grid of the unit cube, interior nodes only, dof order of
    interior_cells3 (element matrix a_c * h * K_REF3, h = 1/n)."""
    n = a.shape[0]
    m = n - 1
    h = 1.0 / n
    cz, cy, cx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    cz, cy, cx = cz.ravel(), cy.ravel(), cx.ravel()
    av = a.ravel() * h
    corners = [(cx + (c & 1), cy + ((c >> 1) & 1), cz + ((c >> 2) & 1)) for c in range(8)]
    rows, cols, vals = [], [], []
    for p in range(8):
        xp, yp, zp = corners[p]
        inp = (xp >= 1) & (xp <= m) & (yp >= 1) & (yp <= m) & (zp >= 1) & (zp <= m)
        for r in range(8):
            xr, yr, zr = corners[r]
            inr = (xr >= 1) & (xr <= m) & (yr >= 1) & (yr <= m) & (zr >= 1) & (zr <= m)
            keep = inp & inr
            rows.append(((zp[keep] - 1) * m + (yp[keep] - 1)) * m + (xp[keep] - 1))
            cols.append(((zr[keep] - 1) * m + (yr[keep] - 1)) * m + (xr[keep] - 1))
            vals.append(av[keep] * K_REF3[p, r])
    A = sp.coo_matrix((np.concatenate(vals),
                       (np.concatenate(rows), np.concatenate(cols))),
                      shape=(m ** 3, m ** 3)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


def make_problem3(n: int, contrast: float, seed: int,
                  scales: int | None = None) -> Problem:
    """Rough-coefficient problem on the unit cube: coefficient, then g, from
    one generator (``Problem.log_a`` is [cz, cy, cx], ``cells`` n x 3)."""
    q = int(round(np.log2(n)))
    scales = q if scales is None else scales
    rng = np.random.default_rng(seed)
    log_a = rough_log_coefficient3(n, scales, contrast, rng)
    g = rng.standard_normal((n - 1) ** 3)
    A = assemble_q1_3d(np.exp(log_a))
    return Problem(n=n, q=q, log_a=log_a, A=A, g=g, cells=interior_cells3(n),
                   contrast=float(contrast))
