"""Synthetic rough-coefficient Poisson problems on the unit square.

Recipe (stated once so both sides generate identical inputs):

* Mesh: ``n`` x ``n`` square cells of side h = 1/n (n a power of two),
  interior nodes (ix, iy) with 1 <= ix, iy <= n-1, numbered row-major
  ``dof = (iy-1)*(n-1) + (ix-1)``.
* Coefficient: piecewise constant per cell, log a = sum_{s=1..S} xi_s, where
  xi_s is constant on the dyadic squares of side 2^-s and
  xi_s ~ U[-1/2, 1/2] * ln(C) / S, so a has contrast at most C.
  Draw order: ``rng = numpy.random.default_rng(seed)``; for s = 1..S draw
  4^s uniforms laid out row-major over (sy, sx).
* Right-hand side: g_i ~ N(0, 1) iid per interior node, drawn from the same
  generator after the coefficient, row-major over (iy, ix).
* Fine operator: Q1 (bilinear) elements, element matrix
  a_c * K_REF with corners ordered counter-clockwise from (cx, cy); in 2-D
  this matrix does not depend on h.  Boundary rows/columns are dropped
  (homogeneous Dirichlet), giving the 9-point stencil matrix A.
* Hierarchy: the level-q cell of node (ix, iy) is (ix, iy) in a 2^q x 2^q
  lattice (q = log2 n); its level-k cell is (ix >> (q-k), iy >> (q-k)).
  Level k < q lattices are full; at level q the cells with ix = 0 or
  iy = 0 hold no node.
* Many-instance workload: problem p draws, from default_rng(seed_p), its
  side from BATCH_SIDES, then log10 C ~ U[2, 6], then coefficient and g.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

# Bilinear element stiffness on a square, corners (0,0),(1,0),(1,1),(0,1).
K_REF = np.array(
    [[4.0, -1.0, -2.0, -1.0],
     [-1.0, 4.0, -1.0, -2.0],
     [-2.0, -1.0, 4.0, -1.0],
     [-1.0, -2.0, -1.0, 4.0]]) / 6.0


@dataclasses.dataclass
class Problem:
    n: int                 # cells per side
    q: int                 # number of levels
    log_a: np.ndarray      # (n, n) log coefficient, indexed [cy, cx]
    A: sp.csr_matrix       # (n-1)^2 x (n-1)^2 fine stiffness (float64)
    g: np.ndarray          # (n-1)^2 right-hand side
    cells: np.ndarray      # (n-1)^2 x 2 int32 level-q lattice cells (x, y)
    contrast: float = 0.0  # C of the coefficient draw

    @property
    def ndof(self) -> int:
        return self.A.shape[0]


def rough_log_coefficient(n: int, scales: int, contrast: float,
                          rng: np.random.Generator) -> np.ndarray:
    """log a on an n x n cell grid, sum of `scales` dyadic piecewise-constant
    layers with amplitude ln(contrast)/scales each."""
    q = int(round(np.log2(n)))
    assert 1 << q == n, "n must be a power of two"
    assert scales <= q
    amp = np.log(contrast) / scales
    log_a = np.zeros((n, n))
    cy, cx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    for s in range(1, scales + 1):
        u = rng.random(4 ** s).reshape(1 << s, 1 << s)  # [sy, sx]
        xi = (u - 0.5) * amp
        log_a += xi[cy >> (q - s), cx >> (q - s)]
    return log_a


def interior_cells(n: int) -> np.ndarray:
    """Level-q lattice cells (x, y) of the interior nodes, dof order."""
    iy, ix = np.meshgrid(np.arange(1, n), np.arange(1, n), indexing="ij")
    return np.stack([ix.ravel(), iy.ravel()], axis=1).astype(np.int32)


def assemble_q1(a: np.ndarray, element: np.ndarray = None) -> sp.csr_matrix:
    """Q1 stiffness matrix for a cellwise coefficient a[cy, cx] on an
    n x n grid, interior nodes only, row-major dof numbering (element
    matrix a_c * K_REF, or a_c * element when given)."""
    E = K_REF if element is None else element
    n = a.shape[0]
    m = n - 1
    cy, cx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    cy = cy.ravel()
    cx = cx.ravel()
    av = a.ravel()
    # corner nodes counter-clockwise
    corners = [(cx, cy), (cx + 1, cy), (cx + 1, cy + 1), (cx, cy + 1)]
    rows, cols, vals = [], [], []
    for p in range(4):
        xp, yp = corners[p]
        inp = (xp >= 1) & (xp <= m) & (yp >= 1) & (yp <= m)
        for r in range(4):
            xr, yr = corners[r]
            inr = (xr >= 1) & (xr <= m) & (yr >= 1) & (yr <= m)
            keep = inp & inr
            rows.append((yp[keep] - 1) * m + (xp[keep] - 1))
            cols.append((yr[keep] - 1) * m + (xr[keep] - 1))
            vals.append(av[keep] * E[p, r])
    A = sp.coo_matrix((np.concatenate(vals),
                       (np.concatenate(rows), np.concatenate(cols))),
                      shape=(m * m, m * m)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


# Bilinear element mass matrix on a square of side h, divided by h^2,
# corners counter-clockwise from (0, 0) as in K_REF.
M_REF = np.array(
    [[4.0, 2.0, 1.0, 2.0],
     [2.0, 4.0, 2.0, 1.0],
     [1.0, 2.0, 4.0, 2.0],
     [2.0, 1.0, 2.0, 4.0]]) / 36.0


def assemble_q1_mass(n: int) -> sp.csr_matrix:
    """Q1 mass matrix M_ij = integral of phi_i phi_j on an n x n grid of the
    unit square (h = 1/n), interior nodes only, row-major dof numbering."""
    return assemble_q1(np.ones((n, n)), element=M_REF / (n * n))


def make_problem(n: int, contrast: float, seed: int,
                 scales: int | None = None) -> Problem:
    """Rough-coefficient problem: coefficient then g from one generator."""
    q = int(round(np.log2(n)))
    scales = q if scales is None else scales
    rng = np.random.default_rng(seed)
    log_a = rough_log_coefficient(n, scales, contrast, rng)
    g = rng.standard_normal((n - 1) * (n - 1))
    A = assemble_q1(np.exp(log_a))
    return Problem(n=n, q=q, log_a=log_a, A=A, g=g, cells=interior_cells(n),
                   contrast=float(contrast))


# Grid sides of the many-instance workload and the range of log10(contrast).
BATCH_SIDES = (128, 256, 512)
BATCH_LOG10_CONTRAST = (2.0, 6.0)


def make_batch_problem(seed: int, sides=BATCH_SIDES,
                       log10_contrast=BATCH_LOG10_CONTRAST) -> Problem:
    """One problem of the many-instance workload.  Draw order from
    ``default_rng(seed)``: the side index (uniform over ``sides``), then
    log10 C ~ U[log10_contrast], then the coefficient (S = q scales) and g
    exactly as in make_problem."""
    rng = np.random.default_rng(seed)
    n = int(sides[int(rng.integers(len(sides)))])
    contrast = float(10.0 ** rng.uniform(*log10_contrast))
    q = int(round(np.log2(n)))
    log_a = rough_log_coefficient(n, q, contrast, rng)
    g = rng.standard_normal((n - 1) * (n - 1))
    A = assemble_q1(np.exp(log_a))
    return Problem(n=n, q=q, log_a=log_a, A=A, g=g, cells=interior_cells(n),
                   contrast=contrast)


def make_batch(nprob: int = 48, first_seed: int = 1, sides=BATCH_SIDES,
               log10_contrast=BATCH_LOG10_CONTRAST) -> list:
    """Problems with seeds first_seed .. first_seed + nprob - 1."""
    return [make_batch_problem(first_seed + p, sides, log10_contrast) for p in range(nprob)]


def example1_coefficient(q: int = 6) -> np.ndarray:
    """Coefficient of the paper's Example 1 (Section 5.1) on the
    (2^q+1) x (2^q+1) cell grid, indexed [j, i] for the cell
    [i/(2^q+1), (i+1)/(2^q+1)) x [j/(2^q+1), (j+1)/(2^q+1))."""
    n = (1 << q) + 1
    j, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    x = i / n
    y = j / n
    a = np.ones((n, n))
    for k in range(1, 7):
        a *= (1 + 0.5 * np.cos(2 ** k * np.pi * (x + y))) * \
             (1 + 0.5 * np.sin(2 ** k * np.pi * (y - 3 * x)))
    return a


def example1_rhs(q: int = 6) -> np.ndarray:
    """Nodal values of g for Example 1 at interior nodes z = (i, j)/(2^q+1),
    row-major over (j, i)."""
    n = (1 << q) + 1
    j, i = np.meshgrid(np.arange(1, n), np.arange(1, n), indexing="ij")
    z1 = (i / n).ravel()
    z2 = (j / n).ravel()
    return np.cos(3 * z1 + z2) + np.sin(3 * z2) + np.sin(7 * z1 - 5 * z2)


def make_example1(q: int = 6) -> Problem:
    """The paper's Example 1 (Section 5.1): (2^q + 1) x (2^q + 1) cells, the
    product coefficient of example1_coefficient, g from example1_rhs; the
    2^q x 2^q interior nodes sit in the cells (ix - 1, iy - 1) of the level-q
    lattice.  The mass matrix of the same grid is assemble_q1_mass(2^q + 1)."""
    n = (1 << q) + 1
    a = example1_coefficient(q)
    A = assemble_q1(a)
    return Problem(n=n, q=q, log_a=np.log(a), A=A, g=example1_rhs(q),
                   cells=np.ascontiguousarray(interior_cells(n) - 1, dtype=np.int32),
                   contrast=float(a.max() / a.min()))


def cell_corner_dofs(n: int) -> np.ndarray:
    """(n*n) x 4 int32 fine unknown of each cell corner (counter-clockwise
    from (cx, cy), the K_REF order), -1 on the Dirichlet boundary; cells in
    row-major (cy, cx) order, matching ``log_a.ravel()``."""
    m = n - 1
    cy, cx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    cy = cy.ravel()
    cx = cx.ravel()
    out = np.full((n * n, 4), -1, dtype=np.int32)
    for p, (xp, yp) in enumerate([(cx, cy), (cx + 1, cy), (cx + 1, cy + 1), (cx, cy + 1)]):
        ok = (xp >= 1) & (xp <= m) & (yp >= 1) & (yp <= m)
        out[ok, p] = (yp[ok] - 1) * m + (xp[ok] - 1)
    return out
