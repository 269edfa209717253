"""Helpers shared by the GPU parity tests (not a test module)."""
import numpy as np
import scipy.sparse as sp


def csr_arrays(A):
    A = sp.csr_matrix(A)
    A.sort_indices()
    return (np.ascontiguousarray(A.indptr, dtype=np.int32),
            np.ascontiguousarray(A.indices, dtype=np.int32),
            np.ascontiguousarray(A.data, dtype=np.float64))


def coo_to_dense(r, c, v, shape):
    M = np.zeros(shape)
    np.add.at(M, (r, c), v)
    return M


def rel(a, b):
    a = a.toarray() if hasattr(a, "toarray") else np.asarray(a)
    b = b.toarray() if hasattr(b, "toarray") else np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def drop_nodes(p, keep):
    """Sub-problem on the kept fine unknowns (Dirichlet on the removed ones)."""
    idx = np.nonzero(keep)[0]
    A = sp.csr_matrix(p.A)[idx][:, idx]
    return sp.csr_matrix(A), p.g[idx].copy(), np.ascontiguousarray(p.cells[idx])


def demorton(m):
    """(x, y) of a Morton index: x from the even bits, y from the odd bits."""
    x = y = 0
    for b in range(16):
        x |= ((m >> (2 * b)) & 1) << b
        y |= ((m >> (2 * b + 1)) & 1) << b
    return x, y


def pack_problems(probs):
    """The placement gamblet_setup_batched documents: largest problems first
    (stable), each in the aligned subtree starting at the running Morton
    offset of a 2^Q lattice; unknowns numbered problem after problem.
    Returns (A, g, cells, Q, offsets) of the combined block-diagonal system."""
    order = sorted(range(len(probs)), key=lambda p: -probs[p].q)
    base, total = {}, 0
    for p in order:
        base[p] = total
        total += 4 ** probs[p].q
    Q = max(max(pr.q for pr in probs), 2)
    while 4 ** Q < total:
        Q += 1
    cells = []
    for p, pr in enumerate(probs):
        x0, y0 = demorton(base[p])
        cells.append(pr.cells + np.array([x0, y0], dtype=np.int32))
    offsets = np.concatenate([[0], np.cumsum([pr.ndof for pr in probs])]).astype(np.int64)
    A = sp.block_diag([pr.A for pr in probs], format="csr")
    g = np.concatenate([pr.g for pr in probs])
    return A, g, np.ascontiguousarray(np.concatenate(cells), dtype=np.int32), Q, offsets


def _dense(a):
    return a.toarray() if hasattr(a, "toarray") else np.asarray(a, dtype=np.float64)


def max_dev(a, b):
    """Element-wise deviation max_ij |a_ij - b_ij| / max_ij |b_ij|."""
    a, b = _dense(a), _dense(b)
    assert a.shape == b.shape, (a.shape, b.shape)
    return float(np.abs(a - b).max(initial=0.0) / max(np.abs(b).max(initial=0.0), 1e-300))


def row_dev(a, b):
    """Element-wise deviation with each row scaled by its own largest |b_ij|:
    max_i max_j |a_ij - b_ij| / max_j |b_ij|.  For R every row is one
    patch's gamblet, whose entries decay exponentially away from its cell
    (Sec. 4.10), so this guards the small tails that a whole-matrix scale
    would hide."""
    a, b = _dense(a), _dense(b)
    assert a.shape == b.shape, (a.shape, b.shape)
    scale = np.abs(b).max(axis=1, keepdims=True)
    scale[scale == 0] = 1.0
    return float((np.abs(a - b) / scale).max(initial=0.0))


def check_op(a, b, tol, what=None):
    """Level operator parity, element by element: |a - b| <= tol max|b|."""
    d = max_dev(a, b)
    assert d <= tol, (what, d, tol)


def check_R(a, b, tol, what=None):
    """Interpolation parity: element-wise within tol of each row's largest
    entry, and the same nonzero pattern (the patch support of Definition
    defb: a GPU entry outside the oracle's patch, or a missing one inside
    it, fails regardless of size)."""
    a, b = _dense(a), _dense(b)
    d = row_dev(a, b)
    assert d <= tol, (what, d, tol)
    sa, sb = a != 0, b != 0
    assert np.array_equal(sa, sb), (what, "support", int((sa & ~sb).sum()), int((sb & ~sa).sum()))
