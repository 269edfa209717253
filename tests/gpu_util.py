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
