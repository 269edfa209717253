"""ctypes binding of libgamblet.so (include/gamblet.h), argument marshalling
only: every step of the method runs in the library's CUDA kernels.

Array arguments may be torch tensors (CPU or CUDA) or NumPy arrays; they must
be contiguous and of the dtype the C ABI names (int32 indices, float64
values).  Failures raise GambletError carrying the library's status code and
message.  Importing this module loads the library and raises if it has not
been built: there is no other implementation to fall back to.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgamblet.so")

OK = 0
ERR_INVALID_ARG = 1
ERR_NOT_SPD = 2
ERR_NOT_CONVERGED = 3
ERR_CUDA = 4
ERR_OUT_OF_MEMORY = 5
ERR_UNSUPPORTED = 6
FP64 = 0
MIXED = 1


class GambletError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class Csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("colind", ctypes.c_void_p),
                ("val", ctypes.c_void_p)]


class Opts(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_double), ("nbr_rule", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("level_tol", ctypes.c_double),
                ("level_max_iter", ctypes.c_int32), ("refine_tol", ctypes.c_double),
                ("refine_max_iter", ctypes.c_int32), ("patch_tol", ctypes.c_double),
                ("use_graph", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("galerkin_variant", ctypes.c_int32), ("patch_gather", ctypes.c_int32),
                ("stream", ctypes.c_void_p)]


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("q", ctypes.c_int32),
                ("outer_iters", ctypes.c_int32), ("level_iters", ctypes.c_int32 * 32),
                ("rel_residual", ctypes.c_double), ("setup_ms", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("patch_iters_max", ctypes.c_int32),
                ("patch_iters_mean", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {"status": self.status, "q": self.q, "outer_iters": self.outer_iters,
                "level_iters": list(self.level_iters)[: self.q + 1],
                "rel_residual": self.rel_residual, "setup_ms": self.setup_ms,
                "solve_ms": self.solve_ms, "patch_iters_max": self.patch_iters_max,
                "patch_iters_mean": self.patch_iters_mean}


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64),
                ("ms", ctypes.c_double), ("bytes", ctypes.c_double), ("flops", ctypes.c_double)]


# name -> (restype, argtypes)
SIGNATURES = {
    "gamblet_default_opts": (None, [ctypes.POINTER(Opts)]),
    "gamblet_setup": (ctypes.c_int, [ctypes.POINTER(Csr), ctypes.c_int32, ctypes.c_void_p,
                                     ctypes.POINTER(Opts), ctypes.POINTER(ctypes.c_void_p)]),
    "gamblet_setup_mass": (ctypes.c_int, [ctypes.POINTER(Csr), ctypes.POINTER(Csr), ctypes.c_int32,
                                          ctypes.c_void_p, ctypes.c_double, ctypes.POINTER(Opts),
                                          ctypes.POINTER(ctypes.c_void_p)]),
    "gamblet_setup_batched": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(Csr),
                                             ctypes.POINTER(ctypes.c_int32),
                                             ctypes.POINTER(ctypes.c_void_p),
                                             ctypes.POINTER(Opts), ctypes.POINTER(ctypes.c_void_p),
                                             ctypes.POINTER(ctypes.c_int32)]),
    "gamblet_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.POINTER(Info)]),
    "gamblet_level_condition": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                               ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                               ctypes.POINTER(ctypes.c_double)]),
    "gamblet_compress": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                        ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_int64)]),
    "gamblet_solve_many": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.POINTER(Info)]),
    "gamblet_solve_truncated": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.POINTER(Info)]),
    "gamblet_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(Info)]),
    "gamblet_grad_onepass": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(Info)]),
    "gamblet_assemble_cells": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p]),
    "gamblet_launch_shapes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32,
                                             ctypes.POINTER(ctypes.c_int32)]),
    "gamblet_level_size": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int32)]),
    "gamblet_get_operator": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "gamblet_device_bytes": (ctypes.c_int64, [ctypes.c_void_p]),
    "gamblet_kernel_stats": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(KernelStat),
                                              ctypes.c_int32]),
    "gamblet_reset_kernel_stats": (None, [ctypes.c_void_p]),
    "gamblet_kernel_launches": (ctypes.c_int64, []),
    "gamblet_plan_check": (ctypes.c_int, [ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                          ctypes.c_void_p]),
    "gamblet_objective_noalloc": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p,
                                                 ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_void_p]),
    "gamblet_destroy": (None, [ctypes.c_void_p]),
    # three-dimensional path (include/gamblet3d.h)
    "gamblet3d_setup": (ctypes.c_int, [ctypes.POINTER(Csr), ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.POINTER(Opts), ctypes.POINTER(ctypes.c_void_p)]),
    "gamblet3d_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.POINTER(Info)]),
    "gamblet3d_level_size": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32,
                                            ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ctypes.c_int32)]),
    "gamblet3d_get_operator": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "gamblet3d_level_geometry": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32,
                                                ctypes.POINTER(ctypes.c_int32)]),
    "gamblet3d_kernel_stats": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(KernelStat),
                                                ctypes.c_int32]),
    "gamblet3d_reset_kernel_stats": (None, [ctypes.c_void_p]),
    "gamblet3d_device_bytes": (ctypes.c_int64, [ctypes.c_void_p]),
    "gamblet3d_destroy": (None, [ctypes.c_void_p]),
    "gamblet_status_string": (ctypes.c_char_p, [ctypes.c_int32]),
    "gamblet_last_error": (ctypes.c_char_p, []),
}


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build it with `python -m paper_1503_03467_gb300.build` "
            "(nvcc, sm_103a); there is no fallback implementation")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = load()


def _ptr(x, dtype=None):
    if x is None:
        return None
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if not x.is_contiguous():
                raise ValueError("tensor must be contiguous")
            if dtype is not None and x.dtype != {np.int32: torch.int32,
                                                 np.float64: torch.float64}[dtype]:
                raise TypeError(f"expected {dtype}, got {x.dtype}")
            return ctypes.c_void_p(x.data_ptr())
    except ImportError:  # pragma: no cover
        pass
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        if dtype is not None and x.dtype != dtype:
            raise TypeError(f"expected {np.dtype(dtype)}, got {x.dtype}")
        return ctypes.c_void_p(x.ctypes.data)
    raise TypeError(f"unsupported array type {type(x)}")


def _check(st: int) -> int:
    if st not in (OK, ERR_NOT_CONVERGED):
        raise GambletError(st, _lib.gamblet_last_error().decode())
    return st


def gamblet_default_opts() -> Opts:
    o = Opts()
    _lib.gamblet_default_opts(ctypes.byref(o))
    return o


def gamblet_setup(rowptr, colind, val, q: int, cells, opts: Opts | None = None) -> int:
    n = int(rowptr.shape[0]) - 1
    csr = Csr(n, int(colind.shape[0]), _ptr(rowptr, np.int32), _ptr(colind, np.int32),
              _ptr(val, np.float64))
    h = ctypes.c_void_p()
    st = _lib.gamblet_setup(ctypes.byref(csr), int(q), _ptr(cells, np.int32),
                            ctypes.byref(opts) if opts is not None else None, ctypes.byref(h))
    _check(st)
    return h.value


def gamblet_setup_mass(A_csr, M_csr, q: int, cells, rho_q: float, opts: Opts | None = None) -> int:
    """A_csr, M_csr: (rowptr, colind, val) of the stiffness and mass matrices."""
    def csr(t):
        rowptr, colind, val = t
        return Csr(int(rowptr.shape[0]) - 1, int(colind.shape[0]), _ptr(rowptr, np.int32),
                   _ptr(colind, np.int32), _ptr(val, np.float64))
    a, m = csr(A_csr), csr(M_csr)
    h = ctypes.c_void_p()
    st = _lib.gamblet_setup_mass(ctypes.byref(a), ctypes.byref(m), int(q), _ptr(cells, np.int32),
                                 float(rho_q), ctypes.byref(opts) if opts is not None else None,
                                 ctypes.byref(h))
    _check(st)
    return h.value


def gamblet_setup_batched(problems, opts: Opts | None = None):
    """problems: sequence of (rowptr, colind, val, q, cells) as for
    gamblet_setup.  Returns (handle, offsets): problem p owns entries
    offsets[p]:offsets[p + 1] of the vectors passed to gamblet_solve."""
    problems = list(problems)
    nprob = len(problems)
    csrs = (Csr * nprob)()
    qs = (ctypes.c_int32 * nprob)()
    cells = (ctypes.c_void_p * nprob)()
    for p, (rowptr, colind, val, q, cl) in enumerate(problems):
        csrs[p] = Csr(int(rowptr.shape[0]) - 1, int(colind.shape[0]), _ptr(rowptr, np.int32),
                      _ptr(colind, np.int32), _ptr(val, np.float64))
        qs[p] = int(q)
        cells[p] = _ptr(cl, np.int32)
    offsets = (ctypes.c_int32 * (nprob + 1))()
    h = ctypes.c_void_p()
    st = _lib.gamblet_setup_batched(nprob, csrs, qs, cells,
                                    ctypes.byref(opts) if opts is not None else None,
                                    ctypes.byref(h), offsets)
    _check(st)
    return h.value, np.array(offsets[:], dtype=np.int64)


def gamblet_launch_shapes(h: int, k: int) -> dict:
    out = (ctypes.c_int32 * 4)()
    _check(_lib.gamblet_launch_shapes(ctypes.c_void_p(h), int(k), out))
    return {"patch_spp": out[0], "patch_gather": out[1], "galerkin_variant": out[2],
            "cg_spp": out[3]}


def gamblet_solve(h: int, g, u, components=None, info: Info | None = None) -> int:
    info = info if info is not None else Info()
    st = _lib.gamblet_solve(ctypes.c_void_p(h), _ptr(g, np.float64), _ptr(u, np.float64),
                            _ptr(components, np.float64), ctypes.byref(info))
    return _check(st)


def gamblet_level_condition(h: int, k: int, steps: int = 60, construction: int = 2):
    """(lmin, lmax) estimates of the extreme eigenvalues of B^(k) = W A W^T
    (Lanczos) for W of Construction const2 (2) or const1 (1)."""
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _check(_lib.gamblet_level_condition(ctypes.c_void_p(h), int(k), int(construction), int(steps),
                                        ctypes.byref(lo), ctypes.byref(hi)))
    return lo.value, hi.value


def gamblet_compress(h: int, g, eps: float, u):
    """u <- g's solution rebuilt from its normalised coefficients >= eps *
    max; returns (kept, total)."""
    kept, total = ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.gamblet_compress(ctypes.c_void_p(h), _ptr(g, np.float64), float(eps),
                                 _ptr(u, np.float64), ctypes.byref(kept), ctypes.byref(total)))
    return kept.value, total.value


def gamblet_solve_many(h: int, G, U, info: Info | None = None) -> int:
    """G, U: (nrhs, n) float64 arrays or tensors (row r = right-hand side r)."""
    info = info if info is not None else Info()
    nrhs = int(G.shape[0])
    st = _lib.gamblet_solve_many(ctypes.c_void_p(h), nrhs, _ptr(G, np.float64), _ptr(U, np.float64),
                                 ctypes.byref(info))
    return _check(st)


def gamblet_solve_truncated(h: int, k: int, g, u, info: Info | None = None) -> int:
    info = info if info is not None else Info()
    st = _lib.gamblet_solve_truncated(ctypes.c_void_p(h), int(k), _ptr(g, np.float64),
                                      _ptr(u, np.float64), ctypes.byref(info))
    return _check(st)


def gamblet_grad(h: int, cell_nodes, cell_a, K_ref, u, u_obs, dJ,
                 info: Info | None = None) -> float:
    info = info if info is not None else Info()
    J = ctypes.c_double()
    ncell = int(cell_a.shape[0])
    st = _lib.gamblet_grad(ctypes.c_void_p(h), ncell, _ptr(cell_nodes, np.int32),
                           _ptr(cell_a, np.float64), _ptr(K_ref, np.float64),
                           _ptr(u, np.float64), _ptr(u_obs, np.float64), _ptr(dJ, np.float64),
                           ctypes.byref(J), ctypes.byref(info))
    _check(st)
    return J.value


def gamblet_grad_onepass(h: int, cell_nodes, cell_a, K_ref, g, u_obs, dJ, u=None, dJ_dg=None,
                         info: Info | None = None) -> float:
    """Gradient of J = 1/2 |u_loc - u_obs|^2 through the one-pass localized
    transform (setup included); returns J, writes dJ (and u_loc, dJ/dg)."""
    info = info if info is not None else Info()
    J = ctypes.c_double()
    ncell = int(cell_a.shape[0])
    st = _lib.gamblet_grad_onepass(ctypes.c_void_p(h), ncell, _ptr(cell_nodes, np.int32),
                                   _ptr(cell_a, np.float64), _ptr(K_ref, np.float64),
                                   _ptr(g, np.float64), _ptr(u_obs, np.float64),
                                   _ptr(u, np.float64), _ptr(dJ, np.float64),
                                   _ptr(dJ_dg, np.float64), ctypes.byref(J), ctypes.byref(info))
    _check(st)
    return J.value


def gamblet_objective_noalloc(n: int, u, u_obs, J, stream=None) -> int:
    """J = 1/2 |u - u_obs|^2 into J (a 1-element float64 tensor or array);
    u and u_obs must be CUDA tensors of the current device.  Allocates no
    device memory.  The C side cannot see the lengths of the buffers, so
    they are checked here."""
    n = int(n)
    for name, a in (("u", u), ("u_obs", u_obs)):
        if a is None or n > int(a.numel() if hasattr(a, "numel") else np.asarray(a).size):
            raise ValueError(f"gamblet_objective_noalloc: {name} holds fewer than n = {n} values")
    if J is None or int(J.numel() if hasattr(J, "numel") else np.asarray(J).size) < 1:
        raise ValueError("gamblet_objective_noalloc: J must hold one value")
    return _check(_lib.gamblet_objective_noalloc(int(n), _ptr(u, np.float64),
                                                 _ptr(u_obs, np.float64), _ptr(J, np.float64),
                                                 stream))


def gamblet_assemble_cells(rowptr, colind, cell_nodes, log_a, K_ref, val, cell_a=None,
                           stream=None) -> int:
    """CSR values of sum_c exp(log_a_c) K_ref into `val` (CUDA tensors);
    optionally exp(log_a) into `cell_a`."""
    n = int(rowptr.shape[0]) - 1
    return _check(_lib.gamblet_assemble_cells(
        n, _ptr(rowptr, np.int32), _ptr(colind, np.int32), int(colind.shape[0]),
        int(log_a.shape[0]), _ptr(cell_nodes, np.int32), _ptr(log_a, np.float64),
        _ptr(K_ref, np.float64), _ptr(val, np.float64), _ptr(cell_a, np.float64), stream))


def gamblet_level_size(h: int, k: int) -> tuple[int, int]:
    a, b = ctypes.c_int32(), ctypes.c_int32()
    _check(_lib.gamblet_level_size(ctypes.c_void_p(h), int(k), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def gamblet_get_operator(h: int, which: int, k: int):
    """COO triplets (rows, cols, vals) of A^(k) (0), R^(k-1,k) (1), B^(k) (2)."""
    nnz = ctypes.c_int64()
    _check(_lib.gamblet_get_operator(ctypes.c_void_p(h), int(which), int(k), 0,
                                     ctypes.byref(nnz), None, None, None))
    r = np.zeros(nnz.value, dtype=np.int32)
    c = np.zeros(nnz.value, dtype=np.int32)
    v = np.zeros(nnz.value, dtype=np.float64)
    _check(_lib.gamblet_get_operator(ctypes.c_void_p(h), int(which), int(k), nnz.value,
                                     ctypes.byref(nnz), _ptr(r), _ptr(c), _ptr(v)))
    return r, c, v


def gamblet_kernel_stats(h: int) -> list[dict]:
    n = _lib.gamblet_kernel_stats(ctypes.c_void_p(h), None, 0)
    arr = (KernelStat * max(n, 1))()
    n = _lib.gamblet_kernel_stats(ctypes.c_void_p(h), arr, n)
    return [{"name": arr[i].name.decode(), "launches": arr[i].launches, "ms": arr[i].ms,
             "bytes": arr[i].bytes, "flops": arr[i].flops} for i in range(n)]


def gamblet_reset_kernel_stats(h: int) -> None:
    _lib.gamblet_reset_kernel_stats(ctypes.c_void_p(h))


def gamblet_kernel_launches() -> int:
    return int(_lib.gamblet_kernel_launches())


def gamblet_plan_check(q: int, rho: float, nbr_rule: int = 0) -> dict:
    """Host-only consistency check of the symbolic plan of a 2^q square (no
    GPU needed); raises GambletError on the first violated property."""
    counts = (ctypes.c_int64 * 5)()
    _check(_lib.gamblet_plan_check(int(q), float(rho), int(nbr_rule),
                                   ctypes.cast(counts, ctypes.c_void_p)))
    return {"levels": counts[0], "phase1_entries": counts[1], "phase1_items": counts[2],
            "phase2_incidences": counts[3], "half_offsets": counts[4]}


def gamblet_device_bytes(h: int) -> int:
    return int(_lib.gamblet_device_bytes(ctypes.c_void_p(h)))


def gamblet_destroy(h: int) -> None:
    _lib.gamblet_destroy(ctypes.c_void_p(h))


def gamblet_status_string(st: int) -> str:
    return _lib.gamblet_status_string(int(st)).decode()


def gamblet_last_error() -> str:
    return _lib.gamblet_last_error().decode()


# ---------------------------------------------------------------- three dimensions
def gamblet3d_setup(rowptr, colind, val, q: int, cells, opts: Opts | None = None) -> int:
    """cells: n x 3 int32 level-q lattice cells (x, y, z)."""
    n = int(rowptr.shape[0]) - 1
    csr = Csr(n, int(colind.shape[0]), _ptr(rowptr, np.int32), _ptr(colind, np.int32),
              _ptr(val, np.float64))
    h = ctypes.c_void_p()
    st = _lib.gamblet3d_setup(ctypes.byref(csr), int(q), _ptr(cells, np.int32),
                              ctypes.byref(opts) if opts is not None else None, ctypes.byref(h))
    if st not in (OK, ERR_NOT_CONVERGED) and h.value:
        _lib.gamblet3d_destroy(h)
    _check(st)
    return h.value


def gamblet3d_solve(h: int, g, u, components=None, info: Info | None = None) -> int:
    return _check(_lib.gamblet3d_solve(ctypes.c_void_p(h), _ptr(g, np.float64),
                                       _ptr(u, np.float64), _ptr(components, np.float64),
                                       ctypes.byref(info) if info is not None else None))


def gamblet3d_level_size(h: int, k: int) -> tuple[int, int]:
    a, b = ctypes.c_int32(), ctypes.c_int32()
    _check(_lib.gamblet3d_level_size(ctypes.c_void_p(h), int(k), ctypes.byref(a),
                                     ctypes.byref(b)))
    return a.value, b.value


def gamblet3d_get_operator(h: int, which: int, k: int):
    """COO triplets (rows, cols, vals) of A^(k) (0), R^(k-1,k) (1), B^(k) (2)."""
    nnz = ctypes.c_int64()
    _check(_lib.gamblet3d_get_operator(ctypes.c_void_p(h), int(which), int(k), 0,
                                       ctypes.byref(nnz), None, None, None))
    r = np.zeros(nnz.value, dtype=np.int32)
    c = np.zeros(nnz.value, dtype=np.int32)
    v = np.zeros(nnz.value, dtype=np.float64)
    _check(_lib.gamblet3d_get_operator(ctypes.c_void_p(h), int(which), int(k), nnz.value,
                                       ctypes.byref(nnz), _ptr(r), _ptr(c), _ptr(v)))
    return r, c, v


def gamblet3d_level_geometry(h: int, k: int) -> dict:
    g = (ctypes.c_int32 * 4)()
    _check(_lib.gamblet3d_level_geometry(ctypes.c_void_p(h), int(k), g))
    return {"neighbours": g[0], "block_offsets": g[1], "patch_iters_max": g[2],
            "dilated_offsets": g[3]}


def gamblet3d_kernel_stats(h: int) -> list[dict]:
    n = _lib.gamblet3d_kernel_stats(ctypes.c_void_p(h), None, 0)
    arr = (KernelStat * max(n, 1))()
    n = _lib.gamblet3d_kernel_stats(ctypes.c_void_p(h), arr, n)
    return [{"name": arr[i].name.decode(), "launches": arr[i].launches, "ms": arr[i].ms,
             "bytes": arr[i].bytes, "flops": arr[i].flops} for i in range(n)]


def gamblet3d_reset_kernel_stats(h: int) -> None:
    _lib.gamblet3d_reset_kernel_stats(ctypes.c_void_p(h))


def gamblet3d_device_bytes(h: int) -> int:
    return int(_lib.gamblet3d_device_bytes(ctypes.c_void_p(h)))


def gamblet3d_destroy(h: int) -> None:
    _lib.gamblet3d_destroy(ctypes.c_void_p(h))
