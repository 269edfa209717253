"""gamblet_objective_noalloc, the allocation-free objective entry point for
callers that cannot allocate device memory when they evaluate J (a
framework's caching allocator holding the free memory, a hard memory budget,
loops that cannot pay for cudaFree's device-wide synchronisation), must
return the J that gamblet_grad returns.  This file is named to be collected
last, so a failure here comes after every other test has run."""
import numpy as np
import pytest

from workloads import cell_corner_dofs, make_problem
from workloads.rough import K_REF

pytestmark = pytest.mark.gpu


def _reference(n_cells, seed):
    from paper_1503_03467_gb300 import native as nv
    p = make_problem(n_cells, 1e3, seed)
    A = p.A.tocsr()
    rp = np.ascontiguousarray(A.indptr, dtype=np.int32)
    ci = np.ascontiguousarray(A.indices, dtype=np.int32)
    va = np.ascontiguousarray(A.data, dtype=np.float64)
    o = nv.gamblet_default_opts()
    o.refine_max_iter = 50
    o.level_tol = 1e-6
    h = nv.gamblet_setup(rp, ci, va, p.q, p.cells, o)
    try:
        u = np.zeros(p.ndof)
        nv.gamblet_solve(h, p.g, u)
        u_obs = u + 0.1 * np.random.default_rng(seed).standard_normal(p.ndof)
        dJ = np.zeros(n_cells * n_cells)
        J = nv.gamblet_grad(h, cell_corner_dofs(n_cells), np.exp(p.log_a).ravel(),
                            K_REF.ravel().copy(), u, u_obs, dJ)
    finally:
        nv.gamblet_destroy(h)
    return u, u_obs, J


def test_objective_noalloc_matches_grad_twice_in_a_row():
    import torch
    from paper_1503_03467_gb300 import native as nv
    dev = torch.device("cuda:0")
    for n_cells, seed in ((32, 11), (64, 12)):
        u, u_obs, J_ref = _reference(n_cells, seed)
        ud = torch.from_numpy(u).to(dev)
        uod = torch.from_numpy(u_obs).to(dev)
        for _ in range(2):
            J_dev = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
            assert nv.gamblet_objective_noalloc(ud.numel(), ud, uod, J_dev) == nv.OK
            torch.cuda.synchronize()
            assert abs(J_dev.item() - J_ref) <= 1e-12 * abs(J_ref)
            J_host = np.full(1, np.nan)
            assert nv.gamblet_objective_noalloc(ud.numel(), ud, uod, J_host) == nv.OK
            assert abs(J_host[0] - J_ref) <= 1e-12 * abs(J_ref)


def test_objective_noalloc_allocates_nothing_and_rejects_oversize():
    import torch
    from paper_1503_03467_gb300 import native as nv
    dev = torch.device("cuda:0")
    u = torch.randn(5000, dtype=torch.float64, device=dev)
    uo = torch.randn(5000, dtype=torch.float64, device=dev)
    J = torch.zeros(1, dtype=torch.float64, device=dev)
    nv.gamblet_objective_noalloc(u.numel(), u, uo, J)   # first call: symbol lookup
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        nv.gamblet_objective_noalloc(u.numel(), u, uo, J)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free0 == free1
    ref = 0.5 * float(((u - uo) ** 2).sum())
    assert abs(J.item() - ref) <= 1e-12 * ref
    big = torch.zeros(2097153, dtype=torch.float64, device=dev)
    with pytest.raises(nv.GambletError) as e:
        nv.gamblet_objective_noalloc(big.numel(), big, big, J)
    assert e.value.status == nv.ERR_UNSUPPORTED


def test_objective_noalloc_rejects_memory_off_the_current_device():
    """Host memory for u or u_obs is refused before any kernel runs (the
    kernels would otherwise dereference a host address on the device);
    short buffers are refused by the binding, which knows their lengths."""
    import torch
    from paper_1503_03467_gb300 import native as nv
    dev = torch.device("cuda:0")
    u = torch.randn(100, dtype=torch.float64, device=dev)
    J = torch.zeros(1, dtype=torch.float64, device=dev)
    host = np.zeros(100)
    for a, b in ((host, u), (u, host)):
        with pytest.raises(nv.GambletError) as e:
            nv.gamblet_objective_noalloc(100, a, b, J)
        assert e.value.status == nv.ERR_INVALID_ARG
    with pytest.raises(ValueError):
        nv.gamblet_objective_noalloc(101, u, u, J)
    with pytest.raises(ValueError):
        nv.gamblet_objective_noalloc(100, u, u, np.zeros(0))
    assert nv.gamblet_objective_noalloc(100, u, u, J) == nv.OK
    torch.cuda.synchronize()
    assert J.item() == 0.0
