"""Gradient of J = 1/2 |u_loc - u_obs|^2 through the one-pass localized
transform (gamblet_grad_onepass, float64, patch solves to 1e-13 and level
solves to 1e-12) against the CPU oracle's reverse pass (oracle/local_adjoint.py), and at
256 x 256 cells against central differences of the GPU's own one-pass map."""
import numpy as np
import pytest

from oracle import direct, local_adjoint
from workloads import assemble_q1, cell_corner_dofs, make_problem
from workloads.rough import K_REF

from gpu_util import csr_arrays

pytestmark = pytest.mark.gpu


def _opts(rho, precision=0, rule=0):
    from paper_1503_03467_gb300 import native as nv
    o = nv.gamblet_default_opts()
    o.precision = precision
    o.rho = rho
    o.nbr_rule = rule
    o.patch_tol = 1e-13
    o.level_tol = 1e-12
    o.level_max_iter = 5000
    return o


def _gpu_grad(A, p, u_obs, rho, log_a=None, g=None, cells=None, cell_nodes=None, rule=0):
    from paper_1503_03467_gb300 import native as nv
    log_a = p.log_a.ravel() if log_a is None else log_a
    g = p.g if g is None else g
    cells = p.cells if cells is None else cells
    cell_nodes = cell_corner_dofs(p.n) if cell_nodes is None else cell_nodes
    rp, ci, va = csr_arrays(A)
    h = nv.gamblet_setup(rp, ci, va, p.q, cells, _opts(rho, rule=rule))
    try:
        ncell = p.n * p.n
        dJ = np.zeros(ncell)
        u = np.zeros(A.shape[0])
        dg = np.zeros(A.shape[0])
        info = nv.Info()
        J = nv.gamblet_grad_onepass(h, cell_nodes, np.exp(log_a), K_REF.ravel().copy(),
                                    g, u_obs, dJ, u=u, dJ_dg=dg, info=info)
        assert info.status == 0
    finally:
        nv.gamblet_destroy(h)
    return J, dJ, u, dg


@pytest.mark.parametrize("n,rho", [(4, 1.0), (8, 2.0), (16, 1.0), (16, 2.0), (16, 3.0),
                                   (32, 3.0), (32, 1.5)])
def test_onepass_gradient_matches_oracle(n, rho):
    p = make_problem(n, 1e4, 0)
    obs = make_problem(n, 1e4, 7)
    u_obs, _ = direct.solve(obs.A, p.g)
    J, dJ, u, dg = _gpu_grad(p.A, p, u_obs, rho)
    r = local_adjoint.gradient_one_pass(p.A, p.g, u_obs, n, np.exp(p.log_a), K_REF, p.cells,
                                        p.q, rho)
    assert np.linalg.norm(u - r["u"]) <= 1e-10 * np.linalg.norm(r["u"])
    assert abs(J - r["J"]) <= 1e-10 * r["J"]
    assert np.linalg.norm(dg - r["dJ_dg"]) <= 1e-9 * np.linalg.norm(r["dJ_dg"])
    assert np.abs(dJ - r["grad"]).max() <= 1e-8 * np.abs(r["grad"]).max()


def _close(J, dJ, u, dg, r):
    assert np.linalg.norm(u - r["u"]) <= 1e-10 * np.linalg.norm(r["u"])
    assert abs(J - r["J"]) <= 1e-10 * r["J"]
    assert np.linalg.norm(dg - r["dJ_dg"]) <= 1e-9 * np.linalg.norm(r["dJ_dg"])
    assert np.abs(dJ - r["grad"]).max() <= 1e-8 * np.abs(r["grad"]).max()


def test_onepass_gradient_on_domains_with_holes():
    """Removed nodes (Dirichlet there) leave parents with one to three
    children and cells with none: the child masks of every reverse kernel."""
    n = 32
    p = make_problem(n, 1e3, 8)
    x, y = p.cells[:, 0], p.cells[:, 1]
    masks = [~((x >= 10) & (x <= 17) & (y >= 12) & (y <= 14)) & ~((x == 3) & (y == 29)),
             ~((x >= 16) & (y >= 16)) & ~((x >= 9) & (x <= 11) & (y <= 4))]
    for keep in masks:
        idx = np.nonzero(keep)[0]
        new = -np.ones(p.ndof, dtype=np.int64)
        new[idx] = np.arange(len(idx))
        cd = cell_corner_dofs(n)
        cn = np.ascontiguousarray(np.where(cd >= 0, new[np.maximum(cd, 0)], -1), dtype=np.int32)
        A = p.A[idx][:, idx]
        g = np.ascontiguousarray(p.g[idx])
        cells = np.ascontiguousarray(p.cells[idx])
        u_obs = np.random.default_rng(11).standard_normal(len(idx))
        J, dJ, u, dg = _gpu_grad(A, p, u_obs, 3.0, g=g, cells=cells, cell_nodes=cn)
        r = local_adjoint.gradient_one_pass(A, g, u_obs, n, np.exp(p.log_a), K_REF, cells, p.q,
                                            3.0, cell_nodes=cn)
        _close(J, dJ, u, dg, r)


def test_onepass_gradient_chebyshev_patches():
    n = 16
    p = make_problem(n, 1e4, 4)
    u_obs = np.random.default_rng(12).standard_normal(p.ndof)
    J, dJ, u, dg = _gpu_grad(p.A, p, u_obs, 2.0, rule=1)
    r = local_adjoint.gradient_one_pass(p.A, p.g, u_obs, n, np.exp(p.log_a), K_REF, p.cells,
                                        p.q, 2.0, rule="cheb")
    _close(J, dJ, u, dg, r)


def test_onepass_gradient_of_uniform_coefficient_misfit_zero():
    """u_obs = u_loc: J = 0 and every derivative vanishes."""
    p = make_problem(16, 10.0, 2)
    _, _, u, _ = _gpu_grad(p.A, p, np.zeros(p.ndof), 2.0)
    J, dJ, _, dg = _gpu_grad(p.A, p, u, 2.0)
    assert J <= 1e-26 * float(u @ u)
    assert np.abs(dJ).max() <= 1e-12 and np.abs(dg).max() <= 1e-12


def test_onepass_gradient_at_256_matches_central_differences():
    """The derivative along a random direction of log a against central
    differences of J through the GPU's one-pass map (5 setups of 65,025
    unknowns, rho = 3)."""
    n = 256
    p = make_problem(n, 1e3, 0)
    obs = make_problem(n, 1e3, 7)
    u_obs = direct.solve(obs.A, p.g)[0]
    J0, dJ, _, _ = _gpu_grad(p.A, p, u_obs, 3.0)
    d = np.random.default_rng(5).standard_normal(n * n)
    # fourth-order central differences: a step large enough that the noise
    # of the iterative solves (1e-12) stays far below the tolerance, with a
    # truncation error of order h^4
    h = 1e-4
    Js = {}
    for m in (2, 1, -1, -2):
        la = p.log_a.ravel() + m * h * d
        A = assemble_q1(np.exp(la).reshape(n, n))
        Js[m] = _gpu_grad(A, p, u_obs, 3.0, log_a=la)[0]
    fd = (8 * (Js[1] - Js[-1]) - (Js[2] - Js[-2])) / (12 * h)
    assert abs(fd - dJ @ d) <= 1e-6 * abs(fd)


def test_onepass_gradient_mixed_precision():
    """The mixed path's float32 hierarchy: the reverse pass in float32 (patch
    and level solves to 1e-6) against the oracle's float64 gradient."""
    from paper_1503_03467_gb300 import native as nv
    n = 32
    p = make_problem(n, 1e4, 0)
    obs = make_problem(n, 1e4, 7)
    u_obs, _ = direct.solve(obs.A, p.g)
    rp, ci, va = csr_arrays(p.A)
    o = _opts(3.0, precision=nv.MIXED)
    o.patch_tol = 1e-6
    o.level_tol = 1e-6
    h = nv.gamblet_setup(rp, ci, va, p.q, p.cells, o)
    try:
        dJ = np.zeros(n * n)
        u = np.zeros(p.ndof)
        dg = np.zeros(p.ndof)
        J = nv.gamblet_grad_onepass(h, cell_corner_dofs(n), np.exp(p.log_a.ravel()),
                                    K_REF.ravel().copy(), p.g, u_obs, dJ, u=u, dJ_dg=dg)
    finally:
        nv.gamblet_destroy(h)
    r = local_adjoint.gradient_one_pass(p.A, p.g, u_obs, n, np.exp(p.log_a), K_REF, p.cells,
                                        p.q, 3.0)
    assert np.linalg.norm(u - r["u"]) <= 1e-4 * np.linalg.norm(r["u"])
    assert abs(J - r["J"]) <= 1e-4 * r["J"]
    assert np.linalg.norm(dg - r["dJ_dg"]) <= 1e-4 * np.linalg.norm(r["dJ_dg"])
    assert np.linalg.norm(dJ - r["grad"]) <= 1e-3 * np.linalg.norm(r["grad"])


def test_onepass_gradient_needs_iterative_patch_solves():
    from paper_1503_03467_gb300 import native as nv
    p = make_problem(16, 10.0, 0)
    rp, ci, va = csr_arrays(p.A)
    o = _opts(2.0)
    o.patch_tol = -1.0  # dense Cholesky patch solves
    h = nv.gamblet_setup(rp, ci, va, p.q, p.cells, o)
    try:
        with pytest.raises(nv.GambletError) as e:
            nv.gamblet_grad_onepass(h, cell_corner_dofs(16), np.exp(p.log_a.ravel()),
                                    K_REF.ravel().copy(), p.g, np.zeros(p.ndof),
                                    np.zeros(256))
        assert e.value.status == nv.ERR_UNSUPPORTED
    finally:
        nv.gamblet_destroy(h)


def test_autograd_one_pass_gradients_match_oracle():
    """The autograd wrapper: dL/dlog a and dL/dg of L = 1/2 |u_loc - u_obs|^2."""
    import torch
    from paper_1503_03467_gb300.solver import Q1Mesh, gamblet_one_pass
    n, rho = 32, 2.0
    p = make_problem(n, 1e4, 1)
    obs = make_problem(n, 1e4, 7)
    u_obs_np, _ = direct.solve(obs.A, p.g)
    dev = torch.device("cuda:0")
    rp, ci, _ = csr_arrays(p.A)
    mesh = Q1Mesh(rp, ci, p.cells, cell_corner_dofs(n), K_REF, p.q, dev)
    log_a = torch.tensor(p.log_a.ravel(), dtype=torch.float64, device=dev, requires_grad=True)
    g = torch.tensor(p.g, device=dev, requires_grad=True)
    o = _opts(rho)
    u = gamblet_one_pass(log_a, g, mesh, o)
    assert o.refine_max_iter == _opts(rho).refine_max_iter  # the caller's options are untouched
    L = 0.5 * ((u - torch.tensor(u_obs_np, device=dev)) ** 2).sum()
    L.backward()
    r = local_adjoint.gradient_one_pass(p.A, p.g, u_obs_np, n, np.exp(p.log_a), K_REF, p.cells,
                                        p.q, rho)
    assert np.linalg.norm(u.detach().cpu().numpy() - r["u"]) <= 1e-10 * np.linalg.norm(r["u"])
    ga = log_a.grad.cpu().numpy()
    assert np.abs(ga - r["grad"]).max() <= 1e-8 * np.abs(r["grad"]).max()
    gg = g.grad.cpu().numpy()
    assert np.linalg.norm(gg - r["dJ_dg"]) <= 1e-9 * np.linalg.norm(r["dJ_dg"])


def test_onepass_outputs_at_512_equal_one_pass_solves():
    """At 512 x 512 (mixed, bench level tolerance): u_loc and dJ/dg of
    gamblet_grad_onepass equal gamblet_solve's one-pass output (no outer
    refinement) for g and for the misfit u_loc - u_obs, through the same
    handle (G_loc is symmetric)."""
    from paper_1503_03467_gb300 import native as nv
    n = 512
    p = make_problem(n, 1e4, 0)
    rp, ci, va = csr_arrays(p.A)
    o = _opts(3.0, precision=nv.MIXED)
    o.patch_tol = 0.0  # the mixed default
    o.level_tol = 0.05
    o.refine_max_iter = 0
    h = nv.gamblet_setup(rp, ci, va, p.q, p.cells, o)
    try:
        u_obs = np.random.default_rng(21).standard_normal(p.ndof)
        dJ = np.zeros(n * n)
        u = np.zeros(p.ndof)
        dg = np.zeros(p.ndof)
        J = nv.gamblet_grad_onepass(h, cell_corner_dofs(n), np.exp(p.log_a.ravel()),
                                    K_REF.ravel().copy(), p.g, u_obs, dJ, u=u, dJ_dg=dg)
        u1 = np.zeros(p.ndof)
        nv.gamblet_solve(h, p.g, u1)
        dg1 = np.zeros(p.ndof)
        nv.gamblet_solve(h, u1 - u_obs, dg1)
    finally:
        nv.gamblet_destroy(h)
    assert np.linalg.norm(u - u1) <= 1e-6 * np.linalg.norm(u1)
    assert abs(J - 0.5 * float((u1 - u_obs) @ (u1 - u_obs))) <= 1e-6 * J
    assert np.linalg.norm(dg - dg1) <= 1e-5 * np.linalg.norm(dg1)
    assert np.all(np.isfinite(dJ)) and np.abs(dJ).max() > 0
