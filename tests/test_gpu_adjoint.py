"""Adjoint gradient through the autograd wrapper (setup + solve + adjoint
kernel) against the CPU oracle's direct-solve adjoint and central finite
differences, both in float64."""
import numpy as np
import pytest

from oracle import adjoint, direct
from workloads import assemble_q1, cell_corner_dofs, make_problem
from workloads.rough import K_REF

from gpu_util import csr_arrays

pytestmark = pytest.mark.gpu


def _mesh(p):
    from paper_1503_03467_gb300.solver import Q1Mesh
    rp, ci, _ = csr_arrays(p.A)
    return Q1Mesh(rp, ci, p.cells, cell_corner_dofs(p.n), K_REF, p.q)


def _opts(precision=0):
    from paper_1503_03467_gb300 import native as nv
    o = nv.gamblet_default_opts()
    o.precision = precision
    o.refine_max_iter = 60
    o.refine_tol = 1e-13
    o.level_tol = 1e-3
    return o


def _gpu_solve(A, g, q, cells):
    from paper_1503_03467_gb300 import native as nv
    rp, ci, va = csr_arrays(A)
    h = nv.gamblet_setup(rp, ci, va, q, cells, _opts())
    try:
        u = np.zeros(A.shape[0])
        nv.gamblet_solve(h, g, u)
    finally:
        nv.gamblet_destroy(h)
    return u


@pytest.mark.parametrize("precision", [0, 1])
def test_autograd_gradient_matches_oracle_adjoint(precision):
    import torch
    from paper_1503_03467_gb300.solver import gamblet_solve
    n = 32
    p = make_problem(n, 1e3, 0)
    obs = make_problem(n, 1e3, 7)
    u_obs_np, _ = direct.solve(obs.A, p.g)
    dev = torch.device("cuda:0")
    mesh = _mesh(p)
    log_a = torch.tensor(p.log_a.ravel(), dtype=torch.float64, device=dev, requires_grad=True)
    g = torch.tensor(p.g, device=dev)
    u_obs = torch.tensor(u_obs_np, device=dev)
    u = gamblet_solve(log_a, g, mesh, _opts(precision))
    J = 0.5 * ((u - u_obs) ** 2).sum()
    J.backward()
    J_ref, grad_ref, u_ref = adjoint.gradient(p.A, p.g, u_obs_np, n, np.exp(p.log_a), K_REF)
    ud = u.detach().cpu().numpy()
    assert np.linalg.norm(ud - u_ref) / np.linalg.norm(u_ref) < 1e-9
    assert abs(J.item() - J_ref) <= 1e-9 * J_ref
    gr = log_a.grad.cpu().numpy()
    assert np.linalg.norm(gr - grad_ref) / np.linalg.norm(grad_ref) < 1e-8


def test_gradient_matches_central_differences_on_gpu_solves():
    import torch
    from paper_1503_03467_gb300.solver import gamblet_solve
    n = 16
    p = make_problem(n, 1e3, 3)
    obs = make_problem(n, 1e3, 7)
    u_obs = direct.solve(obs.A, p.g)[0]
    dev = torch.device("cuda:0")
    log_a = torch.tensor(p.log_a.ravel(), dtype=torch.float64, device=dev, requires_grad=True)
    u = gamblet_solve(log_a, torch.tensor(p.g, device=dev), _mesh(p), _opts())
    (0.5 * ((u - torch.tensor(u_obs, device=dev)) ** 2).sum()).backward()
    grad = log_a.grad.cpu().numpy()
    rng = np.random.default_rng(7)
    h = 1e-6
    for c in rng.choice(n * n, 8, replace=False):
        lp = p.log_a.ravel().copy()
        lm = p.log_a.ravel().copy()
        lp[c] += h
        lm[c] -= h
        Ap = assemble_q1(np.exp(lp).reshape(n, n))
        Am = assemble_q1(np.exp(lm).reshape(n, n))
        um = _gpu_solve(Am, p.g, p.q, p.cells)
        # J+ - J- = delta^T (u- - u_obs) + 1/2 delta^T delta, A+ delta = -(A+ - A-) u-
        delta = _gpu_solve(Ap, -((Ap - Am) @ um), p.q, p.cells)
        fd = (delta @ (um - u_obs) + 0.5 * delta @ delta) / (2 * h)
        assert abs(fd - grad[c]) <= 1e-6 * max(abs(grad[c]), 1e-3 * np.abs(grad).max())


def test_assemble_cells_matches_host_assembly():
    import torch
    from paper_1503_03467_gb300 import native as nv
    p = make_problem(32, 1e4, 5)
    mesh = _mesh(p)
    dev = torch.device("cuda:0")
    la = torch.tensor(p.log_a.ravel(), device=dev)
    val = torch.empty(mesh.colind.numel(), dtype=torch.float64, device=dev)
    a = torch.empty_like(la)
    nv.gamblet_assemble_cells(mesh.rowptr, mesh.colind, mesh.cell_nodes, la, mesh.K_ref, val, a)
    _, _, va = csr_arrays(p.A)
    assert np.abs(val.cpu().numpy() - va).max() <= 1e-13 * np.abs(va).max()
    assert np.allclose(a.cpu().numpy(), np.exp(p.log_a.ravel()), rtol=1e-15)


def test_recomputed_hierarchy_gives_the_same_gradient():
    """keep_hierarchy=False releases the hierarchy after the forward solve
    and recomputes it in the backward pass: the gradient is the one of the
    kept hierarchy (the setup is deterministic)."""
    import torch
    from paper_1503_03467_gb300.solver import gamblet_solve
    n = 32
    p = make_problem(n, 1e3, 2)
    obs = make_problem(n, 1e3, 7)
    u_obs = torch.tensor(direct.solve(obs.A, p.g)[0], device="cuda:0")
    g = torch.tensor(p.g, device="cuda:0")
    mesh = _mesh(p)
    grads = []
    for keep in (True, False):
        log_a = torch.tensor(p.log_a.ravel(), dtype=torch.float64, device="cuda:0",
                             requires_grad=True)
        u = gamblet_solve(log_a, g, mesh, _opts(1), keep_hierarchy=keep)
        (0.5 * ((u - u_obs) ** 2).sum()).backward()
        grads.append(log_a.grad.cpu().numpy())
    assert np.linalg.norm(grads[1] - grads[0]) <= 1e-12 * np.linalg.norm(grads[0])


def test_gradient_at_256x256_matches_direct_adjoint_and_central_differences():
    """The adjoint workload at its stated size: 256 x 256 cells (65,025
    unknowns), q = 8, contrast 1e3, coefficient and g from seed 0, u_obs the
    float64 direct solution for the field of seed 7.  The gradient comes
    from the autograd wrapper with the hierarchy released after the forward
    solve and recomputed level by level in the backward pass.  It must match
    the oracle's direct-solve adjoint element by element (1e-8 of its largest
    entry) and central differences in log a (step 1e-6, exact difference
    form, GPU solves) on 32 cells drawn with default_rng(7) to 1e-6."""
    import torch
    from paper_1503_03467_gb300.solver import gamblet_solve
    n = 256
    p = make_problem(n, 1e3, 0)
    obs = make_problem(n, 1e3, 7)
    u_obs_np = direct.solve(obs.A, p.g)[0]
    dev = torch.device("cuda:0")
    o = _opts()
    o.refine_tol = 1e-14
    log_a = torch.tensor(p.log_a.ravel(), dtype=torch.float64, device=dev, requires_grad=True)
    u = gamblet_solve(log_a, torch.tensor(p.g, device=dev), _mesh(p), o, keep_hierarchy=False)
    (0.5 * ((u - torch.tensor(u_obs_np, device=dev)) ** 2).sum()).backward()
    grad = log_a.grad.cpu().numpy()
    _, grad_ref, _ = adjoint.gradient(p.A, p.g, u_obs_np, n, np.exp(p.log_a), K_REF)
    assert np.abs(grad - grad_ref).max() <= 1e-8 * np.abs(grad_ref).max()

    def solve(A, g):
        from paper_1503_03467_gb300 import native as nv
        rp, ci, va = csr_arrays(A)
        h = nv.gamblet_setup(rp, ci, va, p.q, p.cells, o)
        try:
            x = np.zeros(A.shape[0])
            nv.gamblet_solve(h, g, x)
        finally:
            nv.gamblet_destroy(h)
        return x

    rng = np.random.default_rng(7)
    step = 1e-6
    for c in rng.choice(n * n, 32, replace=False):
        lp = p.log_a.ravel().copy()
        lm = p.log_a.ravel().copy()
        lp[c] += step
        lm[c] -= step
        Ap = assemble_q1(np.exp(lp).reshape(n, n))
        Am = assemble_q1(np.exp(lm).reshape(n, n))
        um = solve(Am, p.g)
        # J+ - J- = delta^T (u- - u_obs) + 1/2 delta^T delta, A+ delta = -(A+ - A-) u-
        delta = solve(Ap, -((Ap - Am) @ um))
        fd = (delta @ (um - u_obs_np) + 0.5 * delta @ delta) / (2 * step)
        assert abs(fd - grad[c]) <= 1e-6 * max(abs(grad[c]), 1e-3 * np.abs(grad).max()), c
