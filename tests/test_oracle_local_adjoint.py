"""Pins of the one-pass localized gradient oracle (oracle/local_adjoint.py):
central differences of the one-pass map J(theta) = 1/2 |u_loc(theta) - u_obs|^2
itself (Algorithm 2 forward only), the exact-solution adjoint when every
patch covers the domain (Algorithm 2 then reduces to Algorithm 1, whose u is
A^-1 g), and dJ/dg = G_loc (u_loc - u_obs), G_loc being symmetric.  Planted
mistakes in the reverse pass (on the CPU) must fail the difference check."""
import inspect
import types

import numpy as np
import pytest

import oracle.local_adjoint as la
from oracle import adjoint, direct
from oracle.local import gamblet_local_setup, gamblet_local_solve
from workloads import assemble_q1, cell_corner_dofs, make_problem
from workloads.rough import K_REF

N, CONTRAST, RHO = 16, 1e4, 1.0


def _case():
    p = make_problem(N, CONTRAST, 0)
    obs = make_problem(N, CONTRAST, 7)
    u_obs, _ = direct.solve(obs.A, p.g)
    return p, u_obs


def _J(p, u_obs, log_a, rho):
    A = assemble_q1(np.exp(log_a).reshape(N, N))
    S = gamblet_local_setup(A, p.cells, p.q, rho)
    u = gamblet_local_solve(S, p.g)["u"]
    return 0.5 * float((u - u_obs) @ (u - u_obs))


def _fd_directional(p, u_obs, d, rho, h=1e-5):
    la0 = p.log_a.ravel()
    return (_J(p, u_obs, la0 + h * d, rho) - _J(p, u_obs, la0 - h * d, rho)) / (2 * h)


@pytest.mark.parametrize("rho", [1.0, 2.0])
def test_one_pass_gradient_matches_central_differences(rho):
    p, u_obs = _case()
    r = la.gradient_one_pass(p.A, p.g, u_obs, N, np.exp(p.log_a), K_REF, p.cells, p.q, rho)
    assert abs(r["J"] - _J(p, u_obs, p.log_a.ravel(), rho)) <= 1e-13 * r["J"]
    rng = np.random.default_rng(3)
    d = rng.standard_normal(N * N)
    fd = _fd_directional(p, u_obs, d, rho)
    assert abs(fd - r["grad"] @ d) <= 1e-8 * abs(fd)
    # single cells, the largest and a few random ones
    cells = [int(np.argmax(np.abs(r["grad"])))] + list(rng.choice(N * N, 3, replace=False))
    for c in cells:
        e = np.zeros(N * N)
        e[c] = 1.0
        fd = _fd_directional(p, u_obs, e, rho)
        assert abs(fd - r["grad"][c]) <= 1e-7 * np.abs(r["grad"]).max()


def test_localized_gradient_differs_from_exact_adjoint():
    """At rho = 1 the one-pass map is not A^-1: its gradient is a different
    quantity (so the difference check above is not the exact adjoint's)."""
    p, u_obs = _case()
    a = np.exp(p.log_a)
    r = la.gradient_one_pass(p.A, p.g, u_obs, N, a, K_REF, p.cells, p.q, RHO)
    _, ge, _ = adjoint.gradient(p.A, p.g, u_obs, N, a, K_REF)
    assert np.abs(r["grad"] - ge).max() > 1e-3 * np.abs(ge).max()


def test_patches_covering_the_domain_give_the_exact_adjoint():
    p, u_obs = _case()
    a = np.exp(p.log_a)
    r = la.gradient_one_pass(p.A, p.g, u_obs, N, a, K_REF, p.cells, p.q, 100.0)
    J, ge, u = adjoint.gradient(p.A, p.g, u_obs, N, a, K_REF)
    assert np.abs(r["u"] - u).max() <= 1e-10 * np.abs(u).max()
    assert np.abs(r["grad"] - ge).max() <= 1e-10 * np.abs(ge).max()


def test_rhs_gradient_is_the_one_pass_solve_of_the_misfit():
    p, u_obs = _case()
    r = la.gradient_one_pass(p.A, p.g, u_obs, N, np.exp(p.log_a), K_REF, p.cells, p.q, RHO)
    ref = gamblet_local_solve(r["setup"], r["u"] - u_obs)["u"]
    assert np.abs(r["dJ_dg"] - ref).max() <= 1e-12 * np.abs(ref).max()


def _holed(p):
    """Nodes of a rectangle and a single node removed (Dirichlet there): some
    parents have fewer than four children and some cells none."""
    x, y = p.cells[:, 0], p.cells[:, 1]
    keep = ~((x >= 5) & (x <= 8) & (y >= 6) & (y <= 7)) & ~((x == 2) & (y == 13))
    idx = np.nonzero(keep)[0]
    new = -np.ones(p.ndof, dtype=np.int64)
    new[idx] = np.arange(len(idx))
    cd = cell_corner_dofs(N)
    cn = np.where(cd >= 0, new[np.maximum(cd, 0)], -1)
    return idx, cn


def test_one_pass_gradient_on_a_domain_with_holes():
    p, _ = _case()
    idx, cn = _holed(p)
    u_obs = np.random.default_rng(11).standard_normal(len(idx))
    g = p.g[idx]

    def J(log_a):
        A = assemble_q1(np.exp(log_a).reshape(N, N))[idx][:, idx]
        S = gamblet_local_setup(A, p.cells[idx], p.q, 2.0)
        u = gamblet_local_solve(S, g)["u"]
        return 0.5 * float((u - u_obs) @ (u - u_obs))

    A = p.A[idx][:, idx]
    r = la.gradient_one_pass(A, g, u_obs, N, np.exp(p.log_a), K_REF, p.cells[idx], p.q, 2.0,
                             cell_nodes=cn)
    d = np.random.default_rng(3).standard_normal(N * N)
    h = 1e-5
    la0 = p.log_a.ravel()
    fd = (J(la0 + h * d) - J(la0 - h * d)) / (2 * h)
    assert abs(fd - r["grad"] @ d) <= 1e-8 * abs(fd)


MUTATIONS = {
    "galerkin_R_adjoint_without_factor_2": ("Rbar[k] += 2.0 * Xbar", "Rbar[k] += 1.0 * Xbar"),
    "galerkin_A_adjoint_dropped": ("Abar[k] += R[k].T @ Xbar @ R[k]", "pass"),
    "patch_matrix_adjoint_dropped": ("Bbar[np.ix_(chi, chi)] -= np.outer(mu, y)", "pass"),
    "patch_rhs_adjoint_dropped": ("rhsbar[chi, i] += mu", "pass"),
    "prolongation_outer_product_dropped": ("Rbar[k] += np.outer(v[k - 1], vbar[k])", "pass"),
    "restriction_outer_product_dropped": ("Rbar[k] += np.outer(gbar[k - 1], gk[k])", "pass"),
    "no_symmetrisation": ("Xbar = 0.5 * (Abar[k - 1] + Abar[k - 1].T)", "Xbar = Abar[k - 1]"),
    "level_solve_adjoint_sign": ("Abar[k] += W[k].T @ (-np.outer(lam[k], w[k])) @ W[k]",
                                 "Abar[k] += W[k].T @ np.outer(lam[k], w[k]) @ W[k]"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_difference_check_catches_mutation(name):
    src = inspect.getsource(la)
    old, new = MUTATIONS[name]
    assert old in src, name
    mod = types.ModuleType("oracle.local_adjoint_mut")
    mod.__dict__["__package__"] = "oracle"
    exec(compile(src.replace(old, new), "<mutant>", "exec"), mod.__dict__)
    p, u_obs = _case()
    r = mod.gradient_one_pass(p.A, p.g, u_obs, N, np.exp(p.log_a), K_REF, p.cells, p.q, RHO)
    d = np.random.default_rng(3).standard_normal(N * N)
    fd = _fd_directional(p, u_obs, d, RHO)
    assert abs(fd - r["grad"] @ d) > 1e-6 * abs(fd)
