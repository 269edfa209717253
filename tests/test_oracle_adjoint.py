"""Pin of the adjoint-gradient oracle by central finite differences."""
import numpy as np

from oracle import adjoint, direct
from workloads import assemble_q1, make_problem
from workloads.rough import K_REF


def test_adjoint_matches_central_differences():
    n = 16
    p = make_problem(n, 1e3, 0)
    obs = make_problem(n, 1e3, 7)
    u_obs, _ = direct.solve(obs.A, p.g)
    a = np.exp(p.log_a)
    J, grad, u = adjoint.gradient(p.A, p.g, u_obs, n, a, K_REF)
    rng = np.random.default_rng(7)
    cells = rng.choice(n * n, 32, replace=False)
    h = 1e-6
    for c in cells:
        la_p = p.log_a.copy().ravel()
        la_m = p.log_a.copy().ravel()
        la_p[c] += h
        la_m[c] -= h
        Ap = assemble_q1(np.exp(la_p).reshape(n, n))
        Am = assemble_q1(np.exp(la_m).reshape(n, n))
        um, _ = direct.solve(Am, p.g)
        # exact difference form: with A+ delta = -(A+ - A-) u-,
        # J+ - J- = delta^T (u- - u_obs) + 1/2 delta^T delta (no cancellation)
        delta, _ = direct.solve(Ap, -((Ap - Am) @ um))
        dJ = delta @ (um - u_obs) + 0.5 * delta @ delta
        fd = dJ / (2 * h)
        assert abs(fd - grad[c]) <= 1e-6 * max(abs(grad[c]), 1e-3 * np.abs(grad).max())


def test_adjoint_gradient_zero_at_observation():
    n = 8
    p = make_problem(n, 10, 1)
    u, _ = direct.solve(p.A, p.g)
    J, grad, _ = adjoint.gradient(p.A, p.g, u, n, np.exp(p.log_a), K_REF)
    assert J < 1e-25
    assert np.abs(grad).max() < 1e-12
