"""Pins of the compression in the normalised gamblet basis (oracle)."""
import numpy as np

from oracle.compress import compress, normalised_coefficients
from oracle.local import gamblet_local_setup, gamblet_local_solve
from workloads import make_problem


def test_no_threshold_reproduces_the_one_pass_solution():
    p = make_problem(16, 1e3, 0)
    s = gamblet_local_setup(p.A, p.cells, p.q, 3.0)
    u, kept, total = compress(s, p.g, 0.0)
    assert kept == total == p.ndof  # one coefficient per unknown (I^(1) plus every J^(k))
    assert np.allclose(u, gamblet_local_solve(s, p.g)["u"], rtol=0, atol=1e-12)


def test_dropped_energy_is_the_sum_over_levels():
    """Exact transform: the components of different levels are
    A-orthogonal (Theorem thmgugyug2), so the energy of u - u_c is the sum
    of the level energies of the dropped coefficients,
    w_d^T B^(k) w_d and U_d^T A^(1) U_d."""
    p = make_problem(16, 1e3, 1)
    s = gamblet_local_setup(p.A, p.cells, p.q, np.inf)
    c, res = normalised_coefficients(s, p.g)
    eps = 0.05
    u_c, kept, total = compress(s, p.g, eps)
    cmax = max(np.abs(v).max() for v in c.values())
    drop = {k: np.abs(v) < eps * cmax for k, v in c.items()}
    Ud = np.where(drop[1], res["U1"], 0.0)
    e = Ud @ (s["A"][1] @ Ud)
    for k in range(2, p.q + 1):
        wd = np.where(drop[k], res["w"][k], 0.0)
        e += wd @ (s["B"][k] @ wd)
    d = res["u"] - u_c
    assert 0 < kept < total
    assert np.isclose(d @ (p.A @ d), e, rtol=1e-9)


def test_representation_is_sparse_for_example1():
    """The paper's observation on Example 1 (Sec. 5.1, figures of the
    coefficients and of the compressed solution): most normalised
    coefficients are negligible; a 1e-3 relative threshold keeps about 5 %
    of them and loses about 1e-4 of the energy (a white-noise right-hand
    side, active on every scale, is not sparse: that is the paper's point)."""
    from workloads import make_example1
    p = make_example1(6)
    s = gamblet_local_setup(p.A, p.cells, p.q, 3.0)
    u = gamblet_local_solve(s, p.g)["u"]
    u_c, kept, total = compress(s, p.g, 1e-3)
    d = u - u_c
    assert kept < 0.1 * total
    assert d @ (p.A @ d) < 1e-3 * (u @ (p.A @ u))
