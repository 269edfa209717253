"""GPU parity of the mass-matrix initialisation (Algorithm 1 lines 1-5;
Algorithm 2 lines 2a-5 with Definition deflocinvm) against the oracle."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.massinit import gamblet_mass_setup, gamblet_mass_solve, mass_initialised_operator
from workloads import assemble_q1_mass, make_example1, make_problem

from gpu_util import check_R, check_op, coo_to_dense, csr_arrays, rel

pytestmark = pytest.mark.gpu


def _opts(precision=0, refine=0):
    from paper_1503_03467_gb300 import native as nv
    o = nv.gamblet_default_opts()
    o.precision = precision
    o.level_tol = 1e-14 if refine == 0 else 0.1
    o.level_max_iter = 5000
    o.refine_max_iter = refine
    o.refine_tol = 1e-12
    return o


def _setup(p, M, rho_q, o):
    from paper_1503_03467_gb300 import native as nv
    return nv.gamblet_setup_mass(csr_arrays(p.A), csr_arrays(M), p.q, p.cells, rho_q, o)


@pytest.mark.parametrize("rho_q", [1.0, 2.0])
def test_mass_initialised_operators_and_one_pass_match_oracle(rho_q):
    from paper_1503_03467_gb300 import native as nv
    p = make_problem(32, 1e3, 3)
    M = assemble_q1_mass(32)
    ref = gamblet_mass_setup(p.A, M, p.cells, p.q, 3.0, rho_q)
    u_ref, _ = gamblet_mass_solve(ref, p.g)
    h = _setup(p, M, rho_q, _opts())
    try:
        n = p.ndof
        Aq = coo_to_dense(*nv.gamblet_get_operator(h, 0, p.q), (n, n))
        check_op(Aq, ref["A"][p.q], 1e-12, ("A", p.q))
        for k in range(2, p.q + 1):
            nkm1, _ = nv.gamblet_level_size(h, k - 1)
            nk, _ = nv.gamblet_level_size(h, k)
            R = coo_to_dense(*nv.gamblet_get_operator(h, 1, k), (nkm1, nk))
            check_R(R, ref["R"][k], 1e-10, ("R", k))
        u = np.zeros(n)
        assert nv.gamblet_solve(h, p.g, u) == nv.OK
        assert rel(u, u_ref) < 1e-9
    finally:
        nv.gamblet_destroy(h)


@pytest.mark.parametrize("precision", [0, 1])
def test_mass_initialised_refined_solve(precision):
    """u = M^-1,loc U with A^(q),loc U = g solved to 1e-12."""
    from paper_1503_03467_gb300 import native as nv
    p = make_problem(64, 1e4, 4)
    M = assemble_q1_mass(64)
    Aq, Minv = mass_initialised_operator(p.A, M, p.cells, p.q, 2.0)
    u_ref = Minv @ spla.spsolve(Aq.tocsc(), p.g)
    h = _setup(p, M, 2.0, _opts(precision, refine=60))
    try:
        u = np.zeros(p.ndof)
        info = nv.Info()
        assert nv.gamblet_solve(h, p.g, u, None, info) == nv.OK
        assert info.rel_residual < 1e-12
        assert rel(u, u_ref) < 1e-9
        with pytest.raises(nv.GambletError) as e:
            nv.gamblet_grad(h, np.zeros((4, 4), np.int32), np.ones(4), np.eye(4).ravel(), u, u,
                            np.zeros(4))
        assert e.value.status == nv.ERR_UNSUPPORTED
    finally:
        nv.gamblet_destroy(h)


def test_example1_with_mass_initialisation():
    """The paper's Example 1 (65 x 65 cells, q = 6) in its own setting: mass
    initialisation, localized one-pass transform against the oracle."""
    from paper_1503_03467_gb300 import native as nv
    p = make_example1(6)
    M = assemble_q1_mass(p.n)
    ref = gamblet_mass_setup(p.A, M, p.cells, p.q, 3.0, 2.0)
    u_ref, _ = gamblet_mass_solve(ref, p.g)
    h = _setup(p, M, 2.0, _opts())
    try:
        u = np.zeros(p.ndof)
        assert nv.gamblet_solve(h, p.g, u) == nv.OK
        assert rel(u, u_ref) < 1e-9
    finally:
        nv.gamblet_destroy(h)
