"""Pins of the mass-matrix initialisation (Algorithm 1 lines 1-5; Algorithm
2 lines 2a-5 with Definition deflocinvm) in the oracle."""
import numpy as np
import scipy.sparse.linalg as spla

from oracle.local import gamblet_local_solve
from oracle.massinit import (gamblet_mass_setup, gamblet_mass_solve, localized_mass_inverse,
                             mass_initialised_operator)
from workloads import M_REF, assemble_q1_mass, make_problem


def test_mass_matrix_integrates_the_nodal_basis():
    # element: the integrals of products of bilinear hat functions on the unit
    # square (corners counter-clockwise), whose total is the area
    assert np.isclose(M_REF.sum(), 1.0)
    x = np.array([0.0, 1.0, 1.0, 0.0])  # nodal values of the function x
    assert np.isclose(x @ M_REF @ x, 1.0 / 3.0)      # integral of x^2
    assert np.isclose(np.ones(4) @ M_REF @ x, 0.5)   # integral of x
    n = 16
    M = assemble_q1_mass(n).toarray()
    assert np.allclose(M, M.T)
    # an interior node away from the boundary: integral of its hat = h^2
    i = 7 * (n - 1) + 7
    assert np.isclose(M[i].sum(), 1.0 / n ** 2)
    assert np.all(np.linalg.eigvalsh(M) > 0)


def test_exact_initialisation_solves_the_fem_system_with_mass_load():
    p = make_problem(16, 1e2, 0)
    M = assemble_q1_mass(16)
    setup = gamblet_mass_setup(p.A, M, p.cells, p.q, np.inf, np.inf)
    u, _ = gamblet_mass_solve(setup, p.g)
    u_ref = spla.spsolve(p.A.tocsc(), M @ p.g)
    assert np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref) < 1e-12


def test_localized_inverse_is_exact_on_its_patch_and_decays():
    p = make_problem(16, 1e2, 1)
    M = assemble_q1_mass(16)
    Mexact = np.linalg.inv(M.toarray())
    errs = []
    for rq in (1.0, 2.0, 3.0):
        Mi = localized_mass_inverse(M, p.cells, p.q, rq)
        P = (M @ Mi).toarray()
        for i in (0, 40, 120):
            sup = Mi[:, i].nonzero()[0]
            e = np.zeros(len(sup))
            e[sup == i] = 1.0
            assert np.allclose(P[sup, i], e, atol=1e-12)   # Definition deflocinvm
        errs.append(np.linalg.norm(Mi.toarray() - Mexact) / np.linalg.norm(Mexact))
    assert errs[0] > 2 * errs[1] > 4 * errs[2]


def test_mass_initialised_operator_is_spd_and_hierarchy_exact():
    p = make_problem(16, 1e3, 2)
    M = assemble_q1_mass(16)
    Aq, Minv = mass_initialised_operator(p.A, M, p.cells, p.q, 2.0)
    ev = np.linalg.eigvalsh(Aq.toarray())
    assert ev.min() > 0
    # with unbounded patches the transform of A^(q) is exact (Theorem
    # thmgugyug2): the one-pass solve equals the direct solve of A^(q) U = g
    setup = gamblet_mass_setup(p.A, M, p.cells, p.q, np.inf, 2.0)
    U = gamblet_local_solve(setup, p.g)["u"]
    U_ref = np.linalg.solve(Aq.toarray(), p.g)
    assert np.linalg.norm(U - U_ref) / np.linalg.norm(U_ref) < 1e-10
