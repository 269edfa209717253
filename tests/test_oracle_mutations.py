"""Plant plausible mistakes in the exact oracle (on the CPU) and check that
the pins of test_oracle_pins.py catch each of them."""
import inspect
import types

import numpy as np
import pytest

import oracle.exact as ex
from oracle import direct
from oracle.brute import brute
from workloads import make_problem

MUTATIONS = {
    "sign_of_D_in_R": ("R = pibar + D.T @ W", "R = pibar - D.T @ W"),
    "pi_instead_of_pibar": ("pibar = H.pibar(k).toarray()", "pibar = H.pi(k).toarray()"),
    "transposed_B": ("B = W @ Ak @ W.T", "B = W @ Ak.T @ W.T + 1e-3 * np.eye(W.shape[0])"),
    "g_restricted_by_pibar": ("gkm1 = R @ gk", "gkm1 = pibar @ gk"),
    "dropped_detail_term": ("comps[k - 1] = P[k] @ (out[\"W\"][k].T @ out[\"w\"][k])",
                            "comps[k - 1] = 0.0 * P[k][:, 0]"),
    "wrong_D_rhs": ("D = -sla.cho_solve(cf, W @ Ak @ pibar.T)",
                    "D = -sla.cho_solve(cf, W @ pibar.T)"),
}


def _mutated(name):
    src = inspect.getsource(ex)
    old, new = MUTATIONS[name]
    assert old in src, name
    mod = types.ModuleType("oracle.exact_mut")
    mod.__dict__["__package__"] = "oracle"
    exec(compile(src.replace(old, new), "<mutant>", "exec"), mod.__dict__)
    return mod.gamblet_exact


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_mutation(name):
    p = make_problem(8, 1e2, 1)
    ud, _ = direct.solve(p.A, p.g)
    b = brute(p.A, p.g, p.cells, p.q)
    r = _mutated(name)(p.A, p.g, p.cells, p.q)
    sum_ok = np.linalg.norm(r["u"] - ud) / np.linalg.norm(ud) < 1e-12
    comps_ok = np.linalg.norm(r["comps"] - b["comps"]) / np.linalg.norm(b["comps"]) < 1e-11
    A_ok = all(np.linalg.norm(r["A"][k] - b["Ak"][k]) / np.linalg.norm(b["Ak"][k]) < 1e-11
               for k in range(1, p.q + 1))
    assert not (sum_ok and comps_ok and A_ok)


def test_unmutated_passes_same_checks():
    p = make_problem(8, 1e2, 1)
    ud, _ = direct.solve(p.A, p.g)
    b = brute(p.A, p.g, p.cells, p.q)
    r = ex.gamblet_exact(p.A, p.g, p.cells, p.q)
    assert np.linalg.norm(r["u"] - ud) / np.linalg.norm(ud) < 1e-12
    assert np.linalg.norm(r["comps"] - b["comps"]) / np.linalg.norm(b["comps"]) < 1e-11


MASS_MUTATIONS = {
    "missing_right_factor": ("Aq = sp.csr_matrix(Minv.T @ sp.csr_matrix(A) @ Minv)",
                             "Aq = sp.csr_matrix(Minv.T @ sp.csr_matrix(A))"),
    "rhs_not_unit": ("e = (idx == i).astype(np.float64)", "e = np.ones(len(idx))"),
    "output_not_mapped": ("return setup[\"Minv\"] @ U, U", "return U, U"),
}


@pytest.mark.parametrize("name", sorted(MASS_MUTATIONS))
def test_mass_pins_catch_mutation(name):
    """The direct solve of A u = M g (exact inverse) or the patch exactness of
    the localized inverse catches each planted mistake."""
    import scipy.sparse.linalg as spla
    import oracle.massinit as mi
    from workloads import assemble_q1_mass
    src = inspect.getsource(mi)
    old, new = MASS_MUTATIONS[name]
    assert old in src, name
    mod = types.ModuleType("oracle.massinit_mut")
    mod.__dict__["__package__"] = "oracle"
    exec(compile(src.replace(old, new), "<mutant>", "exec"), mod.__dict__)
    p = make_problem(8, 1e2, 2)
    M = assemble_q1_mass(8)
    u_ref = spla.spsolve(p.A.tocsc(), M @ p.g)
    setup = mod.gamblet_mass_setup(p.A, M, p.cells, p.q, np.inf, np.inf)
    u, _ = mod.gamblet_mass_solve(setup, p.g)
    exact_ok = np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref) < 1e-12
    Mi = mod.localized_mass_inverse(M, p.cells, p.q, 1.0)
    P = (M @ Mi).toarray()
    patch_ok = all(np.allclose(P[Mi[:, i].nonzero()[0], i],
                               (Mi[:, i].nonzero()[0] == i).astype(float), atol=1e-12)
                   for i in range(0, M.shape[0], 7))
    assert not (exact_ok and patch_ok)
