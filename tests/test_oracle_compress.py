"""Pins of the compression in the normalised gamblet basis (oracle)."""
import numpy as np
import pytest

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


# ---- the normalisation itself, pinned against the basis functions -------
#
# Sec. 5.1 normalises each coefficient by the energy norm of its basis
# function: psi^(1)_i / ||psi^(1)_i||_a and chi^(k)_j / ||chi^(k)_j||_a.  The
# pin builds those functions in fine coordinates without the level recursion:
# psi^(k) from the brute-force projections (Sec. 4.2, psi^(k) = A^-1 Pi_k^T
# Theta^(k)^-1), chi^(k)_j = sum_i W_ji psi^(k)_i (Sec. 4.4), energies as
# f^T A f, and the coefficients by expanding the exact level components
# u^(1) = sum_i U_i psi^(1)_i and u^(k) - u^(k-1) = sum_j w_j chi^(k)_j
# (Theorem thddwedmgugyug) in those functions.

def _brute_normalised(p):
    from oracle.brute import brute
    from oracle.hierarchy import Hierarchy
    b = brute(p.A, p.g, p.cells, p.q)
    H = Hierarchy(p.cells, p.q)
    Ad = p.A.toarray()
    c = {}
    psi1 = b["psi"][1]
    U, *_ = np.linalg.lstsq(psi1, b["uk"][1], rcond=None)
    c[1] = U * np.sqrt(np.einsum("ni,nm,mi->i", psi1, Ad, psi1))
    for k in range(2, p.q + 1):
        chi = b["psi"][k] @ H.W(k).toarray().T          # n_q x |J^(k)|
        w, *_ = np.linalg.lstsq(chi, b["uk"][k] - b["uk"][k - 1], rcond=None)
        c[k] = w * np.sqrt(np.einsum("nj,nm,mj->j", chi, Ad, chi))
    return c


def _max_dev(c, cb):
    scale = max(np.abs(v).max() for v in cb.values())
    return max(np.abs(c[k] - cb[k]).max() for k in cb) / scale


@pytest.mark.parametrize("n,C,seed", [(8, 1e2, 0), (16, 1e3, 3)])
def test_normalised_coefficients_equal_energy_norms_of_basis_functions(n, C, seed):
    p = make_problem(n, C, seed)
    s = gamblet_local_setup(p.A, p.cells, p.q, np.inf)
    c, _ = normalised_coefficients(s, p.g)
    cb = _brute_normalised(p)
    assert set(c) == set(cb)
    for k in cb:
        assert c[k].shape == cb[k].shape, k
    assert _max_dev(c, cb) < 1e-9


# plausible mistakes in the normalisation, planted in a copy of the oracle
NORM_MUTATIONS = {
    "no_detail_normalisation": ('res["w"][k] * np.sqrt(setup["B"][k].diagonal())',
                                'res["w"][k] * 1.0'),
    "detail_norm_from_diagonal_only": (
        'res["w"][k] * np.sqrt(setup["B"][k].diagonal())',
        'res["w"][k] * np.sqrt(abs(setup["W"][k]).power(2) @ setup["A"][k].diagonal())'),
    "detail_norm_squared": ('res["w"][k] * np.sqrt(setup["B"][k].diagonal())',
                            'res["w"][k] * setup["B"][k].diagonal()'),
    "coarse_norm_from_level_2": ('res["U1"] * np.sqrt(setup["A"][1].diagonal())',
                                 'res["U1"] * np.sqrt(setup["A"][2].diagonal()[:res["U1"].size])'),
    "no_coarse_normalisation": ('res["U1"] * np.sqrt(setup["A"][1].diagonal())',
                                'res["U1"] * 1.0'),
}


@pytest.mark.parametrize("name", sorted(NORM_MUTATIONS))
def test_normalisation_pin_catches_planted_mistake(name):
    import inspect
    import types
    import oracle.compress as oc
    src = inspect.getsource(oc)
    old, new = NORM_MUTATIONS[name]
    assert old in src, name
    mod = types.ModuleType("oracle.compress_mut")
    mod.__dict__["__package__"] = "oracle"
    exec(compile(src.replace(old, new), "<mutant>", "exec"), mod.__dict__)
    p = make_problem(8, 1e2, 0)
    s = gamblet_local_setup(p.A, p.cells, p.q, np.inf)
    c, _ = mod.normalised_coefficients(s, p.g)
    cb = _brute_normalised(p)
    assert _max_dev(c, cb) > 1e-6
