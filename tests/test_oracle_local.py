"""Pins of the localized oracle (Algorithm 2, Definition defb)."""
import numpy as np
import pytest

from oracle import direct
from oracle.exact import gamblet_exact
from oracle.local import gamblet_local_setup, gamblet_local_solve
from workloads import make_problem


def rel(a, b):
    a = a.toarray() if hasattr(a, "toarray") else np.asarray(a)
    b = b.toarray() if hasattr(b, "toarray") else np.asarray(b)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def p16():
    return make_problem(16, 1e3, 6)


def test_unbounded_radius_equals_exact(p16):
    p = p16
    ex = gamblet_exact(p.A, p.g, p.cells, p.q)
    s = gamblet_local_setup(p.A, p.cells, p.q, rho=1e9)
    r = gamblet_local_solve(s, p.g, return_components=True)
    for k in range(2, p.q + 1):
        assert rel(s["R"][k], ex["R"][k]) < 1e-12
        assert rel(s["A"][k - 1], ex["A"][k - 1]) < 1e-12
    assert rel(r["u"], ex["u"]) < 1e-12
    assert rel(r["comps"], ex["comps"]) < 1e-11


def test_patch_solve_is_local_constrained_minimiser(p16):
    # Remark rmklocalgfast (2): psi^(k-1),loc_i minimises the energy over
    # span{psi^(k),loc_l : l^(k-1) in i^rho} subject to the level-(k-1)
    # constraints on i^rho; in level-k coefficients that is a KKT system on
    # the children S of i^rho, independent of W.
    p = p16
    s = gamblet_local_setup(p.A, p.cells, p.q, rho=1)
    H = s["hier"]
    for k in (p.q, p.q - 1):
        Ak = s["A"][k].toarray()
        P = H.pi(k).toarray()
        nb = H.neighbours(k - 1, 1)
        R = s["R"][k].toarray()
        for i in (0, 5, H.n(k - 1) // 2):
            N = nb[i]
            S = np.nonzero(P[N].sum(axis=0) > 0)[0]
            PN = P[np.ix_(N, S)]
            K = np.block([[Ak[np.ix_(S, S)], PN.T],
                          [PN, np.zeros((len(N), len(N)))]])
            e = np.zeros(len(S) + len(N))
            e[len(S) + int(np.nonzero(N == i)[0][0])] = 1.0
            c = np.linalg.solve(K, e)[:len(S)]
            row = np.zeros(H.n(k))
            row[S] = c
            assert np.abs(R[i] - row).max() < 1e-11 * np.abs(row).max()


def test_coarse_operators_symmetric_and_restriction_identity(p16):
    p = p16
    s = gamblet_local_setup(p.A, p.cells, p.q, rho=2)
    H = s["hier"]
    for k in range(2, p.q + 1):
        Ak = s["A"][k - 1]
        assert abs(Ak - Ak.T).max() < 1e-12 * abs(Ak).max()
        P = H.pi(k)
        assert abs(P @ s["R"][k].T - np.eye(H.n(k - 1))).max() < 1e-12


def test_localization_error_decays_with_radius():
    # Sec. 4.10 Theorem thmerrorpropagation and Sec. 5.4 Theorem tmdiscrete:
    # the error decays exponentially in the localization radius
    p = make_problem(32, 1e4, 0)
    ud, _ = direct.solve(p.A, p.g)
    errs = []
    for rho in (1, 2, 3):
        s = gamblet_local_setup(p.A, p.cells, p.q, rho=rho)
        u = gamblet_local_solve(s, p.g)["u"]
        errs.append(np.linalg.norm(u - ud) / np.linalg.norm(ud))
    assert errs[0] < 0.5
    assert errs[1] < 0.3 * errs[0]
    assert errs[2] < 0.3 * errs[1]
