"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own formulas: closed forms
from other theorems, brute-force projections without the level recursion,
invariants, and the direct sparse solve.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import direct
from oracle.brute import brute, measurement
from oracle.exact import gamblet_exact
from oracle.hierarchy import Hierarchy, helmert_u, helmert_ubar
from workloads import make_problem


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


# --------------------------------------------------------------- hierarchy
@pytest.mark.parametrize("n", [2, 3, 4, 5, 8])
def test_helmert_rows_orthogonal_last_row_ones(n):
    # Sec. 4.6, Lemma const0
    U = helmert_u(n)
    G = U @ U.T
    assert np.allclose(G, np.diag(np.diag(G)))
    assert np.allclose(U[-1], 1.0)
    Ub = helmert_ubar(n)
    assert np.allclose(Ub @ Ub.T, np.eye(n), atol=1e-15)


@pytest.mark.parametrize("n", [4, 8, 16])
def test_pi_w_identities(n):
    p = make_problem(n, 10, 1)
    H = Hierarchy(p.cells, p.q)
    for k in range(2, p.q + 1):
        P = H.pi(k).toarray()
        Pb = H.pibar(k).toarray()
        W2 = H.W(k, "const2").toarray()
        W1 = H.W(k, "const1").toarray()
        assert np.allclose(P @ Pb.T, np.eye(H.n(k - 1)))
        # Lemma lemwk: Im W^T = Ker pi, |J| = |I^(k)| - |I^(k-1)|
        assert W2.shape[0] == H.n(k) - H.n(k - 1)
        assert np.abs(P @ W2.T).max() < 1e-14
        assert np.abs(P @ W1.T).max() < 1e-14
        assert np.linalg.matrix_rank(np.vstack([W2, P])) == H.n(k)
        # Construction const2: W W^T = J (identity)
        assert np.allclose(W2 @ W2.T, np.eye(W2.shape[0]), atol=1e-14)


def test_level_sizes_and_uneven_children():
    p = make_problem(32, 10, 0)
    H = Hierarchy(p.cells, p.q)
    assert [H.n(k) for k in range(1, 6)] == [4, 16, 64, 256, 961]
    m = np.bincount(H.levels[5].parent)
    assert sorted(set(m.tolist())) == [1, 2, 4]
    assert np.count_nonzero(m == 1) == 1


def test_neighbourhood_counts():
    # rho = 3 in the interior: 61 parents (Euclidean distance between closed
    # squares), 49 with the Chebyshev box rule
    p = make_problem(64, 10, 0)
    H = Hierarchy(p.cells, p.q)
    k = 5
    c = H.levels[k].cells
    nb_e = H.neighbours(k, 3, "euclid")
    nb_c = H.neighbours(k, 3, "cheb")
    i = int(np.nonzero((c[:, 0] == 16) & (c[:, 1] == 16))[0][0])
    assert len(nb_e[i]) == 61
    assert len(nb_c[i]) == 49
    # brute-force the definition with geometric squares
    def dist(a, b):
        ex = max(abs(a[0] - b[0]) - 1, 0)
        ey = max(abs(a[1] - b[1]) - 1, 0)
        return np.hypot(ex, ey)
    expect = [j for j in range(len(c)) if dist(c[i], c[j]) <= 3 + 1e-12]
    assert sorted(nb_e[i].tolist()) == expect


# --------------------------------------------------------------- Algorithm 1
@pytest.fixture(scope="module")
def c1():
    p = make_problem(32, 100, 0)
    return p, gamblet_exact(p.A, p.g, p.cells, p.q)


def test_components_sum_to_direct_solve(c1):
    # Theorem thmgugyug2 / Algorithm 1 final line
    p, r = c1
    ud, _ = direct.solve(p.A, p.g)
    assert rel(r["u"], ud) < 1e-12


def test_components_a_orthogonal(c1):
    # Theorem thmgugyug2 (1): orthogonal direct sum w.r.t. <.,.>_a
    p, r = c1
    C = r["comps"]
    G = C @ (p.A @ C.T)
    nrm = np.sqrt(np.diag(G))
    off = G - np.diag(np.diag(G))
    assert np.abs(off).max() <= 1e-12 * nrm.max() ** 2
    assert np.all(np.abs(off) <= 1e-12 * np.outer(nrm, nrm) + 1e-300)


def test_restriction_identities_and_closed_form(c1):
    # Theorem thmhggfees5: pi R^T = I and R = A^(k-1) pi Theta^(k);
    # with Theta^(k) = Pi_k A^-1 Pi_k^T this is
    # R^(k-1,k) = A^(k-1) pi^(k-1,k) Pi_k A^-1 Pi_k^T.
    p, r = c1
    H = r["hier"]
    Ainv = np.linalg.inv(p.A.toarray())
    for k in range(2, p.q + 1):
        P = H.pi(k).toarray()
        R = r["R"][k]
        assert np.abs(P @ R.T - np.eye(H.n(k - 1))).max() < 1e-13
        Pk = measurement(p.cells, p.q, k)
        Theta = Pk @ Ainv @ Pk.T
        Rc = r["A"][k - 1] @ P @ Theta
        assert rel(R, Rc) < 1e-10
        # Theorem thmhggfees5: R^T b minimises c^T A c subject to pi c = b
        # (KKT with Lagrange multipliers, solved as one dense system)
        Ak = r["A"][k]
        nk, nkm1 = H.n(k), H.n(k - 1)
        K = np.block([[Ak, P.T], [P, np.zeros((nkm1, nkm1))]])
        rhs = np.vstack([np.zeros((nk, nkm1)), np.eye(nkm1)])
        sol = np.linalg.solve(K, rhs)[:nk]
        assert rel(R.T, sol) < 1e-9


def test_stiffness_closed_form(c1):
    # A^(k) = Theta^(k)^-1 (Sec. 4.5) with Theta^(k) = Pi_k A^-1 Pi_k^T
    p, r = c1
    Ainv = np.linalg.inv(p.A.toarray())
    for k in range(1, p.q + 1):
        Pk = measurement(p.cells, p.q, k)
        Ak = np.linalg.inv(Pk @ Ainv @ Pk.T)
        assert rel(r["A"][k], Ak) < 1e-9


def test_w_construction_independence():
    # A^(k), R and the components do not depend on the choice of W
    # (Lemma lemwk: only Im W^T = Ker pi matters)
    p = make_problem(16, 100, 4)
    r2 = gamblet_exact(p.A, p.g, p.cells, p.q, "const2")
    r1 = gamblet_exact(p.A, p.g, p.cells, p.q, "const1")
    for k in range(1, p.q + 1):
        assert rel(r1["A"][k], r2["A"][k]) < 1e-11
    for k in range(2, p.q + 1):
        assert rel(r1["R"][k], r2["R"][k]) < 1e-11
    assert rel(r1["comps"], r2["comps"]) < 1e-11
    # ... whereas B^(k) does depend on it
    assert rel(r1["B"][p.q], r2["B"][p.q]) > 1e-3


@pytest.mark.parametrize("n,seed", [(4, 0), (8, 1), (8, 2)])
def test_brute_force_tiny_grids(n, seed):
    p = make_problem(n, 1e3, seed)
    r = gamblet_exact(p.A, p.g, p.cells, p.q)
    b = brute(p.A, p.g, p.cells, p.q)
    assert rel(r["comps"], b["comps"]) < 1e-11
    for k in range(1, p.q + 1):
        assert rel(r["A"][k], b["Ak"][k]) < 1e-11
    for k in range(2, p.q + 1):
        assert rel(r["R"][k], b["R"][k]) < 1e-11


def test_brute_force_projection_is_a_orthogonal():
    # independent sanity of the brute-force itself: u - u^(k) is A-orthogonal
    # to V^(k) = span psi^(k)
    p = make_problem(8, 1e2, 5)
    b = brute(p.A, p.g, p.cells, p.q)
    A = p.A.toarray()
    for k in range(1, p.q + 1):
        assert np.abs(b["psi"][k].T @ A @ (b["u"] - b["uk"][k])).max() < 1e-10


def test_condition_numbers_bounded_as_q_grows():
    # Sec. 4.8 Theorem thmodhehiudhehd: cond(B^(k)) bounded independently of
    # the level and of q at fixed contrast, while cond(A^(q)) grows like 4^q.
    conds = {}
    condA = {}
    for n in (8, 16, 32, 64):
        p = make_problem(n, 100, 0)
        r = gamblet_exact(p.A, p.g, p.cells, p.q)
        ev = [np.linalg.eigvalsh(r["B"][k]) for k in range(2, p.q + 1)]
        conds[n] = max(e[-1] / e[0] for e in ev)
        ea = np.linalg.eigvalsh(p.A.toarray())
        condA[n] = ea[-1] / ea[0]
    assert conds[64] < 3 * conds[16]
    assert condA[64] > 30 * condA[8]
    assert max(conds.values()) < 200


def test_energy_error_of_level_approximation_decays():
    # Theorem thmgugyug0: |u - u^(k)|_a <= C H_k |g|_L2 with H_k = 2^-k, and
    # the error is zero at k = q (Sec. 5.2, Example after Algorithm 1).  A
    # smooth source (Example ex1's g, load vector h^2 g(z_i)) makes |u|_a
    # O(1), so the relative energy error must fall by about H = 1/2 per level.
    p = make_problem(64, 10, 2)
    n = p.n
    iy, ix = np.meshgrid(np.arange(1, n), np.arange(1, n), indexing="ij")
    z1 = (ix / n).ravel()
    z2 = (iy / n).ravel()
    g = (np.cos(3 * z1 + z2) + np.sin(3 * z2) + np.sin(7 * z1 - 5 * z2)) / n ** 2
    r = gamblet_exact(p.A, g, p.cells, p.q)
    A = p.A
    u = r["u"]
    cum = np.cumsum(r["comps"], axis=0)
    err = [np.sqrt((u - cum[k]) @ (A @ (u - cum[k])) / (u @ (A @ u)))
           for k in range(p.q)]
    assert err[-1] < 1e-12
    for k in range(p.q - 2):
        assert err[k + 1] < 0.55 * err[k]


def test_direct_solver_residual():
    p = make_problem(64, 1e4, 3)
    u, _ = direct.solve(p.A, p.g)
    r = direct.residual_ext(p.A, u, p.g)
    assert float(np.linalg.norm(np.asarray(r, dtype=np.float64))) < 1e-13 * np.linalg.norm(p.g)
    ud = np.linalg.solve(p.A.toarray(), p.g)
    assert rel(u, ud) < 1e-9
