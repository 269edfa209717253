"""Pins of the three-dimensional inputs and of the oracle at d = 3.

The paper states the method for a domain of R^d (Sec. 4; the complexity of
Sec. 5.4 is given in d).  These checks fix the 3-D trilinear operator by
quadrature, the 3-D hierarchy by its identities and by brute-force distance,
Algorithm 1 by the direct solve and by the brute-force projections of Sec.
4.2, and Algorithm 2 by its limit rho -> infinity, its local energy
minimisation and the decay of the localization error.
"""
import itertools

import numpy as np
import pytest

from oracle import direct
from oracle.brute import brute
from oracle.exact import gamblet_exact
from oracle.hierarchy import Hierarchy
from oracle.local import gamblet_local_setup, gamblet_local_solve
from workloads import K_REF3, assemble_q1_3d, interior_cells3, make_problem3


def rel(a, b):
    a = a.toarray() if hasattr(a, "toarray") else np.asarray(a)
    b = b.toarray() if hasattr(b, "toarray") else np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _trilinear_grad(c, x):
    """Gradient of the trilinear shape function of corner c (bits bx, by, bz)
    at the point x of the unit cube."""
    b = [(c >> a) & 1 for a in range(3)]
    f = [x[a] if b[a] else 1.0 - x[a] for a in range(3)]
    df = [1.0 if b[a] else -1.0 for a in range(3)]
    return np.array([df[0] * f[1] * f[2], f[0] * df[1] * f[2], f[0] * f[1] * df[2]])


def _gauss_points():
    # two-point Gauss-Legendre rule on [0, 1]: exact for degree 3 per variable
    t = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])
    return [(np.array(p), 0.125) for p in itertools.product(t, t, t)]


# --------------------------------------------------------------- inputs
def test_trilinear_stiffness_equals_quadrature():
    K = np.zeros((8, 8))
    for x, w in _gauss_points():
        G = np.array([_trilinear_grad(c, x) for c in range(8)])
        K += w * G @ G.T
    assert np.abs(K - K_REF3).max() < 1e-15
    assert np.abs(K_REF3.sum(axis=1)).max() < 1e-15


def test_q1_3d_stencil_constant_coefficient():
    # Interior row with a = 1, h = 1/n: a node is a corner of 8 cubes; the
    # coupling to a node differing in b coordinates collects 2^(3-b) cubes:
    # centre 8 h/3, face neighbours 0, edge diagonals 2 h (-1/12) = -h/6,
    # body diagonals -h/12; the row sums to zero.
    n = 8
    h = 1.0 / n
    A = assemble_q1_3d(np.ones((n, n, n))).toarray()
    m = n - 1
    i = (3 * m + 3) * m + 3
    expect = {0: 8 * h / 3, 1: 0.0, 2: -h / 6, 3: -h / 12}
    for dz, dy, dx in itertools.product((-1, 0, 1), repeat=3):
        j = i + (dz * m + dy) * m + dx
        b = abs(dx) + abs(dy) + abs(dz)
        assert A[i, j] == pytest.approx(expect[b], abs=1e-15)
    assert abs(A[i].sum()) < 1e-15
    assert np.allclose(A, A.T)
    assert np.linalg.eigvalsh(A).min() > 0


def test_q1_3d_energy_by_quadrature():
    # u^T A u = sum_c a_c int_c |grad u_h|^2 for the trilinear interpolant
    # u_h (zero on the boundary), integrated cell by cell by quadrature
    n = 4
    h = 1.0 / n
    rng = np.random.default_rng(5)
    a = np.exp(rng.uniform(-1.5, 1.5, (n, n, n)))
    A = assemble_q1_3d(a)
    u = rng.standard_normal((n - 1) ** 3)
    full = np.zeros((n + 1, n + 1, n + 1))
    full[1:n, 1:n, 1:n] = u.reshape(n - 1, n - 1, n - 1)   # [iz, iy, ix]
    energy = 0.0
    pts = _gauss_points()
    for cz, cy, cx in itertools.product(range(n), repeat=3):
        vals = [full[cz + ((c >> 2) & 1), cy + ((c >> 1) & 1), cx + (c & 1)] for c in range(8)]
        for x, w in pts:
            gr = sum(v * _trilinear_grad(c, x) for c, v in enumerate(vals)) / h
            energy += a[cz, cy, cx] * w * h ** 3 * (gr @ gr)
    assert u @ (A @ u) == pytest.approx(energy, rel=1e-13)


def test_q1_3d_reproduces_linear_functions():
    # constant a: the discrete operator annihilates u = x at nodes whose
    # stencil does not touch the boundary
    n = 8
    A = assemble_q1_3d(np.full((n, n, n), 2.5))
    c = interior_cells3(n)
    r = A @ c[:, 0].astype(float)
    inner = np.all((c >= 2) & (c <= n - 2), axis=1)
    assert np.abs(r[inner]).max() < 1e-13


def test_rough_3d_coefficient_bounds_and_determinism():
    p = make_problem3(16, 1e3, 2)
    assert p.A.shape == (15 ** 3, 15 ** 3)
    assert p.cells.shape == (15 ** 3, 3)
    assert np.exp(p.log_a.max() - p.log_a.min()) <= 1e3 * (1 + 1e-12)
    q = make_problem3(16, 1e3, 2)
    assert np.array_equal(p.g, q.g) and np.array_equal(p.log_a, q.log_a)


# --------------------------------------------------------------- hierarchy
@pytest.mark.parametrize("n", [4, 8])
def test_pi_w_identities_3d(n):
    p = make_problem3(n, 10, 1)
    H = Hierarchy(p.cells, p.q)
    assert [H.n(k) for k in range(1, p.q + 1)] == [8 ** k for k in range(1, p.q)] + [(n - 1) ** 3]
    for k in range(2, p.q + 1):
        P = H.pi(k).toarray()
        Pb = H.pibar(k).toarray()
        W2 = H.W(k, "const2").toarray()
        assert np.allclose(P @ Pb.T, np.eye(H.n(k - 1)))
        assert W2.shape[0] == H.n(k) - H.n(k - 1)
        assert np.abs(P @ W2.T).max() < 1e-14
        assert np.linalg.matrix_rank(np.vstack([W2, P])) == H.n(k)
        assert np.allclose(W2 @ W2.T, np.eye(W2.shape[0]), atol=1e-14)
    # fine level: a parent holds 8, 4, 2 or 1 interior nodes
    m = np.bincount(H.levels[p.q].parent)
    assert sorted(set(m.tolist())) == [1, 2, 4, 8]
    # child order: slot (x & 1) + 2 (y & 1) + 4 (z & 1) increases within a parent
    c = H.levels[p.q].cells
    for ch in H.children(p.q):
        slot = (c[ch, 0] & 1) + 2 * (c[ch, 1] & 1) + 4 * (c[ch, 2] & 1)
        assert np.all(np.diff(slot) > 0)


def test_neighbourhood_counts_3d():
    # interior cell, rho = 1: the 27 cubes of the box plus, for the
    # Euclidean distance between closed cubes, the 54 at offset 2 along one
    # axis (distance exactly 1); rho = 2 brute-forced from the definition
    p = make_problem3(32, 10, 0)
    H = Hierarchy(p.cells, p.q)
    k = 4
    c = H.levels[k].cells
    i = int(np.nonzero((c == 8).all(axis=1))[0][0])
    assert len(H.neighbours(k, 1, "cheb")[i]) == 27
    assert len(H.neighbours(k, 1, "euclid")[i]) == 81

    def dist(a, b):
        e = np.maximum(np.abs(a - b) - 1, 0)
        return np.sqrt((e * e).sum())
    expect = [j for j in range(len(c)) if dist(c[i], c[j]) <= 2 + 1e-12]
    assert sorted(H.neighbours(k, 2, "euclid")[i].tolist()) == expect


# --------------------------------------------------------------- Algorithm 1
@pytest.fixture(scope="module")
def e8():
    p = make_problem3(8, 100, 0)
    return p, gamblet_exact(p.A, p.g, p.cells, p.q)


def test_components_sum_to_direct_solve_3d(e8):
    p, r = e8
    ud, _ = direct.solve(p.A, p.g)
    assert rel(r["u"], ud) < 1e-12


def test_components_a_orthogonal_3d(e8):
    p, r = e8
    C = r["comps"]
    G = C @ (p.A @ C.T)
    nrm = np.sqrt(np.diag(G))
    off = G - np.diag(np.diag(G))
    assert np.all(np.abs(off) <= 1e-12 * np.outer(nrm, nrm) + 1e-300)


@pytest.mark.parametrize("n,seed", [(4, 0), (8, 3)])
def test_brute_force_3d(n, seed):
    p = make_problem3(n, 1e3, seed)
    r = gamblet_exact(p.A, p.g, p.cells, p.q)
    b = brute(p.A, p.g, p.cells, p.q)
    assert rel(r["comps"], b["comps"]) < 1e-11
    for k in range(1, p.q + 1):
        assert rel(r["A"][k], b["Ak"][k]) < 1e-11
    for k in range(2, p.q + 1):
        assert rel(r["R"][k], b["R"][k]) < 1e-11


# --------------------------------------------------------------- Algorithm 2
def test_unbounded_radius_equals_exact_3d(e8):
    p, ex = e8
    s = gamblet_local_setup(p.A, p.cells, p.q, rho=1e9)
    r = gamblet_local_solve(s, p.g, return_components=True)
    for k in range(2, p.q + 1):
        assert rel(s["R"][k], ex["R"][k]) < 1e-12
        assert rel(s["A"][k - 1], ex["A"][k - 1]) < 1e-12
    assert rel(r["u"], ex["u"]) < 1e-12


def test_patch_solve_is_local_constrained_minimiser_3d(e8):
    # R row i minimises the level-k energy over coefficients supported on the
    # children of i^rho subject to the level-(k-1) constraints on i^rho
    # (a KKT system on that support, independent of W)
    p, _ = e8
    s = gamblet_local_setup(p.A, p.cells, p.q, rho=1, rule="cheb")
    H = s["hier"]
    k = p.q
    Ak = s["A"][k].toarray()
    P = H.pi(k).toarray()
    nb = H.neighbours(k - 1, 1, "cheb")
    R = s["R"][k].toarray()
    for i in (0, 21, H.n(k - 1) - 1):
        N = nb[i]
        S = np.nonzero(P[N].sum(axis=0) > 0)[0]
        PN = P[np.ix_(N, S)]
        K = np.block([[Ak[np.ix_(S, S)], PN.T], [PN, np.zeros((len(N), len(N)))]])
        e = np.zeros(len(S) + len(N))
        e[len(S) + int(np.nonzero(N == i)[0][0])] = 1.0
        c = np.linalg.solve(K, e)[:len(S)]
        row = np.zeros(H.n(k))
        row[S] = c
        assert np.abs(R[i] - row).max() < 1e-11 * np.abs(row).max()


def test_localization_error_decays_with_radius_3d():
    # Sec. 4.10 Theorem thmerrorpropagation: exponential decay in rho
    p = make_problem3(16, 1e3, 0)
    ud, _ = direct.solve(p.A, p.g)
    errs = []
    for rho in (1, 2):
        s = gamblet_local_setup(p.A, p.cells, p.q, rho=rho, rule="cheb")
        u = gamblet_local_solve(s, p.g)["u"]
        errs.append(np.linalg.norm(u - ud) / np.linalg.norm(ud))
    assert errs[0] < 0.8
    assert errs[1] < 0.4 * errs[0]
