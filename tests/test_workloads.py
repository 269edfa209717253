"""Input generators: Q1 assembly, coefficient family, Example ex1 contrast."""
from fractions import Fraction
import os

import numpy as np
import pytest

from workloads import (assemble_q1, example1_coefficient, interior_cells,
                       make_problem, rough_log_coefficient)

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    out = {}
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, v = line.split()
        out[k] = v
    return out


def test_example1_contrast_matches_paper():
    gold = _read_golden("example1_contrast.txt")
    a = example1_coefficient(int(gold["q"]))
    c = a.max() / a.min()
    assert abs(c - float(gold["contrast"])) <= float(gold["rounding"])


def test_q1_stencil_constant_coefficient():
    gold = {k: float(Fraction(v)) for k, v in _read_golden("q1_stencil.txt").items()}
    n = 8
    A = assemble_q1(np.ones((n, n))).toarray()
    m = n - 1
    i = 3 * m + 3  # interior node (4, 4)
    assert A[i, i] == pytest.approx(gold["center"], abs=1e-15)
    for d in (1, -1, m, -m):
        assert A[i, i + d] == pytest.approx(gold["edge"], abs=1e-15)
    for d in (m + 1, m - 1, -m + 1, -m - 1):
        assert A[i, i + d] == pytest.approx(gold["diagonal"], abs=1e-15)
    assert np.count_nonzero(A[i]) == 9
    # symmetric positive definite
    assert np.allclose(A, A.T)
    assert np.linalg.eigvalsh(A).min() > 0


def test_q1_energy_of_linear_function_and_cellwise_scaling():
    # u(x,y) = x on the full grid: energy over the whole square of a*|grad u|^2
    # equals sum_c a_c h^2 * (1/h)^2 = sum_c a_c (boundary values included)
    n = 8
    rng = np.random.default_rng(3)
    a = np.exp(rng.uniform(-1, 1, (n, n)))
    from workloads.rough import K_REF
    # element check: K_REF applied to nodal values of x on a unit cell
    ux = np.array([0.0, 1.0, 1.0, 0.0])
    assert ux @ K_REF @ ux == pytest.approx(1.0)
    uy = np.array([0.0, 0.0, 1.0, 1.0])
    assert uy @ K_REF @ uy == pytest.approx(1.0)
    assert np.allclose(K_REF @ np.ones(4), 0)
    # assembled matrix scales linearly with a per cell
    A1 = assemble_q1(a).toarray()
    A2 = assemble_q1(2 * a).toarray()
    assert np.allclose(A2, 2 * A1)


def test_rough_coefficient_bounds_and_determinism():
    n, C = 64, 1e4
    la = rough_log_coefficient(n, 6, C, np.random.default_rng(0))
    assert la.max() - la.min() <= np.log(C) + 1e-12
    assert np.abs(la).max() <= 0.5 * np.log(C) + 1e-12
    la2 = rough_log_coefficient(n, 6, C, np.random.default_rng(0))
    assert np.array_equal(la, la2)
    # finest scale layer is constant on 1x1 dyadic squares of side 2^-6
    p = make_problem(32, 100, 0)
    assert p.A.shape == (961, 961)
    assert p.A.nnz == (3 * 31 - 2) ** 2
    assert p.cells.shape == (961, 2)
    assert interior_cells(4).tolist() == [[1, 1], [2, 1], [3, 1], [1, 2], [2, 2],
                                          [3, 2], [1, 3], [2, 3], [3, 3]]


def test_batch_workload_draw_protocol():
    from workloads import make_batch, make_batch_problem
    # the documented draw order: side index, log10 contrast, then the fields
    rng = np.random.default_rng(5)
    n = (8, 16, 32)[int(rng.integers(3))]
    C = 10.0 ** rng.uniform(2.0, 6.0)
    la = rough_log_coefficient(n, int(np.log2(n)), C, rng)
    g = rng.standard_normal((n - 1) ** 2)
    p = make_batch_problem(5, sides=(8, 16, 32))
    assert p.n == n and p.contrast == C
    assert np.array_equal(p.log_a, la) and np.array_equal(p.g, g)
    assert p.log_a.max() - p.log_a.min() <= np.log(C) + 1e-12
    probs = make_batch(12, first_seed=1, sides=(8, 16, 32))
    assert [q.n for q in probs] == [make_batch_problem(s, sides=(8, 16, 32)).n
                                    for s in range(1, 13)]
    assert all(1e2 <= q.contrast <= 1e6 for q in probs)
    assert all(q.A.shape == ((q.n - 1) ** 2,) * 2 for q in probs)


def test_example1_problem_layout():
    from workloads import assemble_q1_mass, make_example1
    p = make_example1(4)
    assert p.n == 17 and p.q == 4 and p.A.shape == (256, 256)
    assert p.cells.min() == 0 and p.cells.max() == 15          # 2^q x 2^q lattice, all cells used
    assert len({(int(x), int(y)) for x, y in p.cells}) == 256
    assert assemble_q1_mass(17).shape == (256, 256)
    assert p.g.shape == (256,)
