"""GPU parity of the exact (non-localized) transform, Algorithm 1, against the
CPU oracle: every level operator and component, float64, 1e-10 relative."""
import numpy as np
import pytest

from oracle import direct
from oracle.exact import gamblet_exact
from workloads import make_problem

from gpu_util import check_R, check_op, coo_to_dense, csr_arrays, drop_nodes, rel

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _run_exact(A, g, cells, q):
    from paper_1503_03467_gb300 import native as nv
    rp, ci, va = csr_arrays(A)
    o = nv.gamblet_default_opts()
    o.rho = 0.0
    o.refine_max_iter = 0
    h = nv.gamblet_setup(rp, ci, va, q, cells, o)
    try:
        n = A.shape[0]
        u = np.zeros(n)
        comps = np.zeros((q, n))
        info = nv.Info()
        st = nv.gamblet_solve(h, g, u, comps, info)
        assert st == nv.OK
        ops = {}
        for k in range(1, q + 1):
            nk, _ = nv.gamblet_level_size(h, k)
            ops[("A", k)] = coo_to_dense(*nv.gamblet_get_operator(h, 0, k), (nk, nk))
            if k >= 2:
                nkm1, _ = nv.gamblet_level_size(h, k - 1)
                _, nJ = nv.gamblet_level_size(h, k)
                ops[("R", k)] = coo_to_dense(*nv.gamblet_get_operator(h, 1, k), (nkm1, nk))
                ops[("B", k)] = coo_to_dense(*nv.gamblet_get_operator(h, 2, k), (nJ, nJ))
        return u, comps, ops
    finally:
        nv.gamblet_destroy(h)


def _compare(A, g, cells, q):
    ex = gamblet_exact(A, g, cells, q)
    u, comps, ops = _run_exact(A, g, cells, q)
    ud, _ = direct.solve(A, g)
    assert rel(u, ud) < TOL
    assert rel(u, ex["u"]) < TOL
    for k in range(1, q + 1):
        assert rel(comps[k - 1], ex["comps"][k - 1]) < TOL * max(
            1.0, np.linalg.norm(ex["u"]) / max(np.linalg.norm(ex["comps"][k - 1]), 1e-300)), k
        check_op(ops[("A", k)], ex["A"][k], TOL, ("A", k))
        if k >= 2:
            check_R(ops[("R", k)], ex["R"][k], TOL, ("R", k))
            check_op(ops[("B", k)], ex["B"][k], TOL, ("B", k))


def test_exact_c1_32x32_q5():
    # 32 x 32 cells, 961 unknowns, contrast 100, seed 0 (the small workload)
    p = make_problem(32, 100, 0)
    _compare(p.A, p.g, p.cells, p.q)


@pytest.mark.parametrize("n,C,seed", [(4, 10, 1), (8, 1e4, 2), (16, 1e6, 3)])
def test_exact_small_grids(n, C, seed):
    p = make_problem(n, C, seed)
    _compare(p.A, p.g, p.cells, p.q)


def test_exact_ragged_domain_with_holes():
    # remove a block of unknowns: parents with 1, 2 and 3 children appear at
    # several levels (uneven m_s, Sec. 4.6)
    p = make_problem(16, 1e3, 4)
    x, y = p.cells[:, 0], p.cells[:, 1]
    keep = ~((x >= 5) & (x <= 9) & (y >= 3) & (y <= 6)) & ~((x == 13) & (y == 11))
    A, g, cells = drop_nodes(p, keep)
    _compare(A, g, cells, p.q)
