"""GPU parity of the three-dimensional path (include/gamblet3d.h) against the
CPU oracle: the exact transform (unbounded patches, Algorithm 1), the
localized setup of Algorithm 2 with both neighbourhood rules, holes in the
domain, the refined solve against the direct solve, and input validation.
Every operator is compared element by element (R row by row with its patch
support); float64 throughout."""
import numpy as np
import pytest

from oracle import direct
from oracle.exact import gamblet_exact
from oracle.local import gamblet_local_setup, gamblet_local_solve
from workloads import make_problem3

from gpu_util import check_R, check_op, coo_to_dense, csr_arrays, rel

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _opts(rho, rule=0, refine=0, patch_tol=1e-13, level_tol=1e-13):
    from paper_1503_03467_gb300 import native as nv
    o = nv.gamblet_default_opts()
    o.rho = rho
    o.nbr_rule = rule
    o.refine_max_iter = refine
    o.refine_tol = 1e-12
    o.patch_tol = patch_tol
    o.level_tol = level_tol
    o.level_max_iter = 2000
    return o


def _run(A, g, cells, q, o, components=True):
    from paper_1503_03467_gb300 import native as nv
    rp, ci, va = csr_arrays(A)
    h = nv.gamblet3d_setup(rp, ci, va, q, np.ascontiguousarray(cells, dtype=np.int32), o)
    try:
        n = A.shape[0]
        u = np.zeros(n)
        comps = np.zeros((q, n)) if components else None
        info = nv.Info()
        st = nv.gamblet3d_solve(h, g, u, comps, info)
        assert st == nv.OK, info.as_dict()
        ops = {}
        for k in range(1, q + 1):
            nk, _ = nv.gamblet3d_level_size(h, k)
            ops[("A", k)] = coo_to_dense(*nv.gamblet3d_get_operator(h, 0, k), (nk, nk))
            if k >= 2:
                nkm1, _ = nv.gamblet3d_level_size(h, k - 1)
                _, nJ = nv.gamblet3d_level_size(h, k)
                ops[("R", k)] = coo_to_dense(*nv.gamblet3d_get_operator(h, 1, k), (nkm1, nk))
                ops[("B", k)] = coo_to_dense(*nv.gamblet3d_get_operator(h, 2, k), (nJ, nJ))
        return u, comps, ops, info
    finally:
        nv.gamblet3d_destroy(h)


@pytest.mark.parametrize("n,seed", [(4, 0), (8, 1)])
def test_exact_transform_3d(n, seed):
    p = make_problem3(n, 100, seed)
    ex = gamblet_exact(p.A, p.g, p.cells, p.q)
    u, comps, ops, _ = _run(p.A, p.g, p.cells, p.q, _opts(0.0))
    ud, _ = direct.solve(p.A, p.g)
    assert rel(u, ud) < TOL
    for k in range(1, p.q + 1):
        scale = max(1.0, np.linalg.norm(ex["u"]) / max(np.linalg.norm(ex["comps"][k - 1]), 1e-300))
        assert rel(comps[k - 1], ex["comps"][k - 1]) < TOL * scale, k
        check_op(ops[("A", k)], ex["A"][k], TOL, ("A", k))
        if k >= 2:
            check_R(ops[("R", k)], ex["R"][k], TOL, ("R", k))
            check_op(ops[("B", k)], ex["B"][k], TOL, ("B", k))


@pytest.mark.parametrize("n,rho,rule,contrast", [(16, 1, "cheb", 1e3), (8, 1, "euclid", 1e3),
                                                  (16, 2, "cheb", 1e3), (16, 1, "cheb", 1e6)])
def test_localized_operators_3d(n, rho, rule, contrast):
    p = make_problem3(n, contrast, 2)
    s = gamblet_local_setup(p.A, p.cells, p.q, rho=rho, rule=rule)
    loc = gamblet_local_solve(s, p.g, return_components=True)
    u, comps, ops, info = _run(p.A, p.g, p.cells, p.q,
                               _opts(rho, rule=1 if rule == "cheb" else 0))
    for k in range(2, p.q + 1):
        check_R(ops[("R", k)], s["R"][k], TOL, ("R", k))
        check_op(ops[("A", k - 1)], s["A"][k - 1], TOL, ("A", k - 1))
        check_op(ops[("B", k)], s["B"][k], TOL, ("B", k))
    assert rel(u, loc["u"]) < 1e-9
    for k in range(1, p.q + 1):
        assert rel(comps[k - 1], loc["comps"][k - 1]) < 1e-9 * max(
            1.0, np.linalg.norm(loc["u"]) / max(np.linalg.norm(loc["comps"][k - 1]), 1e-300)), k
    assert info.patch_iters_max > 0


def test_domain_with_holes_3d():
    # an L-shaped prism: the unknowns with x >= 10 and y >= 10 are removed
    # (Dirichlet there), so parents on the re-entrant faces have 1, 2 or 4
    # of their 8 children
    p = make_problem3(16, 1e2, 3)
    keep = ~((p.cells[:, 0] >= 10) & (p.cells[:, 1] >= 10))
    idx = np.nonzero(keep)[0]
    A = p.A.tocsr()[idx][:, idx].tocsr()
    g = p.g[idx].copy()
    cells = np.ascontiguousarray(p.cells[idx])
    s = gamblet_local_setup(A, cells, p.q, rho=1, rule="cheb")
    loc = gamblet_local_solve(s, g)
    u, _, ops, _ = _run(A, g, cells, p.q, _opts(1, rule=1), components=False)
    for k in range(2, p.q + 1):
        check_R(ops[("R", k)], s["R"][k], TOL, ("R", k))
        check_op(ops[("A", k - 1)], s["A"][k - 1], TOL, ("A", k - 1))
    assert rel(u, loc["u"]) < 1e-9


def test_refined_solve_matches_direct_3d():
    from paper_1503_03467_gb300 import native as nv
    p = make_problem3(32, 1e4, 0)
    o = _opts(1, rule=1, refine=100, patch_tol=1e-6, level_tol=1e-3)
    o.refine_tol = 1e-11
    rp, ci, va = csr_arrays(p.A)
    h = nv.gamblet3d_setup(rp, ci, va, p.q, p.cells, o)
    try:
        u = np.zeros(p.ndof)
        info = nv.Info()
        assert nv.gamblet3d_solve(h, p.g, u, None, info) == nv.OK
        assert info.rel_residual <= 1e-11
        assert 1 <= info.outer_iters < 60
        # device buffers give the same answer
        import torch
        gd = torch.from_numpy(p.g).cuda()
        ud = torch.zeros(p.ndof, dtype=torch.float64, device="cuda")
        assert nv.gamblet3d_solve(h, gd, ud, None, nv.Info()) == nv.OK
        assert rel(ud.cpu().numpy(), u) < 1e-13
        geo = nv.gamblet3d_level_geometry(h, p.q)
        assert geo["neighbours"] == 27 and geo["block_offsets"] == 27
    finally:
        nv.gamblet3d_destroy(h)
    ud, _ = direct.solve(p.A, p.g)
    assert rel(u, ud) < 1e-9


def test_level_sizes_3d():
    from paper_1503_03467_gb300 import native as nv
    p = make_problem3(16, 10, 0)
    rp, ci, va = csr_arrays(p.A)
    h = nv.gamblet3d_setup(rp, ci, va, p.q, p.cells, _opts(1, rule=1))
    try:
        sizes = [nv.gamblet3d_level_size(h, k) for k in range(1, p.q + 1)]
    finally:
        nv.gamblet3d_destroy(h)
    assert [s[0] for s in sizes] == [8, 64, 512, 15 ** 3]
    assert [s[1] for s in sizes] == [0, 56, 448, 15 ** 3 - 512]


def test_input_validation_3d():
    from paper_1503_03467_gb300 import native as nv
    p = make_problem3(8, 10, 0)
    rp, ci, va = csr_arrays(p.A)
    bad = p.cells.copy()
    bad[5] = [8, 1, 1]                      # outside [0, 2^3)
    with pytest.raises(nv.GambletError) as e:
        nv.gamblet3d_setup(rp, ci, va, p.q, bad, _opts(1))
    assert e.value.status == nv.ERR_INVALID_ARG
    dup = p.cells.copy()
    dup[5] = dup[6]                         # two unknowns in one cell
    with pytest.raises(nv.GambletError) as e:
        nv.gamblet3d_setup(rp, ci, va, p.q, dup, _opts(1))
    assert e.value.status == nv.ERR_INVALID_ARG
    with pytest.raises(nv.GambletError) as e:
        nv.gamblet3d_setup(rp, ci, va, 1, p.cells, _opts(1))
    assert e.value.status == nv.ERR_INVALID_ARG
    o = _opts(1)
    o.precision = nv.MIXED
    with pytest.raises(nv.GambletError) as e:
        nv.gamblet3d_setup(rp, ci, va, p.q, p.cells, o)
    assert e.value.status == nv.ERR_UNSUPPORTED
