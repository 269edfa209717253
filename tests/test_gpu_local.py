"""GPU parity of the localized transform (Algorithm 2 with Definition defb)
against the CPU oracle, and of the refined solution against the direct solve."""
import numpy as np
import pytest

from oracle import direct
from oracle.local import gamblet_local_setup, gamblet_local_solve
from workloads import make_problem

from gpu_util import check_R, check_op, coo_to_dense, csr_arrays, drop_nodes, rel

pytestmark = pytest.mark.gpu


def _setup(A, cells, q, rho, rule=0, precision=0, refine=0, level_tol=1e-14, patch_tol=0.0):
    from paper_1503_03467_gb300 import native as nv
    rp, ci, va = csr_arrays(A)
    o = nv.gamblet_default_opts()
    o.rho = rho
    o.nbr_rule = rule
    o.precision = precision
    o.refine_max_iter = refine
    o.level_tol = level_tol
    o.level_max_iter = 5000
    o.patch_tol = patch_tol
    return nv.gamblet_setup(rp, ci, va, q, cells, o)


def _ops(h, q):
    from paper_1503_03467_gb300 import native as nv
    out = {}
    for k in range(1, q + 1):
        nk, _ = nv.gamblet_level_size(h, k)
        out[("A", k)] = coo_to_dense(*nv.gamblet_get_operator(h, 0, k), (nk, nk))
        if k >= 2:
            nkm1, _ = nv.gamblet_level_size(h, k - 1)
            out[("R", k)] = coo_to_dense(*nv.gamblet_get_operator(h, 1, k), (nkm1, nk))
    return out


# (n, contrast, seed, rho, rule, patch solver: 0 = block-Jacobi CG, -1 = Cholesky)
CASES = [(32, 1e4, 0, 3.0, 0, 0.0), (64, 1e4, 1, 3.0, 0, 0.0), (32, 1e2, 2, 2.0, 0, 0.0),
         (32, 1e3, 3, 3.0, 1, 0.0), (64, 1e6, 5, 1.0, 0, 0.0), (32, 1e4, 0, 3.0, 0, -1.0),
         (64, 1e4, 1, 2.0, 1, -1.0)]


@pytest.mark.parametrize("n,C,seed,rho,rule,patch_tol", CASES)
def test_local_operators_and_one_pass(n, C, seed, rho, rule, patch_tol):
    from paper_1503_03467_gb300 import native as nv
    p = make_problem(n, C, seed)
    ref = gamblet_local_setup(p.A, p.cells, p.q, rho, "euclid" if rule == 0 else "cheb")
    one = gamblet_local_solve(ref, p.g)
    h = _setup(p.A, p.cells, p.q, rho, rule, patch_tol=patch_tol)
    try:
        ops = _ops(h, p.q)
        for k in range(2, p.q + 1):
            check_R(ops[("R", k)], ref["R"][k], 1e-10, ("R", k))
            check_op(ops[("A", k - 1)], ref["A"][k - 1], 1e-10, ("A", k - 1))
        u = np.zeros(p.ndof)
        st = nv.gamblet_solve(h, p.g, u)
        assert st == nv.OK
        assert rel(u, one["u"]) < 1e-9
    finally:
        nv.gamblet_destroy(h)


@pytest.mark.parametrize("precision", [0, 1])
def test_refined_solution_matches_direct(precision):
    from paper_1503_03467_gb300 import native as nv
    p = make_problem(64, 1e4, 7)
    ud, _ = direct.solve(p.A, p.g)
    h = _setup(p.A, p.cells, p.q, 3.0, precision=precision, refine=50, level_tol=1e-6)
    try:
        u = np.zeros(p.ndof)
        info = nv.Info()
        st = nv.gamblet_solve(h, p.g, u, None, info)
        assert st == nv.OK
        assert info.rel_residual < 1e-12
        assert rel(u, ud) < 1e-9
    finally:
        nv.gamblet_destroy(h)


def test_local_ragged_domain():
    from paper_1503_03467_gb300 import native as nv
    p = make_problem(32, 1e3, 8)
    x, y = p.cells[:, 0], p.cells[:, 1]
    keep = ~((x >= 10) & (x <= 17) & (y >= 12) & (y <= 14)) & ~((x == 3) & (y == 29))
    A, g, cells = drop_nodes(p, keep)
    ref = gamblet_local_setup(A, cells, p.q, 3.0)
    one = gamblet_local_solve(ref, g)
    h = _setup(A, cells, p.q, 3.0)
    try:
        ops = _ops(h, p.q)
        for k in range(2, p.q + 1):
            check_R(ops[("R", k)], ref["R"][k], 1e-10, ("R", k))
            check_op(ops[("A", k - 1)], ref["A"][k - 1], 1e-10, ("A", k - 1))
        u = np.zeros(A.shape[0])
        assert nv.gamblet_solve(h, g, u) == nv.OK
        assert rel(u, one["u"]) < 1e-9
    finally:
        nv.gamblet_destroy(h)


def test_device_pointers_and_torch_tensors():
    import torch
    from paper_1503_03467_gb300 import native as nv
    p = make_problem(32, 1e4, 9)
    rp, ci, va = csr_arrays(p.A)
    dev = torch.device("cuda:0")
    t = lambda a: torch.from_numpy(a).to(dev)
    o = nv.gamblet_default_opts()
    o.rho = 3.0
    o.refine_max_iter = 30
    o.level_tol = 1e-6
    h = nv.gamblet_setup(t(rp), t(ci), t(va), p.q, t(np.ascontiguousarray(p.cells)), o)
    try:
        g = t(p.g)
        u = torch.zeros_like(g)
        assert nv.gamblet_solve(h, g, u) == nv.OK
        ud, _ = direct.solve(p.A, p.g)
        assert rel(u.cpu().numpy(), ud) < 1e-9
    finally:
        nv.gamblet_destroy(h)


def test_invalid_inputs_are_rejected():
    from paper_1503_03467_gb300 import native as nv
    p = make_problem(8, 10, 0)
    rp, ci, va = csr_arrays(p.A)
    cells = p.cells.copy()
    cells[1] = cells[0]
    with pytest.raises(nv.GambletError) as e:
        nv.gamblet_setup(rp, ci, va, p.q, cells)
    assert e.value.status == nv.ERR_INVALID_ARG
    bad = p.cells.copy()
    bad[0, 0] = 1 << p.q
    with pytest.raises(nv.GambletError) as e:
        nv.gamblet_setup(rp, ci, va, p.q, bad)
    assert e.value.status == nv.ERR_INVALID_ARG
    ci2 = ci.copy()
    ci2[3] = 10 ** 6
    with pytest.raises(nv.GambletError) as e:
        nv.gamblet_setup(rp, ci2, va, p.q, p.cells)
    assert e.value.status == nv.ERR_INVALID_ARG
    # an indefinite operator meets a non-positive pivot
    with pytest.raises(nv.GambletError) as e:
        nv.gamblet_setup(rp, ci, -va, p.q, p.cells)
    assert e.value.status == nv.ERR_NOT_SPD


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (1, 1e-3)])
def test_truncated_solve_sums_leading_components(precision, tol):
    """u^(k) of a truncated solve = the oracle's components of levels 1..k
    (Sec. 5.4); k = q is the one-pass solution."""
    from paper_1503_03467_gb300 import native as nv
    p = make_problem(64, 1e4, 12)
    ref = gamblet_local_setup(p.A, p.cells, p.q, 3.0)
    one = gamblet_local_solve(ref, p.g, return_components=True)
    h = _setup(p.A, p.cells, p.q, 3.0, precision=precision, level_tol=1e-14 if precision == 0 else 1e-7,
               patch_tol=0.0 if precision == 0 else 1e-7)
    try:
        for k in (1, 2, 4, p.q):
            u = np.zeros(p.ndof)
            assert nv.gamblet_solve_truncated(h, k, p.g, u) == nv.OK
            assert rel(u, one["comps"][:k].sum(axis=0)) < tol, k
        with pytest.raises(nv.GambletError):
            nv.gamblet_solve_truncated(h, p.q + 1, p.g, np.zeros(p.ndof))
        # the handle keeps its full depth: a plain solve adds every level
        u = np.zeros(p.ndof)
        assert nv.gamblet_solve(h, p.g, u) == nv.OK
        assert rel(u, one["u"]) < tol
    finally:
        nv.gamblet_destroy(h)


@pytest.mark.parametrize("precision", [0, 1])
def test_autotuned_shapes_are_valid_and_change_nothing_but_rounding(precision):
    """The autotuner picks among launch shapes that compute the same rows
    (only the summation order differs, and on the mixed path the
    tensor-core patch solves round the scaled patch matrix to float16, which
    the refined solve absorbs); 256 x 256 has levels large enough to be
    tuned."""
    from paper_1503_03467_gb300 import native as nv
    p = make_problem(256, 1e4, 13)
    rp, ci, va = csr_arrays(p.A)
    us = []
    for tune in (1, 0, 1):  # the second tuned setup reads the process-wide cache
        o = nv.gamblet_default_opts()
        o.precision = precision
        o.level_tol = 0.1
        o.refine_tol = 1e-12
        o.refine_max_iter = 100
        o.autotune = tune
        h = nv.gamblet_setup(rp, ci, va, p.q, p.cells, o)
        try:
            for k in range(2, p.q + 1):
                sh = nv.gamblet_launch_shapes(h, k)
                simt = sh["patch_spp"] in (1, 2, 4) and sh["patch_gather"] in (0, 1, 2)
                mma = precision == 1 and sh["patch_spp"] == 0 and sh["patch_gather"] in (3, 4)
                assert simt or mma, sh
                assert sh["galerkin_variant"] in range(9) and sh["cg_spp"] in (1, 4, 16)
            u = np.zeros(p.ndof)
            info = nv.Info()
            assert nv.gamblet_solve(h, p.g, u, None, info) == nv.OK
            assert info.rel_residual <= 1e-12
            us.append(u)
        finally:
            nv.gamblet_destroy(h)
    assert rel(us[0], us[1]) < 1e-9 and rel(us[2], us[1]) < 1e-9


@pytest.mark.parametrize("variant,gather", [(0, 0), (1, 1), (2, 0), (2, 1), (3, 0), (3, 2),
                                            (4, 2), (5, 2), (6, 2), (7, 0), (8, 2)])
def test_every_galerkin_kernel_and_gather_matches_oracle(variant, gather):
    """Each Galerkin kernel and patch-CG gather, forced on every level,
    reproduces the oracle's localized operators (the autotuner only picks
    among them)."""
    from paper_1503_03467_gb300 import native as nv
    p = make_problem(64, 1e3, 14)
    ref = gamblet_local_setup(p.A, p.cells, p.q, 3.0)
    rp, ci, va = csr_arrays(p.A)
    o = nv.gamblet_default_opts()
    o.level_tol = 1e-14
    o.level_max_iter = 5000
    o.refine_max_iter = 0
    o.galerkin_variant = variant
    o.patch_gather = gather
    h = nv.gamblet_setup(rp, ci, va, p.q, p.cells, o)
    try:
        for k in range(2, p.q + 1):
            assert nv.gamblet_launch_shapes(h, k)["galerkin_variant"] == variant
            assert nv.gamblet_launch_shapes(h, k)["patch_gather"] == gather
        ops = _ops(h, p.q)
        for k in range(2, p.q + 1):
            check_R(ops[("R", k)], ref["R"][k], 1e-10, ("R", k))
            check_op(ops[("A", k - 1)], ref["A"][k - 1], 1e-10, ("A", k - 1))
    finally:
        nv.gamblet_destroy(h)


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4, 5, 6, 7, 8])
def test_galerkin_kernels_on_ragged_and_prefix_domains(variant):
    """Every Galerkin kernel on a domain with holes and on one whose cells
    fill only a Morton prefix (rows of a tile or window missing)."""
    from paper_1503_03467_gb300 import native as nv
    p = make_problem(32, 1e3, 15)
    x, y = p.cells[:, 0], p.cells[:, 1]
    masks = [~((x >= 10) & (x <= 17) & (y >= 12) & (y <= 14)) & ~((x == 3) & (y == 29)),
             ~((x >= 16) & (y >= 16)) & ~((x >= 9) & (x <= 11) & (y <= 4))]
    for keep in masks:
        A, g, cells = drop_nodes(p, keep)
        ref = gamblet_local_setup(A, cells, p.q, 3.0)
        rp, ci, va = csr_arrays(A)
        o = nv.gamblet_default_opts()
        o.level_tol = 1e-14
        o.level_max_iter = 5000
        o.refine_max_iter = 0
        o.galerkin_variant = variant
        h = nv.gamblet_setup(rp, ci, va, p.q, cells, o)
        try:
            ops = _ops(h, p.q)
            for k in range(2, p.q + 1):
                check_R(ops[("R", k)], ref["R"][k], 1e-10, ("R", k))
                check_op(ops[("A", k - 1)], ref["A"][k - 1], 1e-10, ("A", k - 1))
        finally:
            nv.gamblet_destroy(h)


@pytest.mark.parametrize("variant", [-1, 1, 3])
def test_rho4_operators_match_oracle(variant):
    """rho = 4 (89 neighbour parents, wider windows and stencils) with the
    automatic and the forced Galerkin kernels: float32 operators of the mixed
    path against the float64 oracle, and the float64 path, whose patch blocks
    exceed one CTA's shared memory and are solved by the cluster-distributed
    patch CG, element by element at 1e-10."""
    from paper_1503_03467_gb300 import native as nv
    p = make_problem(64, 1e3, 16)
    ref = gamblet_local_setup(p.A, p.cells, p.q, 4.0)
    one = gamblet_local_solve(ref, p.g)
    rp, ci, va = csr_arrays(p.A)
    o = nv.gamblet_default_opts()
    o.rho = 4.0
    o.precision = nv.MIXED
    o.patch_tol = 1e-7
    o.level_tol = 1e-7
    o.level_max_iter = 5000
    o.refine_max_iter = 0
    o.galerkin_variant = variant
    h = nv.gamblet_setup(rp, ci, va, p.q, p.cells, o)
    try:
        ops = _ops(h, p.q)
        for k in range(2, p.q + 1):
            check_R(ops[("R", k)], ref["R"][k], 1e-4, ("R", k))
            check_op(ops[("A", k - 1)], ref["A"][k - 1], 1e-4, ("A", k - 1))
    finally:
        nv.gamblet_destroy(h)
    o.precision = nv.FP64
    o.patch_tol = 0.0
    o.level_tol = 1e-14
    h = nv.gamblet_setup(rp, ci, va, p.q, p.cells, o)
    try:
        assert any(nv.gamblet_launch_shapes(h, k)["patch_gather"] == 5 for k in range(2, p.q + 1))
        ops = _ops(h, p.q)
        for k in range(2, p.q + 1):
            check_R(ops[("R", k)], ref["R"][k], 1e-10, ("R", k))
            check_op(ops[("A", k - 1)], ref["A"][k - 1], 1e-10, ("A", k - 1))
        u = np.zeros(p.ndof)
        assert nv.gamblet_solve(h, p.g, u) == nv.OK
        assert rel(u, one["u"]) < 1e-9
    finally:
        nv.gamblet_destroy(h)


@pytest.mark.parametrize("rho", [5.0, 6.0])
@pytest.mark.parametrize("precision", [0, 1])
def test_large_patches_over_thread_block_clusters(rho, precision):
    """rho = 5 and 6 (129 and 169 neighbour parents, up to 507 patch unknowns):
    every level's patch blocks exceed one CTA's shared memory and the patch
    CG runs over a cluster of CTAs on one GPU.  Operators against the oracle
    element by element (float64 at 1e-10; float32 with the CG to 1e-7 at
    1e-4), the one-pass solution, and the refined solution."""
    from paper_1503_03467_gb300 import native as nv
    p = make_problem(32, 1e4, 17)
    ref = gamblet_local_setup(p.A, p.cells, p.q, rho)
    one = gamblet_local_solve(ref, p.g)
    tol = 1e-10 if precision == 0 else 1e-4
    h = _setup(p.A, p.cells, p.q, rho, precision=precision,
               patch_tol=0.0 if precision == 0 else 1e-7)
    try:
        shapes = [nv.gamblet_launch_shapes(h, k) for k in range(2, p.q + 1)]
        assert any(sh["patch_gather"] == 5 and sh["patch_spp"] in (2, 4, 8, 16) for sh in shapes)
        ops = _ops(h, p.q)
        for k in range(2, p.q + 1):
            check_R(ops[("R", k)], ref["R"][k], tol, ("R", k))
            check_op(ops[("A", k - 1)], ref["A"][k - 1], tol, ("A", k - 1))
        u = np.zeros(p.ndof)
        assert nv.gamblet_solve(h, p.g, u) == nv.OK
        assert rel(u, one["u"]) < (1e-9 if precision == 0 else 1e-3)
    finally:
        nv.gamblet_destroy(h)
    h = _setup(p.A, p.cells, p.q, rho, precision=precision, refine=60, level_tol=1e-6)
    try:
        u = np.zeros(p.ndof)
        info = nv.Info()
        assert nv.gamblet_solve(h, p.g, u, None, info) == nv.OK
        assert rel(u, direct.solve(p.A, p.g)[0]) < 1e-9
    finally:
        nv.gamblet_destroy(h)


@pytest.mark.parametrize("precision", [0, 1])
def test_several_right_hand_sides(precision):
    """gamblet_solve_many (groups of four sharing the matrix reads) against
    the direct solves and, for the one-pass transform, against gamblet_solve
    one right-hand side at a time."""
    from paper_1503_03467_gb300 import native as nv
    p = make_problem(64, 1e4, 17)
    rng = np.random.default_rng(17)
    G = np.ascontiguousarray(rng.standard_normal((5, p.ndof)))
    G[3] = 0.0  # a zero right-hand side inside a group
    for refine in (0, 60):
        h = _setup(p.A, p.cells, p.q, 3.0, precision=precision, refine=refine,
                   level_tol=1e-12 if refine == 0 and precision == 0 else 0.1)
        try:
            U = np.zeros_like(G)
            info = nv.Info()
            assert nv.gamblet_solve_many(h, G, U, info) == nv.OK
            for r in range(G.shape[0]):
                if refine == 0:
                    u1 = np.zeros(p.ndof)
                    nv.gamblet_solve(h, G[r], u1)
                    tol = 1e-11 if precision == 0 else 1e-4
                    assert np.linalg.norm(U[r] - u1) <= tol * max(np.linalg.norm(u1), 1e-300), r
                else:
                    if r == 3:
                        assert not U[r].any()
                        continue
                    ud, _ = direct.solve(p.A, G[r])
                    assert rel(U[r], ud) < 1e-9, r
            if refine:
                assert info.rel_residual < 1e-12
        finally:
            nv.gamblet_destroy(h)


@pytest.mark.parametrize("precision", [0, 1])
def test_convergence_status_and_iteration_counts(precision):
    """The status and counters a caller relies on: a one-pass solve whose
    level CGs are stopped after a few iterations reports NOT_CONVERGED with
    those iteration counts; an outer iteration stopped short of its
    tolerance reports NOT_CONVERGED with its count; a normal solve reports OK
    and at least one level-CG iteration on every level.  (The counts are
    accumulated on the device and read once per solve.)"""
    from paper_1503_03467_gb300 import native as nv
    p = make_problem(32, 1e3, 3)
    rp, ci, va = csr_arrays(p.A)

    def run(level_tol, level_max_iter, refine_tol, refine_max_iter):
        o = nv.gamblet_default_opts()
        o.precision = precision
        o.level_tol = level_tol
        o.level_max_iter = level_max_iter
        o.refine_tol = refine_tol
        o.refine_max_iter = refine_max_iter
        h = nv.gamblet_setup(rp, ci, va, p.q, p.cells, o)
        try:
            u = np.zeros(p.ndof)
            info = nv.Info()
            st = nv.gamblet_solve(h, p.g, u, None, info)
            return st, info, u
        finally:
            nv.gamblet_destroy(h)

    # one pass, level CGs capped at two iterations and far from 1e-14
    st, info, u = run(1e-14, 2, 1e-10, 0)
    assert st == nv.ERR_NOT_CONVERGED and info.status == nv.ERR_NOT_CONVERGED
    assert np.all(np.isfinite(u)) and np.linalg.norm(u) > 0
    for k in range(2, p.q + 1):
        assert 1 <= info.level_iters[k] <= 2, (k, info.level_iters[k])
    # outer iteration capped at one step, tolerance out of reach
    st, info, u = run(0.1, 1000, 1e-15, 1)
    assert st == nv.ERR_NOT_CONVERGED and info.outer_iters == 1
    # normal solve
    st, info, u = run(0.1, 1000, 1e-10, 100)
    assert st == nv.OK and info.rel_residual <= 1e-10
    assert all(info.level_iters[k] >= 1 for k in range(2, p.q + 1))
    assert rel(u, direct.solve(p.A, p.g)[0]) < 1e-8


# ---- tensor-core patch solves (tcgen05, windows of 1 x 1 or 2 x 2 cells) ----
#
# The tensor-core kernel solves each patch system on the block-Jacobi-scaled
# matrix L^-1 B L^-T stored in float16, with float32 accumulation and float32
# CG vectors.  Rounding the scaled matrix to float16 perturbs every entry by
# at most u = 2^-11 = 4.9e-4 relative, so the patch solutions (the rows of
# R) move by about u times the condition number of the scaled patch matrix
# from the exact ones; measured 0.6e-4 to 1.0e-4 of each row's largest entry
# on these cases with the CG tolerance at 1e-6.  The bound below is 2u per
# row for R and 1e-4 for A^(k-1) (element-wise, of its largest entry), and
# the support of R must be the oracle's patch support exactly.

MMA_CASES = [(32, 1e4, 0, 3.0, 0), (64, 1e4, 1, 3.0, 0), (64, 1e6, 5, 2.0, 0), (32, 1e3, 3, 3.0, 1)]


@pytest.mark.parametrize("force", [3, 4])
@pytest.mark.parametrize("n,C,seed,rho,rule", MMA_CASES)
def test_tensor_core_patch_solves_match_oracle(force, n, C, seed, rho, rule):
    from paper_1503_03467_gb300 import native as nv
    p = make_problem(n, C, seed)
    ref = gamblet_local_setup(p.A, p.cells, p.q, rho, "euclid" if rule == 0 else "cheb")
    rp, ci, va = csr_arrays(p.A)
    o = nv.gamblet_default_opts()
    o.rho = rho
    o.nbr_rule = rule
    o.precision = nv.MIXED
    o.patch_tol = 1e-6
    o.patch_gather = force
    o.level_tol = 1e-7
    o.level_max_iter = 5000
    o.refine_max_iter = 0
    h = nv.gamblet_setup(rp, ci, va, p.q, p.cells, o)
    try:
        for k in range(2, p.q + 1):
            assert nv.gamblet_launch_shapes(h, k)["patch_gather"] == force
        ops = _ops(h, p.q)
        for k in range(2, p.q + 1):
            check_R(ops[("R", k)], ref["R"][k], 2 * 2.0 ** -11, ("R", k))
            check_op(ops[("A", k - 1)], ref["A"][k - 1], 1e-4, ("A", k - 1))
    finally:
        nv.gamblet_destroy(h)


@pytest.mark.parametrize("force", [3, 4])
def test_tensor_core_patch_solves_on_ragged_domain_and_refined_solve(force):
    """Holes (parents with 1, 2 and 3 children, absent union parents at the
    boundary of a hole) through the tensor-core windows, and the refined
    solution of the same handle type against the direct solve."""
    from paper_1503_03467_gb300 import native as nv
    p = make_problem(32, 1e3, 8)
    x, y = p.cells[:, 0], p.cells[:, 1]
    keep = ~((x >= 10) & (x <= 17) & (y >= 12) & (y <= 14)) & ~((x == 3) & (y == 29))
    A, g, cells = drop_nodes(p, keep)
    ref = gamblet_local_setup(A, cells, p.q, 3.0)
    rp, ci, va = csr_arrays(A)
    o = nv.gamblet_default_opts()
    o.rho = 3.0
    o.precision = nv.MIXED
    o.patch_tol = 1e-6
    o.patch_gather = force
    o.level_tol = 1e-7
    o.level_max_iter = 5000
    o.refine_max_iter = 0
    h = nv.gamblet_setup(rp, ci, va, p.q, cells, o)
    try:
        ops = _ops(h, p.q)
        for k in range(2, p.q + 1):
            check_R(ops[("R", k)], ref["R"][k], 2 * 2.0 ** -11, ("R", k))
            check_op(ops[("A", k - 1)], ref["A"][k - 1], 1e-4, ("A", k - 1))
    finally:
        nv.gamblet_destroy(h)
    o.patch_tol = 1e-3
    o.refine_max_iter = 60
    o.level_tol = 1e-6
    h = nv.gamblet_setup(rp, ci, va, p.q, cells, o)
    try:
        u = np.zeros(A.shape[0])
        info = nv.Info()
        assert nv.gamblet_solve(h, g, u, None, info) == nv.OK
        assert info.rel_residual < 1e-12
        assert rel(u, direct.solve(A, g)[0]) < 1e-9
    finally:
        nv.gamblet_destroy(h)


def test_tensor_core_patch_solves_need_the_mixed_path():
    from paper_1503_03467_gb300 import native as nv
    p = make_problem(16, 1e2, 0)
    rp, ci, va = csr_arrays(p.A)
    o = nv.gamblet_default_opts()
    o.rho = 2.0
    o.precision = nv.FP64
    o.patch_gather = 4
    with pytest.raises(nv.GambletError) as e:
        nv.gamblet_setup(rp, ci, va, p.q, p.cells, o)
    assert e.value.status == nv.ERR_UNSUPPORTED


def test_one_pass_gradient_refuses_cluster_patches():
    """The reverse pass has no cluster form of its adjoint patch solves, so a
    handle whose patches needed a thread-block cluster is refused."""
    from paper_1503_03467_gb300 import native as nv
    from workloads import cell_corner_dofs
    from workloads.rough import K_REF
    p = make_problem(64, 1e2, 2)
    h = _setup(p.A, p.cells, p.q, 4.0, precision=0, patch_tol=1e-10)
    try:
        assert any(nv.gamblet_launch_shapes(h, k)["patch_gather"] == 5 for k in range(2, p.q + 1))
        dJ = np.zeros(p.n * p.n)
        with pytest.raises(nv.GambletError) as e:
            nv.gamblet_grad_onepass(h, cell_corner_dofs(p.n), np.exp(p.log_a.ravel()),
                                    K_REF.ravel().copy(), p.g, np.zeros(p.ndof), dJ)
        assert e.value.status == nv.ERR_UNSUPPORTED
    finally:
        nv.gamblet_destroy(h)
