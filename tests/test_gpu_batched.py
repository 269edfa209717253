"""Many independent problems in one hierarchy (gamblet_setup_batched).

The batched setup must equal the localized transform of Algorithm 2 applied
to the combined block-diagonal system on the packed lattice (checked against
the oracle level by level), and its refined solve must reproduce every
problem's direct solution.  Also covers a single problem whose cells fill
only a Morton prefix of its lattice."""
import numpy as np
import pytest

from oracle import direct
from oracle.local import gamblet_local_setup, gamblet_local_solve
from workloads import make_batch, make_problem

from gpu_util import check_R, check_op, coo_to_dense, csr_arrays, drop_nodes, pack_problems, rel

pytestmark = pytest.mark.gpu


def _opts(precision=0, refine=0, level_tol=1e-14, patch_tol=0.0):
    from paper_1503_03467_gb300 import native as nv
    o = nv.gamblet_default_opts()
    o.rho = 3.0
    o.precision = precision
    o.refine_max_iter = refine
    o.level_tol = level_tol
    o.level_max_iter = 5000
    o.patch_tol = patch_tol
    return o


def _batched(probs, o):
    from paper_1503_03467_gb300 import native as nv
    return nv.gamblet_setup_batched(
        [(*csr_arrays(p.A), p.q, p.cells) for p in probs], o)


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


@pytest.mark.parametrize("patch_tol", [0.0, -1.0])
def test_batched_equals_localized_transform_of_packed_system(patch_tol):
    from paper_1503_03467_gb300 import native as nv
    probs = make_batch(5, first_seed=1, sides=(8, 16, 32), log10_contrast=(2.0, 4.0))
    A, g, cells, Q, offsets = pack_problems(probs)
    ref = gamblet_local_setup(A, cells, Q, 3.0)
    one = gamblet_local_solve(ref, g)
    h, off = _batched(probs, _opts(patch_tol=patch_tol))
    try:
        np.testing.assert_array_equal(off, offsets)
        ops = _ops(h, Q)
        for k in range(2, Q + 1):
            check_R(ops[("R", k)], ref["R"][k], 1e-10, ("R", k))
            check_op(ops[("A", k - 1)], ref["A"][k - 1], 1e-10, ("A", k - 1))
        u = np.zeros(A.shape[0])
        assert nv.gamblet_solve(h, g, u) == nv.OK
        assert rel(u, one["u"]) < 1e-9
    finally:
        nv.gamblet_destroy(h)


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_refined_solve_matches_each_direct_solve(precision):
    from paper_1503_03467_gb300 import native as nv
    probs = make_batch(7, first_seed=11, sides=(16, 32, 64))
    h, off = _batched(probs, _opts(precision=precision, refine=60, level_tol=0.1))
    try:
        g = np.concatenate([p.g for p in probs])
        u = np.zeros(g.shape[0])
        info = nv.Info()
        assert nv.gamblet_solve(h, g, u, None, info) == nv.OK
        assert info.rel_residual < 1e-12
        for p, pr in enumerate(probs):
            ud, _ = direct.solve(pr.A, pr.g)
            assert rel(u[off[p]:off[p + 1]], ud) < 1e-9, p
    finally:
        nv.gamblet_destroy(h)


def test_batched_single_problem_equals_plain_setup():
    from paper_1503_03467_gb300 import native as nv
    p = make_problem(32, 1e4, 3)
    rp, ci, va = csr_arrays(p.A)
    h1 = nv.gamblet_setup(rp, ci, va, p.q, p.cells, _opts())
    h2, off = _batched([p], _opts())
    try:
        assert list(off) == [0, p.ndof]
        u1 = np.zeros(p.ndof)
        u2 = np.zeros(p.ndof)
        assert nv.gamblet_solve(h1, p.g, u1) == nv.OK
        assert nv.gamblet_solve(h2, p.g, u2) == nv.OK
        np.testing.assert_array_equal(u1, u2)
    finally:
        nv.gamblet_destroy(h1)
        nv.gamblet_destroy(h2)


def test_prefix_lattice_single_problem():
    """Cells only in the first three level-1 quadrants: the stored Morton
    prefix ends before the last quadrant at every level."""
    from paper_1503_03467_gb300 import native as nv
    p = make_problem(32, 1e3, 4)
    x, y = p.cells[:, 0], p.cells[:, 1]
    keep = ~((x >= 16) & (y >= 16)) & ~((x >= 12) & (x <= 13) & (y >= 8) & (y <= 15))
    A, g, cells = drop_nodes(p, keep)
    ref = gamblet_local_setup(A, cells, p.q, 3.0)
    one = gamblet_local_solve(ref, g)
    rp, ci, va = csr_arrays(A)
    h = nv.gamblet_setup(rp, ci, va, p.q, cells, _opts())
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


def test_batched_rejects_entries_outside_their_problem():
    from paper_1503_03467_gb300 import native as nv
    probs = make_batch(3, first_seed=1, sides=(8, 16))
    items = [[*csr_arrays(p.A), p.q, p.cells] for p in probs]
    bad = [list(it) for it in items]
    ci = bad[1][1].copy()
    ci[0] = probs[1].ndof  # a valid combined index, but outside problem 1
    bad[1][1] = ci
    with pytest.raises(nv.GambletError) as e:
        nv.gamblet_setup_batched(bad, _opts())
    assert e.value.status == nv.ERR_INVALID_ARG
    bad = [list(it) for it in items]
    cl = bad[2][4].copy()
    cl[0, 0] = 1 << probs[2].q
    bad[2][4] = cl
    with pytest.raises(nv.GambletError) as e:
        nv.gamblet_setup_batched(bad, _opts())
    assert e.value.status == nv.ERR_INVALID_ARG
