"""GPU compression in the normalised gamblet basis against the oracle, and
the detail operators B^(k) (which fix that basis) against the oracle's."""
import numpy as np
import pytest

from oracle.compress import compress
from oracle.local import gamblet_local_setup
from workloads import make_example1, make_problem

from gpu_util import check_op, coo_to_dense, csr_arrays, rel

pytestmark = pytest.mark.gpu


def _setup(p):
    from paper_1503_03467_gb300 import native as nv
    o = nv.gamblet_default_opts()
    o.level_tol = 1e-14
    o.level_max_iter = 5000
    o.refine_max_iter = 0
    rp, ci, va = csr_arrays(p.A)
    return nv.gamblet_setup(rp, ci, va, p.q, p.cells, o)


@pytest.mark.parametrize("which", ["rough", "example1"])
def test_compression_matches_oracle(which):
    from paper_1503_03467_gb300 import native as nv
    p = make_problem(32, 1e3, 5) if which == "rough" else make_example1(6)
    ref = gamblet_local_setup(p.A, p.cells, p.q, 3.0)
    h = _setup(p)
    try:
        for k in range(2, p.q + 1):
            nJ = ref["B"][k].shape[0]
            B = coo_to_dense(*nv.gamblet_get_operator(h, 2, k), (nJ, nJ))
            check_op(B, ref["B"][k], 1e-10, ("B", k))
        for eps in (0.0, 1e-3, 1e-2):
            u_ref, kept_ref, total_ref = compress(ref, p.g, eps)
            u = np.zeros(p.ndof)
            kept, total = nv.gamblet_compress(h, p.g, eps, u)
            assert (kept, total) == (kept_ref, total_ref), eps
            assert rel(u, u_ref) < 1e-9, eps
    finally:
        nv.gamblet_destroy(h)


@pytest.mark.parametrize("construction", [2, 1])
def test_level_condition_matches_dense_eigenvalues(construction):
    """Lanczos extremes of B^(k) = W A W^T against the dense eigenvalues of
    the oracle's B^(k) for the same construction of W (exact when the
    Lanczos runs |J^(k)| steps)."""
    from paper_1503_03467_gb300 import native as nv
    p = make_problem(32, 1e3, 6)
    ref = gamblet_local_setup(p.A, p.cells, p.q, 3.0,
                              construction="const1" if construction == 1 else "const2")
    h = _setup(p)
    try:
        for k in range(2, p.q + 1):
            ev = np.linalg.eigvalsh(ref["B"][k].toarray())
            nJ = len(ev)
            steps = nJ if nJ <= 200 else 200
            lo, hi = nv.gamblet_level_condition(h, k, steps, construction)
            tol = 1e-8 if steps == nJ else 1e-3
            assert abs(hi - ev[-1]) <= tol * ev[-1], (k, hi, ev[-1])
            assert abs(lo - ev[0]) <= tol * ev[-1] + tol * ev[0], (k, lo, ev[0])
    finally:
        nv.gamblet_destroy(h)
