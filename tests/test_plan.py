"""Host logic of the symbolic plan (no GPU): gamblet_plan_check rebuilds the
tables of a 2^q square and verifies them against their definitions derived a
second way - the half-plane of each symmetric level stencil (the level CG
stores one block per pair of opposite offsets), the patch block lists and
adjacency (Definition defb), the tensor-core windows, the phase-1 contributions of
the tiled Galerkin product (Eq. eqhuhiuv; every Ahat[o][u] Rhat_r(j) with
u = r + N_j - O_o at a position the outputs read, exactly once) and its
phase-2 incidences, for single targets and for horizontal pairs of targets."""
import pytest

from paper_1503_03467_gb300 import build


@pytest.fixture(scope="module")
def nv():
    build.build()
    from paper_1503_03467_gb300 import native
    return native


@pytest.mark.parametrize("q,rho,rule", [(4, 1.0, 0), (5, 2.0, 0), (6, 3.0, 0), (8, 3.0, 0),
                                        (6, 2.0, 1), (5, 4.0, 0), (7, 1.5, 1), (6, 6.0, 0),
                                        (10, 3.0, 0), (11, 3.0, 0), (9, 4.0, 0)])
def test_plan_tables_match_their_definitions(nv, q, rho, rule):
    c = nv.gamblet_plan_check(q, rho, rule)
    assert c["levels"] == q - 1
    assert c["phase1_entries"] > 0 and c["phase1_items"] > 0 and c["phase2_incidences"] > 0
    # every level stencil has its zero offset in the half-plane, and the
    # finest one (the Q1 3 x 3 block stencil) contributes (9 + 1) / 2
    assert c["half_offsets"] >= 5 + (q - 2)


def test_plan_check_rejects_invalid_arguments(nv):
    for q, rho, rule in ((1, 3.0, 0), (13, 3.0, 0), (6, 0.0, 0), (6, 3.0, 2)):
        with pytest.raises(nv.GambletError) as e:
            nv.gamblet_plan_check(q, rho, rule)
        assert e.value.status == nv.ERR_INVALID_ARG
