"""Pins of the oracle's dynamic coarsest level (Sect. 4.3): the definiteness / diagonal
dominance check of a level operator, the raise to the level above the finest failing
level, the stagnation rule between cycles, and solves with the raised coarsest level."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import multigrid
from oracle import spacetree as stt
import synthetic as syn


def test_audit_rows_by_hand():
    # tridiagonal [-1 2 -1]: interior rows weakly dominant (2 = 1 + 1), end rows strictly
    A = sp.diags([[-1.0] * 3, [2.0] * 4, [-1.0] * 3], [-1, 0, 1]).tocsr()
    assert not multigrid.audit_rows(A, np.ones(4, bool)).any()
    # off-diagonal 1.5 against a diagonal 1: not dominant
    B = sp.csr_matrix(np.array([[1.0, -1.5], [-1.5, 1.0]]))
    assert multigrid.audit_rows(B, np.ones(2, bool)).all()
    # non-positive diagonals fail even without off-diagonal entries
    C = sp.csr_matrix(np.diag([-1.0, 0.0, 3.0]))
    assert multigrid.audit_rows(C, np.ones(3, bool)).tolist() == [True, True, False]
    # rounding allowance: 1 + 1e-14 against 1 passes, 1 + 1e-9 fails
    D = sp.csr_matrix(np.array([[1.0, -(1.0 + 1e-14)], [-(1.0 + 1e-9), 1.0]]))
    assert multigrid.audit_rows(D, np.ones(2, bool)).tolist() == [False, True]
    # rows that are no unknowns are not checked
    assert not multigrid.audit_rows(B, np.zeros(2, bool)).any()


def test_raise_and_stall_rules():
    assert multigrid.raised_coarsest([], 1) == 1
    assert multigrid.raised_coarsest([2], 1) == 3
    assert multigrid.raised_coarsest([1, 3], 2) == 4
    assert not multigrid.stalled([1.0])
    assert not multigrid.stalled([1.0, 0.5])
    assert multigrid.stalled([1.0, 0.96])
    assert multigrid.stalled([1.0, 1.2])


@pytest.mark.parametrize("dim,L", [(2, 4), (3, 3)])
def test_constant_coefficient_keeps_the_coarsest_level(dim, L):
    # constant eps: Galerkin operators equal the rediscretised ones, whose rows are
    # weakly diagonally dominant (a zero row sum with non-positive off-diagonals)
    t = stt.Spacetree(dim, L)
    H = multigrid.Hierarchy(t, {L: syn.constant_eps(L, dim)}, dynamic_coarsest=True)
    assert H.failing_levels == [] and H.coarsest == 1


def test_rough_coefficient_raises_to_the_level_above_the_failing_one():
    t = stt.Spacetree(2, 4)
    eps = syn.lognormal_grf_eps(4, 2, sigma=2.0, seed=1000)
    H = multigrid.Hierarchy(t, {4: eps}, dynamic_coarsest=True)
    assert H.failing_levels == [2] and H.coarsest == 3
    # the failing level has a row whose off-diagonal magnitudes exceed its diagonal
    A = H.ops[2].A.tocsr()
    row = np.nonzero(multigrid.audit_rows(A, H.ops[2].dof))[0][0]
    d = A[row, row]
    assert np.abs(A[row]).sum() - abs(d) > d > 0
    # and the solve with the raised coarsest level reaches the direct solution
    b = t.vertices_to_slots(4, syn.uniform_load(4, 2, 2000))
    u, hist = H.solve(b, 1e-10, 200)
    assert hist[-1] <= 1e-10 * hist[0]
    ref = H.direct(b)
    assert np.abs(u - ref).max() <= 1e-8 * np.abs(ref).max()


def test_no_admissible_coarsest_level_is_an_error():
    t = stt.Spacetree(2, 4)
    eps = syn.lognormal_grf_eps(4, 2, sigma=2.0, seed=1000)
    with pytest.raises(ValueError):
        multigrid.Hierarchy(t, {4: eps}, dynamic_coarsest=True, max_coarse_dofs=100)
