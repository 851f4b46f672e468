"""GPU parity of the dynamic coarsest level (Sect. 4.3) against the oracle: the level the
setup's audit chooses, solves with it (the oracle's cycle count and iterate), the
stagnation rule between cycles, and the error when no admissible level exists."""
import numpy as np
import pytest

from oracle import multigrid
from oracle import spacetree as stt
from tests.gpu_common import Case, galerkin_amplification, lib, parity_check, rel_inf

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,L,eps", [(2, 4, "grf"), (2, 5, "grf"), (2, 4, "const"), (2, 4, "checker")])
def test_dynamic_coarsest_level_matches_oracle(dim, L, eps):
    c = Case(dim, L, eps, oracle=False)
    H = c.mg.Hierarchy(c.grid, dynamic_coarsest=1)
    H.setup(c.eps_dev)
    tree = stt.Spacetree(dim, L)
    O = multigrid.Hierarchy(tree, {L: c.eps}, dynamic_coarsest=True)
    assert H.coarsest() == O.coarsest
    u = c.torch.zeros(c.n(L), dtype=c.torch.float64, device="cuda")
    res = H.solve(u, c.b_dev, rel_tol=1e-10, max_cycles=400)
    ref, hist = O.solve(c.b, 1e-10, 400)
    assert res["cycles"] == len(hist) - 1
    assert H.coarsest() == O.coarsest
    parity_check(f"dynamic solve {dim}d-l{L}-{eps}", rel_inf(c.host(u), ref),
                 galerkin_amplification(O, tree, L, dim), "solve")


def test_stagnation_raises_the_coarsest_level_like_the_oracle():
    # omega = 0.01: the first cycles reduce the residual by less than 1/0.95, so the
    # coarsest level is raised between cycles up to the largest admissible one (level 3,
    # 676 unknowns); the ratios stay at least 0.007 away from 0.95 (robust decisions)
    c = Case(2, 4, "const", omega=0.01, oracle=False)
    H = c.mg.Hierarchy(c.grid, dynamic_coarsest=1, omega=0.01)
    H.setup(c.eps_dev)
    assert H.coarsest() == 1
    tree = stt.Spacetree(2, 4)
    O = multigrid.Hierarchy(tree, {4: c.eps}, omega=0.01, dynamic_coarsest=True)
    u = c.torch.zeros(c.n(4), dtype=c.torch.float64, device="cuda")
    res = H.solve(u, c.b_dev, rel_tol=1e-8, max_cycles=3000)
    ref, hist = O.solve(c.b, 1e-8, 3000)
    assert O.coarsest == 3 and H.coarsest() == 3
    assert res["cycles"] == len(hist) - 1
    parity_check("dynamic solve with raises 2d-l4-const", rel_inf(c.host(u), ref), 1.0, "solve")
    # a second solve starts again from the level of the setup
    u.zero_()
    res2 = H.solve(u, c.b_dev, rel_tol=1e-8, max_cycles=3000)
    assert res2["cycles"] == res["cycles"]


def test_no_admissible_coarsest_level_is_reported():
    # 3D level 3 on the sphere coefficient: the level-2 Galerkin operator is not
    # diagonally dominant, so the coarsest level would have to be the finest one
    mg = lib()
    c = Case(3, 3, "sphere", oracle=False)
    H = mg.Hierarchy(c.grid, dynamic_coarsest=1)
    with pytest.raises(mg.MgError) as e:
        H.setup(c.eps_dev)
    assert e.value.status == 7
    with pytest.raises(ValueError):
        multigrid.Hierarchy(stt.Spacetree(3, 3), {3: c.eps}, dynamic_coarsest=True)


def test_dynamic_coarsest_is_rejected_where_it_cannot_run():
    mg = lib()
    g = mg.Grid(2, 4)
    H = mg.Hierarchy(g, dynamic_coarsest=1)
    with pytest.raises(mg.MgError):
        mg.Hierarchy(g, dynamic_coarsest=1, cycle="additive")
    with pytest.raises(mg.MgError):
        mg.Server(1 << 30, dynamic_coarsest=1)
    del H
