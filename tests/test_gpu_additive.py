"""GPU parity of the additive multigrid (Alg. 2) against the CPU oracle: traversals
(mg_vcycle of an additive hierarchy, on its stored coarse iterates and corrections) and
solves, FP64, within the tolerances of the V-cycle tests."""
import numpy as np
import pytest

from tests.gpu_common import Case, lib, parity_check, rel_inf

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.mark.parametrize("dim,L,eps,transfer,coarse", [
    (2, 4, "checker", "boxmg", "galerkin"),
    (2, 4, "const", "dlinear", "redisc"),
    (3, 3, "sphere", "boxmg", "galerkin"),
    (3, 3, "grf", "dlinear", "galerkin"),
])
def test_traversals_match_oracle(dim, L, eps, transfer, coarse):
    c = Case(dim, L, eps, transfer=transfer, coarse=coarse)
    H = c.mg.Hierarchy(c.grid, transfer=transfer, coarse=coarse, cycle="additive")
    H.setup(c.eps_dev)
    u0 = c.random_vec(L, 11)
    ud = c.dev(u0)
    O = c.O
    u = {lv: np.zeros(O.ops[lv].dof.size) for lv in range(O.coarsest, L + 1)}
    u[L] = u0.copy()
    d = {lv: np.zeros_like(u[lv]) for lv in u}
    for it in range(3):
        H.vcycle(ud, c.b_dev)
        O.additive_traversal(u, d, c.b)
        parity_check(f"additive traversal {dim}d-l{L}-{eps}", rel_inf(c.host(ud), u[L]), c.amplification(), "cycle")


@pytest.mark.parametrize("dim,L,eps", [(2, 4, "checker"), (2, 5, "grf"), (3, 3, "grf")])
def test_additive_solve_matches_oracle(dim, L, eps):
    c = Case(dim, L, eps, omega=0.8)
    H = c.mg.Hierarchy(c.grid, cycle="additive", omega=0.8)
    H.setup(c.eps_dev)
    u = c.torch.zeros(c.n(L), dtype=c.torch.float64, device="cuda")
    res = H.solve(u, c.b_dev, rel_tol=1e-10, max_cycles=2000)
    _, hist = c.O.additive_solve(c.b, rel_tol=1e-10, max_cycles=2000)
    assert res["rel_residual"] <= 1e-10
    assert abs(res["cycles"] - (len(hist) - 1)) <= 1
    assert rel_inf(c.host(u), c.O.direct(c.b)) < 1e-8


def test_additive_rejections():
    mg = lib()
    grid = mg.Grid(2, 3)
    with pytest.raises(mg.MgError):
        mg.Hierarchy(grid, cycle="additive", precision="mixed_bf16")
    with pytest.raises(mg.MgError):
        mg.Hierarchy(grid, cycle="additive", smoother="block")
    with pytest.raises(mg.MgError):
        mg.Server(1 << 30, cycle="additive")
    c = Case(2, 3, "grf", oracle=False)
    H = mg.Hierarchy(c.grid, cycle="additive")
    H.setup(c.eps_dev)
    with pytest.raises(mg.MgError):
        mg.Batch([H])
