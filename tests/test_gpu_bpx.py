"""GPU parity of the BPX traversal (Alg. 3) against the CPU oracle: traversals (mg_vcycle
of a BPX hierarchy, on its stored coarse iterates, corrections and injected c-point
updates) and solves, FP64, within the bounds of the V-cycle tests."""
import numpy as np
import pytest

from tests.gpu_common import Case, lib, parity_check, rel_inf

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,L,eps,transfer,coarse", [
    (2, 4, "checker", "boxmg", "galerkin"),
    (2, 4, "const", "dlinear", "redisc"),
    (3, 3, "sphere", "boxmg", "galerkin"),
    (3, 3, "grf", "dlinear", "galerkin"),
])
def test_bpx_traversals_match_oracle(dim, L, eps, transfer, coarse):
    c = Case(dim, L, eps, transfer=transfer, coarse=coarse)
    H = c.mg.Hierarchy(c.grid, transfer=transfer, coarse=coarse, cycle="bpx")
    H.setup(c.eps_dev)
    u0 = c.random_vec(L, 11)
    ud = c.dev(u0)
    O = c.O
    u = {lv: np.zeros(O.ops[lv].dof.size) for lv in range(O.coarsest, L + 1)}
    u[L] = u0.copy()
    d = {lv: np.zeros_like(u[lv]) for lv in u}
    i = {lv: np.zeros_like(u[lv]) for lv in u}
    for it in range(3):
        H.vcycle(ud, c.b_dev)
        O.bpx_traversal(u, d, i, c.b)
        parity_check(f"bpx traversal {dim}d-l{L}-{eps}", rel_inf(c.host(ud), u[L]), c.amplification(), "cycle")


def test_bpx_first_traversal_leaves_c_points_to_the_coarse_levels():
    # from u = 0 one traversal changes no c-point of the finest level (their updates
    # are injected, not applied), but changes the other DoFs
    c = Case(2, 4, "grf", oracle=False)
    H = c.mg.Hierarchy(c.grid, cycle="bpx")
    H.setup(c.eps_dev)
    u = c.torch.zeros(c.n(4), dtype=c.torch.float64, device="cuda")
    H.vcycle(u, c.b_dev)
    got = c.host(u)
    co = c.grid.tables(4)["coords"]
    cp = (co[:, 0] >= 0) & np.all(co % 3 == 0, axis=1) & c.dof(4)
    assert np.all(got[cp] == 0.0)
    assert np.abs(got[c.dof(4) & ~cp]).max() > 0.0


@pytest.mark.parametrize("dim,L,eps", [(2, 4, "checker"), (2, 5, "grf"), (3, 3, "grf")])
def test_bpx_solve_matches_oracle(dim, L, eps):
    c = Case(dim, L, eps, omega=0.8)
    H = c.mg.Hierarchy(c.grid, cycle="bpx", omega=0.8)
    H.setup(c.eps_dev)
    u = c.torch.zeros(c.n(L), dtype=c.torch.float64, device="cuda")
    res = H.solve(u, c.b_dev, rel_tol=1e-10, max_cycles=3000)
    _, hist = c.O.bpx_solve(c.b, rel_tol=1e-10, max_cycles=3000)
    assert res["rel_residual"] <= 1e-10
    assert abs(res["cycles"] - (len(hist) - 1)) <= 1
    assert rel_inf(c.host(u), c.O.direct(c.b)) < 1e-8


def test_bpx_rejections():
    mg = lib()
    grid = mg.Grid(2, 3)
    with pytest.raises(mg.MgError):
        mg.Hierarchy(grid, cycle="bpx", precision="mixed_bf16")
    with pytest.raises(mg.MgError):
        mg.Hierarchy(grid, cycle="bpx", smoother="block")
