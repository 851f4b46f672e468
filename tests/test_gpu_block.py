"""GPU parity of the block Jacobi smoother (Sect. 4.2) against the CPU oracle.

A block step = Gauss-Seidel sweeps over the iota vertices of every 3^d patch (in place,
lexicographic within the patch), then the damped Jacobi sweep of the other DoFs with
the iota values kept.  FP64 steps, cycles and solves match the oracle's block smoother
within the FP64 tolerances of the Jacobi tests; mixed and composite solves reach the
FP64 discrete solution."""
import numpy as np
import pytest

from tests.gpu_common import parity_check, Case, lib, rel_inf

pytestmark = pytest.mark.gpu

TOL = 1e-12

CASES = [(2, 4, "checker"), (2, 4, "grf"), (3, 3, "sphere"), (3, 3, "grf")]


@pytest.mark.parametrize("gs", [1, 3])
@pytest.mark.parametrize("dim,L,eps", CASES)
def test_block_steps_match_oracle(dim, L, eps, gs):
    c = Case(dim, L, eps, smoother="block", gs_sweeps=gs)
    for lv, nu in ((L, 1), (L, 2), (L - 1, 2), (2, 1)):
        u = c.random_vec(lv, 30 + lv)
        b = c.random_vec(lv, 40 + lv) if lv < L else c.b
        ud = c.dev(u)
        c.H.smooth(lv, ud, c.dev(b), nu)
        ref = c.O.smooth(lv, u, b, nu)
        parity_check(f"block step {dim}d-l{L}-{eps}", rel_inf(c.host(ud), ref), c.amplification(), "cycle")


@pytest.mark.parametrize("dim,L,eps", CASES[:3])
def test_block_cycle_and_solve_match_oracle(dim, L, eps):
    c = Case(dim, L, eps, smoother="block")
    u = c.random_vec(L, 7)
    ud = c.dev(u)
    c.H.vcycle(ud, c.b_dev)
    parity_check(f"block vcycle {dim}d-l{L}-{eps}", rel_inf(c.host(ud), c.O.vcycle(u, c.b)), c.amplification(),
                 "cycle")
    ud = c.torch.zeros(c.n(L), dtype=c.torch.float64, device="cuda")
    res = c.H.solve(ud, c.b_dev, rel_tol=1e-10, max_cycles=500)
    _, hist = c.O.solve(c.b, rel_tol=1e-10, max_cycles=500)
    assert res["rel_residual"] <= 1e-10
    assert abs(res["cycles"] - (len(hist) - 1)) <= 1
    assert rel_inf(c.host(ud), c.O.direct(c.b)) < 1e-8


@pytest.mark.parametrize("prec", ["mixed_bf16", "mixed_bpa"])
@pytest.mark.parametrize("dim,L,eps", [(2, 5, "checker"), (3, 3, "sphere")])
def test_block_mixed_solve_reaches_fp64_solution(dim, L, eps, prec):
    c = Case(dim, L, eps, precision=prec, smoother="block", gs_sweeps=2)
    u = c.torch.zeros(c.n(L), dtype=c.torch.float64, device="cuda")
    res = c.H.solve(u, c.b_dev, rel_tol=1e-10, max_cycles=2000)
    assert res["rel_residual"] <= 1e-10
    ug = c.host(u)
    r = c.O.residual(L, ug, c.b)
    assert np.linalg.norm(r) <= 1.0001e-10 * np.linalg.norm(c.b)
    assert rel_inf(ug, c.O.direct(c.b)) <= 1e-8


@pytest.mark.parametrize("precision", ["fp64", "mixed_bf16"])
def test_block_composite_solve(precision):
    from tests.test_gpu_composite import Comp

    c = Comp(2, 4, precision=precision, eps_kind="grf", seed=5, smoother="block")
    torch = c.torch
    ud = torch.zeros(c.grid.n_slots_total(), dtype=torch.float64, device="cuda")
    bd = torch.from_numpy(c.concat(c.b5, c.b4)).cuda()
    res = c.H.solve(ud, bd, rel_tol=1e-10, max_cycles=3000)
    assert res["rel_residual"] <= 1e-10
    g5, g4 = c.split(ud)
    g5 = np.where(c.C.dof5, g5, 0.0)
    g4 = np.where(c.C.unref4, g4, 0.0)
    d5, d4 = c.C.direct(c.b5, c.b4)
    ds = max(np.abs(d5).max(), np.abs(d4).max())
    assert max(np.abs(g5 - d5).max(), np.abs(g4 - d4).max()) <= 1e-8 * ds


def test_full_size_config2_block_step():
    # 2D level 6 (529,984 DoFs), the checkerboard workload: one block step with one
    # Gauss-Seidel sweep per patch, element by element against the oracle
    c = Case(2, 6, "checker", smoother="block")
    u = c.random_vec(6, 99)
    ud = c.dev(u)
    c.H.smooth(6, ud, c.b_dev, 1)
    assert rel_inf(c.host(ud), c.O.smooth(6, u, c.b, 1)) < TOL


def test_block_hierarchies_are_single_problem():
    mg = lib()
    c = Case(2, 3, "grf", smoother="block", oracle=False)
    with pytest.raises(mg.MgError):
        mg.Batch([c.H])
    with pytest.raises(mg.MgError):
        mg.Server(1 << 30, smoother="block")
    with pytest.raises(mg.MgError):
        mg.Hierarchy(c.grid, smoother="block", gs_sweeps=0)
