"""GPU parity of the float-float finest-level sweeps (mg_options.ff_sweeps) against the
oracle.

The option keeps every vector and the whole setup in FP64 and evaluates the finest
level's Jacobi and residual sweeps (Alg. 1's smoothing update and residual, in-situ
bilinear stencils of Sect. 4) as sums h + l of two binary32 numbers: each result carries
a few 2^-46 of the sum of its absolute terms instead of a few 2^-53.  Single sweeps and
residuals must still match the oracle within 1e-12 relative; V-cycles within
u (2^7 C1 + C2 F) (the C1 term of the FP64 bound grows with the sweep rounding, the
Galerkin term C2 F does not).  Solves run float-float cycles down to 1000 x the tolerance
and FP64 cycles after: they take the oracle's cycle count and end within the same bound.  Cases span several
bricks (2D level 4: 9 bricks of 27^2, level 5: 81; 3D level 3: 27 bricks of 9^3) and the
bricks' padded tails, the adaptive composite grid (hanging vertices on the finest level)
and the timed full-size workload.
"""
import numpy as np
import pytest

from tests.gpu_common import HIST_RTOL, Case, full_size_checker_solve, lib, parity_check, rel_inf
from tests.test_gpu_composite import Comp

pytestmark = pytest.mark.gpu

TOL = 1e-12

CASES = [(2, 4, "checker"), (2, 4, "grf"), (2, 5, "grf"), (3, 3, "sphere"), (3, 3, "grf")]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: "-".join(map(str, c)))
def case(request):
    dim, L, eps = request.param
    return Case(dim, L, eps, ff_sweeps=1)


@pytest.mark.parametrize("nu", [1, 2, 3])
def test_ff_sweeps_match_oracle(case, nu):
    L = case.L
    u = case.random_vec(L, 10 + nu)
    ud = case.dev(u)
    case.H.smooth(L, ud, case.b_dev, nu)
    assert rel_inf(case.host(ud), case.O.smooth(L, u, case.b, nu)) < TOL


def test_ff_residual_and_norm_match(case):
    L = case.L
    u = case.random_vec(L, 30)
    b = case.random_vec(L, 40)
    r = case.torch.zeros(case.n(L), dtype=case.torch.float64, device="cuda")
    n2 = case.H.residual(L, case.dev(u), case.dev(b), r, want_norm=True)
    ref = case.O.residual(L, u, b)
    assert rel_inf(case.host(r), ref) < TOL
    assert abs(n2 - float(ref @ ref)) <= 1e-12 * float(ref @ ref)


@pytest.mark.parametrize("dim,L", [(2, 4), (3, 3)])
def test_ff_path_is_taken(dim, L):
    # the option changes the finest level's arithmetic (the last bits of a sweep differ
    # from the FP64 kernel's) and nothing coarser (level L - 1 sweeps are bit-identical)
    c64 = Case(dim, L, "grf", oracle=False)
    cff = Case(dim, L, "grf", oracle=False, ff_sweeps=1)
    for lv, same in ((L, False), (L - 1, True)):
        u = c64.random_vec(lv, 7)
        b = c64.random_vec(lv, 8)
        a1, a2 = c64.dev(u), cff.dev(u)
        c64.H.smooth(lv, a1, c64.dev(b), 2)
        cff.H.smooth(lv, a2, cff.dev(b), 2)
        x, y = c64.host(a1), cff.host(a2)
        assert np.array_equal(x, y) == same, lv
        assert rel_inf(y, x) < TOL


def test_ff_vcycle_matches(case):
    u = case.random_vec(case.L, 80)
    ud = case.dev(u)
    case.H.vcycle(ud, case.b_dev)
    parity_check(f"ff vcycle {case.dim}d-l{case.L}-{case.O.transfer}", rel_inf(case.host(ud),
                 case.O.vcycle(u, case.b)), case.amplification(), "ff_cycle")


def test_ff_solve_matches_oracle(case):
    u = case.torch.zeros(case.n(case.L), dtype=case.torch.float64, device="cuda")
    res = case.H.solve(u, case.b_dev, rel_tol=1e-10, max_cycles=400)
    ref, hist = case.O.solve(case.b, 1e-10, 400)
    assert res["cycles"] == len(hist) - 1
    assert res["rel_residual"] <= 1e-10
    parity_check(f"ff solve {case.dim}d-l{case.L}", rel_inf(case.host(u), ref), case.amplification(), "ff_solve")
    # residuals of float-float cycles carry ~2^-47 of sum |A| |u| / |b| absolute rounding
    assert np.allclose(res["history"], hist[1:] / hist[0], rtol=HIST_RTOL, atol=1e-11)


@pytest.mark.parametrize("dim,L", [(2, 4), (3, 3)])
def test_ff_composite_solve_matches_oracle(dim, L):
    # adaptive grid: the finest level holds hanging vertices (their values come from the
    # coarser level and pass through the sweep unchanged)
    comp = Comp(dim, L, ff_sweeps=1)
    torch = comp.torch
    ud = torch.zeros(comp.grid.n_slots_total(), dtype=torch.float64, device="cuda")
    bd = torch.from_numpy(comp.concat(comp.b5, comp.b4)).cuda()
    res = comp.H.solve(ud, bd, rel_tol=1e-10, max_cycles=400)
    u5, u4, hist = comp.C.solve(comp.b5, comp.b4, 1e-10, 400)
    assert res["cycles"] == len(hist) - 1
    g5, g4 = comp.split(ud)
    scale = max(np.abs(u5).max(), np.abs(u4).max())
    err = max(np.abs(g5 - u5)[comp.C.dof5].max(), np.abs(g4 - u4)[comp.C.unref4].max())
    parity_check(f"ff composite solve {dim}d-l{L}", err / scale, comp.amplification(), "ff_composite_solve")


def test_ff_full_size_config2_solve_matches_oracle():
    # the timed workload: 2D level 6 (529,984 DoFs), 9x9 checkerboard {1, 1e-4}, BoxMG +
    # Galerkin, V(2,2), solved to a 1e-10 drop with float-float finest sweeps
    c, ref, hist = full_size_checker_solve()
    mg = lib()
    H = mg.Hierarchy(c.grid, ff_sweeps=1)
    H.setup(c.eps_dev)
    u = c.torch.zeros(c.n(6), dtype=c.torch.float64, device="cuda")
    res = H.solve(u, c.b_dev, rel_tol=1e-10, max_cycles=400)
    assert res["cycles"] == len(hist) - 1, (res["cycles"], len(hist) - 1)
    assert res["rel_residual"] <= 1e-10
    parity_check("ff solve 2d-l6-checker (full size)", rel_inf(c.host(u), ref), c.amplification(), "ff_solve")
    # (float-float cycles alone stall near 1.1e-10 here, their residual floor: the solve
    # reaches the tolerance through its FP64 cycles)


def test_ff_option_rules():
    mg = lib()
    g = mg.Grid(2, 4)
    with pytest.raises(mg.MgError):
        mg.Hierarchy(g, precision="mixed_bf16", ff_sweeps=1)
    with pytest.raises(mg.MgError):
        mg.Hierarchy(g, ff_sweeps=2)
    # the block smoother keeps FP64 sweeps (its Jacobi part skips the iota vertices)
    c = Case(2, 4, "grf", smoother="block", ff_sweeps=1)
    u = c.random_vec(4, 5)
    ud = c.dev(u)
    c.H.smooth(4, ud, c.b_dev, 1)
    assert rel_inf(c.host(ud), c.O.smooth(4, u, c.b, 1)) < TOL
