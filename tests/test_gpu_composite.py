"""Adaptive composite grid on the GPU against the oracle's composite system (Sect. 3).

A spacetree complete up to level t = L - 1 and refined to level L around a sphere
shell (the adaptive 3D workload's refinement pattern, at sizes the oracle finishes
in seconds).  The GPU composite cycle (hanging interpolation, injection, d-linear
transfer between t and L, one V-cycle of the uniform levels t .. c) must give the
oracle's iterate up to FP64 rounding amplified by the Galerkin cancellation of
the coarse levels; solves must take the oracle's cycle count and reach the exact
composite solution; the mixed path must reach it within 1e-8.
"""
import numpy as np
import pytest

from oracle import composite
from oracle import spacetree as stt
import synthetic as syn
from tests.gpu_common import HIST_ATOL, HIST_RTOL, galerkin_amplification, lib, parity_bound, parity_check, rel_inf

pytestmark = pytest.mark.gpu

TOL = 1e-12


class Comp:
    def __init__(self, dim, L, precision="fp64", eps_kind="sphere", seed=0, **hier_options):
        import torch

        self.torch = torch
        self.mg = mg = lib()
        self.dim, self.L, self.T = dim, L, L - 1
        T = self.T
        c = (0.5, 0.5, 0.5)[:dim]
        mask = syn.sphere_shell_mask(T, dim, radius=0.3, centre=c)
        self.tree = stt.Spacetree(dim, L, {T: mask})
        if eps_kind == "sphere":
            self.eps = {L: syn.sphere_eps(L, dim, centre=c), T: syn.sphere_eps(T, dim, centre=c)}
        else:
            self.eps = {lv: syn.lognormal_grf_eps(lv, dim, sigma=2.0, seed=seed + lv) for lv in (L, T)}
        self.C = composite.Composite(self.tree, self.eps)
        self.grid = mg.Grid(dim, L, {T: mask})
        self.H = mg.Hierarchy(self.grid, precision=precision, **hier_options)
        self.H.setup(torch.from_numpy(self.grid.cells_to_concat(self.eps)).cuda())
        self.oL, self.nL = self.grid.info(L).slot_offset, self.grid.info(L).n_slots
        self.oT, self.nT = self.grid.info(T).slot_offset, self.grid.info(T).n_slots
        self.b5 = self.tree.vertices_to_slots(L, syn.uniform_load(L, dim, seed + 2))
        self.b4 = np.where(self.C.unref4, self.tree.vertices_to_slots(T, syn.uniform_load(T, dim, seed + 3)), 0.0)

    def concat(self, v5, v4):
        out = np.zeros(self.grid.n_slots_total())
        out[self.oL: self.oL + self.nL] = v5
        out[self.oT: self.oT + self.nT] = v4
        return out

    def split(self, t):
        self.torch.cuda.synchronize()
        a = t.cpu().numpy()
        return a[self.oL: self.oL + self.nL], a[self.oT: self.oT + self.nT]

    def amplification(self):
        return galerkin_amplification(self.C.sub, stt.Spacetree(self.dim, self.T), self.T, self.dim)


CASES = [(2, 4), (3, 3)]


@pytest.fixture(scope="module", params=CASES, ids=lambda p: f"{p[0]}d-L{p[1]}")
def comp(request):
    return Comp(*request.param)


def test_hierarchy_levels_and_tables(comp):
    g = comp.grid
    # the grid is adaptive: level L holds hanging vertices, level t refined and unrefined DoFs
    assert (g.tables(comp.L)["vflags"] & 4).any()
    assert comp.C.ref4.any() and comp.C.unref4.any()
    assert np.array_equal(g.tables(comp.L)["vflags"], comp.tree.levels[comp.L].vflags)


def test_hanging_interpolation_matches(comp):
    torch = comp.torch
    rng = np.random.default_rng(7)
    u4 = np.where(comp.C.unref4, rng.standard_normal(comp.nT), 0.0)
    u5 = rng.standard_normal(comp.nL)
    d5 = torch.from_numpy(u5.copy()).cuda()
    comp.H.interpolate_hanging(comp.L, torch.from_numpy(u4).cuda(), d5)
    got = d5.cpu().numpy()
    hang = (comp.tree.levels[comp.L].vflags & stt.HANGING) != 0
    ref = comp.C.Hmat @ u4
    assert hang.sum() > 0
    assert np.abs(got[hang] - ref[hang]).max() <= 4 * 2.0**-53 * np.abs(u4).max()
    assert np.array_equal(got[~hang], u5[~hang])


def test_composite_cycle_matches(comp):
    torch = comp.torch
    rng = np.random.default_rng(11)
    u5 = np.where(comp.C.dof5, rng.standard_normal(comp.nL), 0.0)
    u4 = np.where(comp.C.unref4, rng.standard_normal(comp.nT), 0.0)
    ud = torch.from_numpy(comp.concat(u5, u4)).cuda()
    bd = torch.from_numpy(comp.concat(comp.b5, comp.b4)).cuda()
    comp.H.vcycle(ud, bd)
    g5, g4 = comp.split(ud)
    r5, r4 = comp.C.cycle(u5, u4, comp.b5, comp.b4)
    scale = max(np.abs(r5).max(), np.abs(r4).max())
    amp = comp.amplification()
    tol = parity_bound(amp, "composite_cycle") * scale
    err = max(np.abs(g5 - np.where(comp.C.dof5, r5, 0.0))[comp.C.dof5].max(), np.abs(g4 - r4)[comp.C.unref4].max())
    parity_check(f"composite cycle {comp.dim}d-l{comp.L}", err / scale, amp, "composite_cycle")
    # on return the level-L hanging and the refined level-t entries hold the filled values
    f5, f4 = comp.C.fill(r5, r4)
    hang = (comp.tree.levels[comp.L].vflags & stt.HANGING) != 0
    assert np.abs(g5 - f5)[hang].max() <= tol
    assert np.abs(g4 - f4)[comp.C.ref4].max() <= tol


def test_composite_solve_matches_oracle(comp):
    torch = comp.torch
    ud = torch.zeros(comp.grid.n_slots_total(), dtype=torch.float64, device="cuda")
    bd = torch.from_numpy(comp.concat(comp.b5, comp.b4)).cuda()
    res = comp.H.solve(ud, bd, rel_tol=1e-10, max_cycles=400)
    u5, u4, hist = comp.C.solve(comp.b5, comp.b4, 1e-10, 400)
    assert res["cycles"] == len(hist) - 1
    assert res["rel_residual"] <= 1e-10
    g5, g4 = comp.split(ud)
    scale = max(np.abs(u5).max(), np.abs(u4).max())
    amp = comp.amplification()
    err = max(np.abs(g5 - u5)[comp.C.dof5].max(), np.abs(g4 - u4)[comp.C.unref4].max())
    parity_check(f"composite solve {comp.dim}d-l{comp.L}", err / scale, amp, "composite_solve")
    hg, ho = np.asarray(res["history"]), hist[1:] / hist[0]
    dev = np.abs(hg - ho) - HIST_RTOL * np.abs(ho)
    assert np.all(dev <= HIST_ATOL), (f"history: worst |gpu - oracle| - rtol |oracle| = {dev.max():.3e} at "
                                      f"{int(dev.argmax())} of {len(ho)} (value {ho[dev.argmax()]:.3e})")
    # and the exact composite solution
    d5, d4 = comp.C.direct(comp.b5, comp.b4)
    ds = max(np.abs(d5).max(), np.abs(d4).max())
    assert np.abs(g5 - d5)[comp.C.dof5].max() <= 1e-8 * ds
    assert np.abs(g4 - d4)[comp.C.unref4].max() <= 1e-8 * ds


@pytest.mark.parametrize("precision", ["mixed_bf16", "mixed_fp16", "mixed_bpa"])
@pytest.mark.parametrize("dim,L", CASES)
def test_composite_mixed_solve_reaches_fp64_solution(dim, L, precision):
    c = Comp(dim, L, precision=precision, eps_kind="grf", seed=5)
    torch = c.torch
    ud = torch.zeros(c.grid.n_slots_total(), dtype=torch.float64, device="cuda")
    bd = torch.from_numpy(c.concat(c.b5, c.b4)).cuda()
    res = c.H.solve(ud, bd, rel_tol=1e-10, max_cycles=3000)
    assert res["rel_residual"] <= 1e-10
    g5, g4 = c.split(ud)
    g5 = np.where(c.C.dof5, g5, 0.0)
    g4 = np.where(c.C.unref4, g4, 0.0)
    r5, r4 = c.C.residual(g5, g4, c.b5, c.b4)
    r0 = np.sqrt(c.b5[c.C.dof5] @ c.b5[c.C.dof5] + c.b4[c.C.unref4] @ c.b4[c.C.unref4])
    assert np.sqrt(r5 @ r5 + r4 @ r4) <= 1.0001e-10 * r0
    d5, d4 = c.C.direct(c.b5, c.b4)
    ds = max(np.abs(d5).max(), np.abs(d4).max())
    assert max(np.abs(g5 - d5).max(), np.abs(g4 - d4).max()) <= 1e-8 * ds


def test_adaptive_entry_points_reject_what_they_do_not_cover(comp):
    torch = comp.torch
    u = torch.zeros(comp.nL, dtype=torch.float32, device="cuda")
    with pytest.raises(RuntimeError):
        comp.H.vcycle_f32(u, u)


def test_full_size_sphere3d_l5_solves_reach_the_oracle_residual():
    # the adaptive 3D workload at full size: uniform to level 4 (81^3 cells) and level 5
    # in the shell around r = 0.3 (1,287,488 composite unknowns).  The oracle's composite
    # system (no cycle) evaluates the residual of the GPU solutions: both the FP64 and
    # the mixed BF16 solve must reach the 1e-10 drop in the oracle's arithmetic.
    import torch

    mg = lib()
    dim, L, T = 3, 5, 4
    mask = syn.sphere_shell_mask(T, dim, radius=0.3)
    eps = {L: syn.sphere_eps(L, dim), T: syn.sphere_eps(T, dim)}
    tree = stt.Spacetree(dim, L, {T: mask})
    C = composite.Composite(tree, eps, cycle=False)
    b5 = tree.vertices_to_slots(L, syn.uniform_load(L, dim, 2))
    b4 = np.where(C.unref4, tree.vertices_to_slots(T, syn.uniform_load(T, dim, 3)), 0.0)
    assert C.dof5.sum() + C.unref4.sum() == 1287488
    grid = mg.Grid(dim, L, {T: mask})
    iL, iT = grid.info(L), grid.info(T)
    cat = np.zeros(grid.n_slots_total())
    cat[iL.slot_offset: iL.slot_offset + iL.n_slots] = b5
    cat[iT.slot_offset: iT.slot_offset + iT.n_slots] = b4
    bd = torch.from_numpy(cat).cuda()
    eps_dev = torch.from_numpy(grid.cells_to_concat(eps)).cuda()
    r0 = np.sqrt(b5[C.dof5] @ b5[C.dof5] + b4[C.unref4] @ b4[C.unref4])
    for precision in ("fp64", "mixed_bf16"):
        H = mg.Hierarchy(grid, precision=precision)
        H.setup(eps_dev)
        ud = torch.zeros_like(bd)
        res = H.solve(ud, bd, rel_tol=1e-10, max_cycles=3000)
        a = ud.cpu().numpy()
        u5 = np.where(C.dof5, a[iL.slot_offset: iL.slot_offset + iL.n_slots], 0.0)
        u4 = np.where(C.unref4, a[iT.slot_offset: iT.slot_offset + iT.n_slots], 0.0)
        r5, r4 = C.residual(u5, u4, b5, b4)
        # two FP64 evaluations of b - A u differ by at most (terms) u sum|terms| per row (Higham)
        f5, f4 = C.fill(u5, u4)
        n5 = np.where(C.dof5, np.abs(b5) + abs(C.A5) @ np.abs(f5), 0.0)
        n4 = np.where(C.unref4, np.abs(b4) + abs(C.A4) @ np.abs(f4), 0.0)
        noise = 64 * 2.0**-53 * np.sqrt(n5 @ n5 + n4 @ n4)
        assert res["rel_residual"] <= 1e-10
        assert np.sqrt(r5 @ r5 + r4 @ r4) <= 1e-10 * r0 + noise, precision
        del H
