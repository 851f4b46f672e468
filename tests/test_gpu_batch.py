"""Batched solves: every problem of a batch gives what it gives alone.

A batch advances problems of different sizes through their V-cycles in lockstep;
the per-vertex arithmetic is the same kernels' as a single solve, so each FP64
problem must take the same number of cycles and reach the same iterate as when
solved alone (1e-12 relative), and mixed-precision problems must reach the FP64
tolerance and the stated 1e-8 error against the exact discrete solution.
"""
import numpy as np
import pytest

from oracle import multigrid
from oracle import spacetree as stt
import synthetic as syn
from tests.gpu_common import lib, rel_inf

pytestmark = pytest.mark.gpu


def _problem(mg, torch, dim, L, seed, precision):
    eps = syn.lognormal_grf_eps(L, dim, sigma=2.0, seed=1000 + seed)
    g = mg.Grid(dim, L)
    H = mg.Hierarchy(g, precision=precision)
    eps_dev = torch.from_numpy(g.cells_to_concat({L: eps})).cuda()
    H.setup(eps_dev)
    b = g.to_slots(L, syn.uniform_load(L, dim, 2000 + seed))
    return dict(g=g, H=H, eps=eps, eps_dev=eps_dev, b=b, b_dev=torch.from_numpy(b).cuda(), L=L, dim=dim)


SIZES_2D = [3, 5, 4, 3, 5, 4, 3]


@pytest.mark.parametrize("dim,levels", [(2, SIZES_2D), (3, [2, 3, 2])])
def test_fp64_batch_equals_single_solves(dim, levels):
    mg = lib()
    import torch

    probs = [_problem(mg, torch, dim, L, i, "fp64") for i, L in enumerate(levels)]
    singles = []
    for p in probs:
        u = torch.zeros_like(p["b_dev"])
        r = p["H"].solve(u, p["b_dev"], rel_tol=1e-10, max_cycles=500)
        singles.append((r, u.cpu().numpy()))
    batch = mg.Batch([p["H"] for p in probs])
    us = [torch.full_like(p["b_dev"], float("nan")) for p in probs]
    status, stats = batch.solve(us, [p["b_dev"] for p in probs], rel_tol=1e-10, max_cycles=500)
    assert status == 0
    for (r, u1), st, u, p in zip(singles, stats, us, probs):
        assert st["cycles"] == r["cycles"]
        assert st["rel_residual"] <= 1e-10
        assert rel_inf(u.cpu().numpy(), u1) < 1e-12
    # re-running the setup of every problem as one batched setup, then a second solve
    # of the same batch (its graph is reused), gives the same answers
    batch.setup([p["eps_dev"] for p in probs])
    us2 = [torch.zeros_like(p["b_dev"]) for p in probs]
    batch.solve(us2, [p["b_dev"] for p in probs], rel_tol=1e-10, max_cycles=500)
    for a, b2 in zip(us, us2):
        assert torch.equal(a, b2)


def test_mixed_batch_reaches_fp64_solution():
    mg = lib()
    import torch

    levels = [3, 4, 5, 4]
    probs = [_problem(mg, torch, 2, L, 10 + i, "mixed_bf16") for i, L in enumerate(levels)]
    batch = mg.Batch([p["H"] for p in probs])
    us = [torch.zeros_like(p["b_dev"]) for p in probs]
    status, stats = batch.solve(us, [p["b_dev"] for p in probs], rel_tol=1e-10, max_cycles=2000)
    assert status == 0
    for p, u, st in zip(probs, us, stats):
        tree = stt.Spacetree(2, p["L"])
        O = multigrid.Hierarchy(tree, {p["L"]: p["eps"]})
        ug = u.cpu().numpy()
        r = O.residual(p["L"], ug, p["b"])
        assert np.linalg.norm(r) <= 1.0001e-10 * np.linalg.norm(p["b"])
        assert rel_inf(ug, O.direct(p["b"])) <= 1e-8


def test_batch_retires_converged_and_reports_unconverged():
    mg = lib()
    import torch

    probs = [_problem(mg, torch, 2, L, 20 + i, "fp64") for i, L in enumerate([3, 4, 4])]
    bs = [p["b_dev"] for p in probs]
    bs[1] = torch.zeros_like(bs[1])  # converged before the first cycle
    batch = mg.Batch([p["H"] for p in probs])
    us = [torch.ones_like(b) for b in bs]
    status, stats = batch.solve(us, bs, rel_tol=1e-10, max_cycles=3, raise_on_fail=False)
    assert status == 4  # MG_ERR_NOT_CONVERGED for the problems that needed more cycles
    assert stats[1]["cycles"] == 0 and float(us[1].abs().max()) == 0.0
    assert stats[0]["cycles"] == 3 and stats[2]["cycles"] == 3


@pytest.mark.parametrize("precision", ["fp64", "mixed_bf16"])
@pytest.mark.parametrize("dim,levels", [(2, SIZES_2D), (3, [2, 3, 2, 3])])
def test_persistent_batch_steps_equal_lockstep_steps(dim, levels, precision):
    # options.persistent: every step of the batch in one persistent launch over a work
    # queue with per-problem progress counters.  The entries run the lockstep schedule's
    # per-vertex arithmetic, so each problem takes the same cycles and reaches the same
    # iterate; only the norm's partial sums are added in another grouping (FP64: within
    # 1e-12; mixed: the scaling sigma moves the FP32 iterates within their own rounding)
    mg = lib()
    import torch

    res, us = {}, {}
    for persistent in (0, 1):
        probs = []
        for i, L in enumerate(levels):
            eps = syn.lognormal_grf_eps(L, dim, sigma=2.0, seed=1000 + i)
            g = mg.Grid(dim, L)
            H = mg.Hierarchy(g, precision=precision, persistent=persistent)
            e = torch.from_numpy(g.cells_to_concat({L: eps})).cuda()
            H.setup(e)
            b = torch.from_numpy(g.to_slots(L, syn.uniform_load(L, dim, 2000 + i))).cuda()
            probs.append((H, b, eps, g, L, i))
        batch = mg.Batch([p[0] for p in probs])
        u = [torch.zeros_like(p[1]) for p in probs]
        status, stats = batch.solve(u, [p[1] for p in probs], rel_tol=1e-10, max_cycles=2000)
        assert status == 0
        res[persistent], us[persistent] = stats, [x.cpu().numpy() for x in u]
        if persistent and precision == "fp64":
            for (H, b, eps, g, L, i), x in zip(probs, us[1]):
                O = multigrid.Hierarchy(stt.Spacetree(dim, L), {L: eps})
                assert rel_inf(x, O.direct(g.to_slots(L, syn.uniform_load(L, dim, 2000 + i)))) < 1e-8
    for a, b_, sa, sb in zip(us[0], us[1], res[0], res[1]):
        assert sb["rel_residual"] <= 1e-10
        if precision == "fp64":
            assert sa["cycles"] == sb["cycles"]
            assert rel_inf(b_, a) < 1e-12
        else:
            assert abs(sa["cycles"] - sb["cycles"]) <= 8  # one refinement step
            assert rel_inf(b_, a) < 1e-8
