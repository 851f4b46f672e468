"""Serving: continuous batching gives each request the result it gets alone.

Requests arrive while others are on the GPU, wait for HBM budget, join the running
batch at a step boundary and retire when they converge.  Each request's
arithmetic is its own (the batch only shares launches), so its result must equal
the result of solving it alone: FP64 against the single-problem solve (same
cycles, 1e-12), mixed against a batch holding only that request (same inner
schedule, 1e-12), and both against the exact discrete solution (1e-8).
"""
import time

import numpy as np
import pytest

from oracle import multigrid
from oracle import spacetree as stt
import synthetic as syn
from tests.gpu_common import lib, rel_inf

pytestmark = pytest.mark.gpu


def _req(mg, torch, L, seed, dim=2):
    eps = syn.lognormal_grf_eps(L, dim, sigma=1.5, seed=1000 + seed)
    g = mg.Grid(dim, L)
    b = g.to_slots(L, syn.uniform_load(L, dim, 2000 + seed))
    return dict(L=L, dim=dim, g=g, eps=eps, eps_dev=torch.from_numpy(g.cells_to_concat({L: eps})).cuda(), b=b,
                b_dev=torch.from_numpy(b).cuda())


# 2D: levels 3..5 (676 .. 58,564 DoFs); 3D: the served workload's shape at sizes the
# oracle checks quickly, levels 2..4 (512, 17,576 and 512,000 DoFs: two of the server's
# size lanes, the largest in the lane of mid-sized problems)
SHAPES = {2: [4, 3, 5, 3, 4, 5, 3], 3: [3, 2, 4, 3, 2, 3, 3]}


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("precision", ["fp64", "mixed_bf16"])
def test_served_results_equal_solo_results(precision, dim):
    mg = lib()
    import torch

    levels = SHAPES[dim]
    reqs = [_req(mg, torch, L, i, dim) for i, L in enumerate(levels)]
    # budget for about two of the largest requests at a time: the rest must queue
    budget = int(2.5 * mg.hier_footprint(reqs[2]["g"], precision=precision))
    sv = mg.Server(budget, precision=precision)
    us = [torch.full_like(r["b_dev"], float("nan")) for r in reqs]
    tickets = []
    for i, (r, u) in enumerate(zip(reqs, us)):
        tickets.append(sv.submit(r["g"], r["eps_dev"], r["b_dev"], u, rel_tol=1e-10, max_cycles=2000))
        if i == 2:
            time.sleep(0.02)  # later requests arrive while the first ones run
    results = [sv.poll(t, wait=True) for t in tickets]
    sv.close()
    for r, u, res in zip(reqs, us, results):
        assert res["status"] == 0, res
        assert res["rel_residual"] <= 1e-10
        H = mg.Hierarchy(r["g"], precision=precision)
        H.setup(r["eps_dev"])
        u1 = torch.zeros_like(r["b_dev"])
        if precision == "fp64":
            solo = H.solve(u1, r["b_dev"], rel_tol=1e-10, max_cycles=2000)
            assert solo["cycles"] == res["cycles"]
        else:
            mg.Batch([H]).solve([u1], [r["b_dev"]], rel_tol=1e-10, max_cycles=2000)
        assert rel_inf(u.cpu().numpy(), u1.cpu().numpy()) < 1e-12
        O = multigrid.Hierarchy(stt.Spacetree(dim, r["L"]), {r["L"]: r["eps"]})
        ug = u.cpu().numpy()
        if dim == 2 or r["L"] <= 3:
            assert rel_inf(ug, O.direct(r["b"])) < 1e-8
        else:  # 512,000 unknowns: the oracle's FP64 residual of the served result instead
            assert np.linalg.norm(O.residual(r["L"], ug, r["b"])) <= 1.0001e-10 * np.linalg.norm(r["b"])


def test_server_rejects_requests_beyond_its_budget():
    mg = lib()
    import torch

    r = _req(mg, torch, 4, 0)
    sv = mg.Server(mg.hier_footprint(r["g"]) // 2)  # half of what its hierarchy needs
    u = torch.zeros_like(r["b_dev"])
    with pytest.raises(mg.MgError) as e:
        sv.submit(r["g"], r["eps_dev"], r["b_dev"], u)
    assert e.value.status == 9
    assert sv.info()["queued"] == 0
    sv.close()
