"""GPU parity of diagonal-tensor coefficients (the paper's `checkerboard` benchmark,
Sect. 7: eps_i = 1 where the cell centre has x_i < 0.5, else 0.1) against the oracle's
directional element matrices: stencils of every level, finest-level sweeps and
residuals, V-cycles and solves (FP64), and the mixed solve's FP64 solution."""
import numpy as np
import pytest

from oracle import multigrid
from oracle import spacetree as stt
import synthetic as syn
from tests.gpu_common import galerkin_amplification, lib, parity_check, rel_inf

pytestmark = pytest.mark.gpu

TOL = 1e-12


class Tensor:
    def __init__(self, dim, L, precision="fp64", omega=0.6):
        import torch

        self.torch, self.mg = torch, lib()
        self.dim, self.L = dim, L
        self.e = syn.axis_checkerboard_eps(L, dim)
        self.grid = self.mg.Grid(dim, L)
        axes = np.concatenate([self.grid.cells_to_concat({L: self.e[..., i]}) for i in range(dim)])
        self.H = self.mg.Hierarchy(self.grid, precision=precision, tensor_coefficients=1, omega=omega)
        self.H.setup_tensor(torch.from_numpy(axes).cuda())
        self.tree = stt.Spacetree(dim, L)
        self.O = multigrid.Hierarchy(self.tree, {L: self.e}, omega=omega)
        self.b = self.grid.to_slots(L, syn.unit_load(L, dim))
        self.b_dev = torch.from_numpy(self.b).cuda()

    def n(self, lv):
        return self.grid.info(lv).n_slots

    def dev(self, a):
        return self.torch.from_numpy(np.ascontiguousarray(a)).cuda()

    def host(self, t):
        self.torch.cuda.synchronize()
        return t.cpu().numpy()


CASES = [(2, 4, 0.6), (3, 3, 0.5)]  # 3D: the anisotropic trilinear elements need omega < 0.55


@pytest.fixture(scope="module", params=CASES, ids=lambda c: f"{c[0]}d-l{c[1]}")
def ten(request):
    dim, L, om = request.param
    return Tensor(dim, L, omega=om)


def test_tensor_stencils_match(ten):
    K = 3**ten.dim
    for lv in range(1, ten.L + 1):
        n = ten.n(lv)
        out = ten.torch.empty(K * n, dtype=ten.torch.float64, device="cuda")
        ten.H.get_stencils(lv, out)
        st = ten.host(out).reshape(K, n).T
        dof = ten.grid.dof_mask(lv)
        # entries towards unknowns only: an entry towards a Dirichlet vertex keeps the
        # rediscretised value (it multiplies u = 0), and the two sides rediscretise coarse
        # levels differently (per-axis means in the oracle, the scalar mean on the GPU,
        # with the anisotropy in A_hat), so only the operator over the unknowns is the same
        nbr = ten.grid.tables(lv)["nbr"]
        has = (nbr >= 0) & dof[np.maximum(nbr, 0)]
        ref = ten.O.ops[lv].st
        scale = np.abs(ref).max(axis=1, keepdims=True)
        err = (np.abs(st - ref) * has)[dof] / np.maximum(scale[dof], 1e-300)
        assert err.max() < TOL * galerkin_amplification(ten.O, ten.tree, ten.L, ten.dim), (lv, err.max())


def test_tensor_finest_sweeps_and_residual_match(ten):
    L = ten.L
    rng = np.random.default_rng(3)
    u = np.where(ten.grid.dof_mask(L), rng.standard_normal(ten.n(L)), 0.0)
    for nu in (1, 2):
        ud = ten.dev(u)
        ten.H.smooth(L, ud, ten.b_dev, nu)
        assert rel_inf(ten.host(ud), ten.O.smooth(L, u, ten.b, nu)) < TOL
    r = ten.torch.zeros(ten.n(L), dtype=ten.torch.float64, device="cuda")
    n2 = ten.H.residual(L, ten.dev(u), ten.b_dev, r, want_norm=True)
    ref = ten.O.residual(L, u, ten.b)
    assert rel_inf(ten.host(r), ref) < TOL
    assert abs(n2 - float(ref @ ref)) <= 1e-12 * float(ref @ ref)


def test_tensor_vcycle_and_solve_match(ten):
    L = ten.L
    amp = galerkin_amplification(ten.O, ten.tree, L, ten.dim)
    rng = np.random.default_rng(5)
    u = np.where(ten.grid.dof_mask(L), rng.standard_normal(ten.n(L)), 0.0)
    ud = ten.dev(u)
    ten.H.vcycle(ud, ten.b_dev)
    parity_check(f"tensor vcycle {ten.dim}d-l{L}", rel_inf(ten.host(ud), ten.O.vcycle(u, ten.b)), amp, "cycle")
    ud = ten.torch.zeros(ten.n(L), dtype=ten.torch.float64, device="cuda")
    res = ten.H.solve(ud, ten.b_dev, rel_tol=1e-10, max_cycles=500)
    ref, hist = ten.O.solve(ten.b, 1e-10, 500)
    assert res["cycles"] == len(hist) - 1
    parity_check(f"tensor solve {ten.dim}d-l{L}", rel_inf(ten.host(ud), ref), amp, "solve")


@pytest.mark.parametrize("dim,L,om", CASES)
def test_tensor_mixed_solve_reaches_fp64_solution(dim, L, om):
    t = Tensor(dim, L, precision="mixed_bf16", omega=om)
    u = t.torch.zeros(t.n(L), dtype=t.torch.float64, device="cuda")
    res = t.H.solve(u, t.b_dev, rel_tol=1e-10, max_cycles=3000)
    assert res["rel_residual"] <= 1e-10
    ug = t.host(u)
    assert np.linalg.norm(t.O.residual(L, ug, t.b)) <= 1.0001e-10 * np.linalg.norm(t.b)
    assert rel_inf(ug, t.O.direct(t.b)) <= 1e-8


def test_isotropic_tensor_equals_scalar_setup():
    # eps_i = eps for every axis gives the scalar operator (the anisotropy vanishes)
    mg = lib()
    import torch

    dim, L = 2, 4
    e = syn.lognormal_grf_eps(L, dim, sigma=1.0, seed=7)
    grid = mg.Grid(dim, L)
    cat = grid.cells_to_concat({L: e})
    Ht = mg.Hierarchy(grid, tensor_coefficients=1)
    Ht.setup_tensor(torch.from_numpy(np.concatenate([cat, cat])).cuda())
    Hs = mg.Hierarchy(grid)
    Hs.setup(torch.from_numpy(cat).cuda())
    n = grid.info(L).n_slots
    a = torch.empty(9 * n, dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    Ht.get_stencils(L, a)
    Hs.get_stencils(L, b)
    assert torch.allclose(a, b, rtol=0, atol=1e-15)
    with pytest.raises(mg.MgError):
        mg.Hierarchy(grid, tensor_coefficients=1, coarse="redisc")
    with pytest.raises(mg.MgError):
        Hs.setup_tensor(torch.zeros(2 * grid.n_slots_total(), dtype=torch.float64, device="cuda"))
