"""Pins of the oracle's additive multigrid (Alg. 2): the exact solution is a fixed point
of a traversal (Galerkin operators make the surplus restriction the coarse residual),
the first traversal from rest is one damped Jacobi sweep, and traversals converge to the
sparse direct solution, geometric and Galerkin / BoxMG."""
import numpy as np
import pytest

from oracle import multigrid
from oracle import spacetree as stt
import synthetic as syn


def state(H, uL):
    u = {lv: np.zeros(H.ops[lv].dof.size) for lv in range(H.coarsest, H.L + 1)}
    u[H.L] = uL.copy()
    d = {lv: np.zeros_like(u[lv]) for lv in u}
    return u, d


@pytest.mark.parametrize("dim,L,eps", [(2, 4, "checker"), (2, 3, "grf"), (3, 3, "grf")])
def test_exact_solution_is_a_fixed_point(dim, L, eps):
    e = (syn.checkerboard_eps(L, dim, seed=0) if eps == "checker"
         else syn.lognormal_grf_eps(L, dim, sigma=2.0, seed=4))
    tree = stt.Spacetree(dim, L)
    H = multigrid.Hierarchy(tree, {L: e})
    b = tree.vertices_to_slots(L, syn.uniform_load(L, dim, 1))
    ustar = H.direct(b)
    u, d = state(H, ustar)
    for lv in range(L, H.coarsest, -1):  # coarse iterates = injections of the solution
        u[lv - 1] = H.inject(lv, u[lv])
    H.additive_traversal(u, d, b)
    scale = np.abs(ustar).max()
    assert np.abs(u[L] - ustar).max() <= 1e-11 * scale
    for lv in d:
        assert np.abs(d[lv]).max() <= 1e-11 * scale


def test_first_traversal_from_rest_is_a_jacobi_sweep():
    dim, L = 2, 4
    tree = stt.Spacetree(dim, L)
    H = multigrid.Hierarchy(tree, {L: syn.checkerboard_eps(L, dim, seed=2)})
    b = tree.vertices_to_slots(L, syn.uniform_load(L, dim, 3))
    rng = np.random.default_rng(1)
    u0 = np.where(H.ops[L].dof, rng.uniform(-1, 1, b.size), 0.0)
    u, d = state(H, u0)
    H.additive_traversal(u, d, b)
    assert np.allclose(u[L], H.smooth(L, u0, b, 1), rtol=0, atol=1e-14)


@pytest.mark.parametrize("case", ["sin-geometric", "checker-galerkin"])
def test_traversals_converge_to_the_direct_solution(case):
    dim, L = 2, 4
    tree = stt.Spacetree(dim, L)
    if case == "sin-geometric":
        H = multigrid.Hierarchy(tree, {L: syn.constant_eps(L, dim)}, transfer="dlinear", coarse="redisc",
                                omega=0.8)
        b = tree.vertices_to_slots(L, syn.sin_load(L, dim))
    else:
        H = multigrid.Hierarchy(tree, {L: syn.checkerboard_eps(L, dim, seed=0)}, omega=0.8)
        b = tree.vertices_to_slots(L, syn.uniform_load(L, dim, 1))
    u, hist = H.additive_solve(b, rel_tol=1e-10, max_cycles=1000)
    assert hist[-1] <= 1e-10 * hist[0]
    ref = H.direct(b)
    assert np.abs(u - ref).max() <= 1e-8 * np.abs(ref).max()
    # additive multigrid contracts slower than the multiplicative V-cycle, but at a rate
    # well below one (a pure Jacobi iteration would need thousands of sweeps here)
    _, vhist = H.solve(b, rel_tol=1e-10, max_cycles=1000)
    assert len(vhist) < len(hist) < 400


# --------------------------------------------------------------------------- BPX (Alg. 3)
@pytest.mark.parametrize("dim,L", [(2, 4), (3, 3)])
def test_bpx_fixed_point_for_any_coarse_state(dim, L):
    # with Galerkin operators R A (u - P u_c) + A_c u_c = R A u for any coarse iterate, so
    # the exact solution is a fixed point whatever the coarse levels hold
    tree = stt.Spacetree(dim, L)
    H = multigrid.Hierarchy(tree, {L: syn.lognormal_grf_eps(L, dim, sigma=1.5, seed=9)})
    b = tree.vertices_to_slots(L, syn.uniform_load(L, dim, 2))
    ustar = H.direct(b)
    rng = np.random.default_rng(4)
    u, d = state(H, ustar)
    for lv in range(H.coarsest, L):
        u[lv] = np.where(H.ops[lv].dof, rng.uniform(-1, 1, u[lv].size), 0.0)
    i = {lv: np.zeros_like(u[lv]) for lv in u}
    H.bpx_traversal(u, d, i, b)
    assert np.abs(u[L] - ustar).max() <= 1e-11 * np.abs(ustar).max()


def test_bpx_first_traversal_skips_c_points():
    dim, L = 2, 4
    tree = stt.Spacetree(dim, L)
    H = multigrid.Hierarchy(tree, {L: syn.checkerboard_eps(L, dim, seed=2)})
    b = tree.vertices_to_slots(L, syn.uniform_load(L, dim, 3))
    rng = np.random.default_rng(1)
    u0 = np.where(H.ops[L].dof, rng.uniform(-1, 1, b.size), 0.0)
    u, d = state(H, u0)
    i = {lv: np.zeros_like(u[lv]) for lv in u}
    H.bpx_traversal(u, d, i, b)
    cp = H.c_points(L)
    jac = H.smooth(L, u0, b, 1)
    assert np.array_equal(u[L][cp], u0[cp])
    assert np.allclose(u[L][~cp], jac[~cp], rtol=0, atol=1e-14)
    # the skipped updates reach the coarser level by injection
    assert np.allclose(i[L - 1], H.inject(L, jac - u0), rtol=0, atol=1e-14)


@pytest.mark.parametrize("case", ["sin-geometric", "checker-galerkin"])
def test_bpx_converges_to_the_direct_solution(case):
    dim, L = 2, 4
    tree = stt.Spacetree(dim, L)
    if case == "sin-geometric":
        H = multigrid.Hierarchy(tree, {L: syn.constant_eps(L, dim)}, transfer="dlinear", coarse="redisc",
                                omega=0.8)
        b = tree.vertices_to_slots(L, syn.sin_load(L, dim))
    else:
        H = multigrid.Hierarchy(tree, {L: syn.checkerboard_eps(L, dim, seed=0)}, omega=0.8)
        b = tree.vertices_to_slots(L, syn.uniform_load(L, dim, 1))
    u, hist = H.bpx_solve(b, rel_tol=1e-10, max_cycles=1000)
    assert hist[-1] <= 1e-10 * hist[0]
    ref = H.direct(b)
    assert np.abs(u - ref).max() <= 1e-8 * np.abs(ref).max()
