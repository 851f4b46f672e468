"""Pins of the oracle's block Jacobi smoother (Sect. 4.2): the iota set by brute force,
Gauss-Seidel's energy decrease, the exact patch solve it tends to (a library solve),
and the paper's statement that block smoothing speeds up convergence."""
import numpy as np
import pytest

from oracle import multigrid
from oracle import spacetree as stt
import synthetic as syn


def hierarchy(dim, L, eps, **kw):
    tree = stt.Spacetree(dim, L)
    return tree, multigrid.Hierarchy(tree, {L: eps}, **kw)


@pytest.mark.parametrize("dim,L", [(2, 2), (2, 3), (3, 2)])
def test_iota_set_brute_force(dim, L):
    tree, H = hierarchy(dim, L, syn.constant_eps(L, dim), smoother="block")
    got = H.iota_vertices(L)
    n = 3 ** L
    want = set()
    for pos in np.ndindex(*(n,) * dim):
        if all(0 < p < n and p % 3 != 0 for p in pos):  # interior, inside a coarse cell
            want.add(int(tree.levels[L].pos2slot[pos]))
    assert set(got.tolist()) == want
    assert len(got) == (2 ** dim) * (3 ** (L - 1)) ** dim  # 2^d per level-(L-1) cell
    # within a patch: lexicographic, x fastest
    c = tree.levels[L].coords[got]
    patch = c // 3
    for i in range(0, len(got), 2 ** dim):
        assert np.all(patch[i:i + 2 ** dim] == patch[i])
        loc = c[i:i + 2 ** dim] - 3 * patch[i]
        rank = [sum(int(x[a] - 1) << a for a in range(dim)) for x in loc]
        assert rank == list(range(2 ** dim))


def energy(A, e):
    return float(e @ (A @ e))


@pytest.mark.parametrize("dim,L", [(2, 3), (3, 2)])
def test_steps_decrease_the_energy_error(dim, L):
    # Gauss-Seidel minimises the energy along each coordinate, and damped Jacobi with
    # omega = 0.6 is a contraction in the energy norm for these stencils: a block step
    # never raises ||u - u*||_A (a sign or index error in the update would)
    eps = syn.checkerboard_eps(L, dim, seed=3, tiles=3, values=(1.0, 0.01))
    tree, H = hierarchy(dim, L, eps, smoother="block")
    o = H.ops[L]
    rng = np.random.default_rng(5)
    b = np.where(o.dof, rng.uniform(-1, 1, o.dof.size), 0.0)
    ustar = H.direct(b)
    u = np.where(o.dof, rng.uniform(-1, 1, o.dof.size), 0.0)
    E0 = energy(o.A, u - ustar)
    H.omega = 0.0  # the Gauss-Seidel part alone
    u1 = H.block_smooth(L, u, b, 1)
    E1 = energy(o.A, u1 - ustar)
    assert E1 < E0
    H.omega = 0.6
    u2 = H.block_smooth(L, u, b, 1)
    assert energy(o.A, u2 - ustar) <= E1 * (1 + 1e-12)  # the Jacobi part on c, gamma DoFs
    assert energy(o.A, H.block_smooth(L, u, b, 3) - ustar) < energy(o.A, u2 - ustar)


def test_many_sweeps_reach_the_exact_patch_solve():
    # with the c and gamma values held, repeated Gauss-Seidel sweeps over a patch's iota
    # vertices converge to the solution of the patch's own 2^d x 2^d system
    dim, L = 2, 3
    eps = syn.lognormal_grf_eps(L, dim, sigma=1.0, seed=7)
    tree, H = hierarchy(dim, L, eps, smoother="block", gs_sweeps=200)
    H.omega = 0.0
    o = H.ops[L]
    rng = np.random.default_rng(2)
    b = np.where(o.dof, rng.uniform(-1, 1, o.dof.size), 0.0)
    u = np.where(o.dof, rng.uniform(-1, 1, o.dof.size), 0.0)
    got = H.block_smooth(L, u, b, 1)
    order = H.iota_vertices(L)
    A = o.A.tocsr()
    for p in range(0, len(order), 4):
        I = order[p:p + 4]
        rest = np.setdiff1d(np.arange(u.size), I)
        rhs = b[I] - A[I][:, rest] @ u[rest]
        exact = np.linalg.solve(A[I][:, I].toarray(), rhs)
        assert np.allclose(got[I], exact, rtol=1e-12, atol=1e-13)
    others = np.setdiff1d(np.arange(u.size), order)
    assert np.array_equal(got[others], u[others])


@pytest.mark.parametrize("eps_kind", ["checker", "grf"])
def test_block_smoothing_speeds_up_convergence(eps_kind):
    # Sect. 7 reports block smoothing up to halving the cycle count: fewer V(2,2) cycles
    dim, L = 2, 4
    eps = (syn.checkerboard_eps(L, dim, seed=0) if eps_kind == "checker"
           else syn.lognormal_grf_eps(L, dim, sigma=2.0, seed=1000))
    tree = stt.Spacetree(dim, L)
    b = tree.vertices_to_slots(L, syn.uniform_load(L, dim, 1))
    counts = {}
    for sm in ("jacobi", "block"):
        H = multigrid.Hierarchy(tree, {L: eps}, smoother=sm)
        _, hist = H.solve(b, rel_tol=1e-10, max_cycles=400)
        assert hist[-1] <= 1e-10 * hist[0]
        counts[sm] = len(hist) - 1
    assert counts["block"] < 0.8 * counts["jacobi"]
