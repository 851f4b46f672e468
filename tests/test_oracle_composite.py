"""Pins of the oracle's adaptive composite system and its FAS cycle (Sect. 3)."""
import numpy as np
import pytest

from oracle import composite, multigrid
from oracle import spacetree as stt
import synthetic as syn


def _tree(dim, L):
    T = L - 1
    c = (0.5, 0.5, 0.5)[:dim]
    return stt.Spacetree(dim, L, {T: syn.sphere_shell_mask(T, dim, radius=0.3, centre=c)}), T, c


@pytest.mark.parametrize("dim,L", [(2, 3), (2, 4), (3, 3)])
def test_composite_operator_is_exact_on_linear_functions(dim, L):
    # eps = 1: every FEM stencil annihilates linear functions and the hanging rule
    # (d-linear interpolation) and the injection rule reproduce them, so the
    # composite operator must vanish on a linear function at rows away from the boundary
    tree, T, _ = _tree(dim, L)
    C = composite.Composite(tree, {L: syn.constant_eps(L, dim), T: syn.constant_eps(T, dim)})
    M, i5, i4 = C.matrix()
    a = np.arange(1, dim + 1) * 0.37 + 0.1
    x = np.concatenate([(tree.levels[L].coords[i5] * tree.levels[L].h) @ a,
                        (tree.levels[T].coords[i4] * tree.levels[T].h) @ a])
    y = M @ x
    c5, c4 = tree.levels[L].coords[i5], tree.levels[T].coords[i4]
    in5 = np.all((c5 >= 4) & (c5 <= 3**L - 5), axis=1)
    in4 = np.all((c4 >= 2) & (c4 <= 3**T - 3), axis=1)
    assert in5.sum() > 10 and in4.sum() > 0
    assert np.abs(y[: len(i5)][in5]).max() < 1e-13
    assert np.abs(y[len(i5):][in4]).max() < 1e-13
    # and constants at every interior row
    assert np.abs((M @ np.ones(M.shape[0]))[: len(i5)][in5]).max() < 1e-13


@pytest.mark.parametrize("dim,L", [(2, 4), (3, 3)])
def test_fas_cycle_converges_to_the_composite_solution(dim, L):
    tree, T, c = _tree(dim, L)
    C = composite.Composite(tree, {L: syn.sphere_eps(L, dim, centre=c), T: syn.sphere_eps(T, dim, centre=c)})
    b5 = tree.vertices_to_slots(L, syn.uniform_load(L, dim, 2))
    b4 = np.where(C.unref4, tree.vertices_to_slots(T, syn.uniform_load(T, dim, 3)), 0.0)
    u5, u4, hist = C.solve(b5, b4, 1e-12, 400)
    assert hist[-1] <= 1e-12 * hist[0]
    d5, d4 = C.direct(b5, b4)
    scale = max(np.abs(d5).max(), np.abs(d4).max())
    assert np.abs(u5 - d5).max() <= 1e-9 * scale and np.abs(u4 - d4).max() <= 1e-9 * scale


def test_fully_refined_composite_is_the_uniform_system():
    dim, L = 2, 3
    tree = stt.Spacetree(dim, L, {L - 1: np.ones((9, 9), bool)})
    eps = syn.checkerboard_eps(L, dim, seed=0, tiles=3, values=(1.0, 0.1))
    C = composite.Composite(tree, {L: eps})
    assert C.unref4.sum() == 0
    M, i5, _ = C.matrix()
    U = multigrid.Hierarchy(stt.Spacetree(dim, L), {L: eps})
    A = U.ops[L].A[i5][:, i5]
    assert abs(M - A).max() < 1e-15


def test_composite_sin_solution_is_consistent():
    # for the smooth `sin` problem the error of a shell-refined composite grid is set
    # by its coarse part: it stays at the O(h_T^2) level of the uniform coarse grid
    # (a wrong hanging or injection rule would leave an O(h) interface error)
    dim, L = 2, 4
    tree, T, _ = _tree(dim, L)
    C = composite.Composite(tree, {L: syn.constant_eps(L, dim), T: syn.constant_eps(T, dim)})
    b5 = tree.vertices_to_slots(L, syn.sin_load(L, dim))
    b4 = np.where(C.unref4, tree.vertices_to_slots(T, syn.sin_load(T, dim)), 0.0)
    u5, u4 = C.direct(b5, b4)
    e5 = np.abs(u5 - tree.vertices_to_slots(L, syn.sin_solution(L, dim)))[C.dof5].max()
    U = multigrid.Hierarchy(stt.Spacetree(dim, T), {T: syn.constant_eps(T, dim)}, transfer="dlinear",
                            coarse="redisc")
    bT = stt.Spacetree(dim, T).vertices_to_slots(T, syn.sin_load(T, dim))
    eT = np.abs(U.direct(bT) - stt.Spacetree(dim, T).vertices_to_slots(T, syn.sin_solution(T, dim))).max()
    e4 = np.abs(u4 - tree.vertices_to_slots(T, syn.sin_solution(T, dim)))[C.unref4].max()
    assert e5 < 1.5 * eT and e4 < 1.5 * eT
