"""Pins of the oracle's diagonal-tensor coefficients (eq. (1) with eps = diag(eps_i); the
paper's `checkerboard` benchmark): directional element matrices in closed form, the
assembled anisotropic stencil, the isotropic special case, and a converging solve."""
import itertools

import numpy as np
import pytest

from oracle import fem, multigrid
from oracle import spacetree as stt
import synthetic as syn


@pytest.mark.parametrize("dim", [2, 3])
def test_directional_element_matrices_closed_form(dim):
    # int d_i phi_a d_i phi_b over a cube of side h = h^(d-2) * (+1 if a_i == b_i else -1)
    # * prod_{j != i} m(a_j, b_j), with the 1D mass entries m = 1/3 (same) or 1/6
    h = 0.37
    Ks = fem.directional_element_matrices(dim, h)
    cs = list(itertools.product(range(2), repeat=dim))
    cs = [c[::-1] for c in cs]  # corners lexicographic with x fastest
    for i in range(dim):
        for a, ca in enumerate(cs):
            for b, cb in enumerate(cs):
                v = (1.0 if ca[i] == cb[i] else -1.0) * h ** (dim - 2)
                for j in range(dim):
                    if j != i:
                        v *= 1.0 / 3.0 if ca[j] == cb[j] else 1.0 / 6.0
                assert Ks[i][a, b] == pytest.approx(v, rel=1e-13, abs=1e-15)
    assert np.allclose(sum(Ks), fem.element_matrix(dim, h), rtol=0, atol=1e-15)


def test_assembled_anisotropic_stencil_2d():
    # constant (eps_x, eps_y): centre 4/3 (ex + ey), east / west -2/3 ex + 1/3 ey,
    # north / south 1/3 ex - 2/3 ey, corners -(ex + ey) / 6 (row sum zero)
    L, ex, ey = 2, 1.0, 0.1
    tree = stt.Spacetree(2, L)
    e = np.empty((3**L, 3**L, 2))
    e[..., 0], e[..., 1] = ex, ey
    H = multigrid.Hierarchy(tree, {L: e}, transfer="dlinear", coarse="redisc")
    st = H.ops[L].st_redisc
    v = tree.levels[L].slot_of(np.array([4, 4]))
    want = [-(ex + ey) / 6, ex / 3 - 2 * ey / 3, -(ex + ey) / 6,
            -2 * ex / 3 + ey / 3, 4 * (ex + ey) / 3, -2 * ex / 3 + ey / 3,
            -(ex + ey) / 6, ex / 3 - 2 * ey / 3, -(ex + ey) / 6]
    assert np.allclose(st[v], want, rtol=0, atol=1e-14)
    assert abs(st[v].sum()) < 1e-14


@pytest.mark.parametrize("dim,L", [(2, 3), (3, 2)])
def test_isotropic_tensor_equals_scalar(dim, L):
    tree = stt.Spacetree(dim, L)
    e = syn.lognormal_grf_eps(L, dim, sigma=1.0, seed=3)
    et = np.repeat(e[..., None], dim, axis=-1)
    A = multigrid.Hierarchy(tree, {L: e})
    B = multigrid.Hierarchy(tree, {L: et})
    for lv in range(1, L + 1):
        assert abs(A.ops[lv].A - B.ops[lv].A).max() <= 1e-13 * abs(A.ops[lv].A).max()
        assert np.allclose(A.ops[lv].st, B.ops[lv].st, rtol=0, atol=1e-13)


@pytest.mark.parametrize("dim,L,omega", [(2, 4, 0.6), (3, 3, 0.5)])
def test_checkerboard_benchmark_solves(dim, L, omega):
    # in 3D the anisotropic trilinear elements give positive face-neighbour entries and
    # lambda_max(D^-1 A) = 3.66 on level 3, so damped Jacobi needs omega < 2 / 3.66
    tree = stt.Spacetree(dim, L)
    e = syn.axis_checkerboard_eps(L, dim)
    assert e.shape == (3**L,) * dim + (dim,)
    H = multigrid.Hierarchy(tree, {L: e}, omega=omega)
    b = tree.vertices_to_slots(L, syn.unit_load(L, dim))
    u, hist = H.solve(b, rel_tol=1e-9, max_cycles=400)
    assert hist[-1] <= 1e-9 * hist[0]
    ref = H.direct(b)
    assert np.abs(u - ref).max() <= 1e-7 * np.abs(ref).max()
    # the coarse rediscretisation coefficient stays the per-axis mean of the children
    ce = fem.coarse_eps(tree, {L: e})
    assert np.allclose(ce[L - 1], e.reshape([3**(L - 1), 3] * dim + [dim]).mean(axis=tuple(range(1, 2 * dim, 2))))
