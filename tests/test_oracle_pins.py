"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test ties an oracle function to something other than itself: values the
paper prints (golden fixtures under tests/golden/), closed forms, invariants,
special cases reducing to textbook results, or brute force on tiny inputs.
"""
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import boxmg, codec, fem, galerkin, multigrid
from oracle import spacetree as stt
import synthetic as syn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- A1 tables
@pytest.mark.parametrize("dim,level", [(2, 1), (2, 2), (2, 3), (3, 1), (3, 2)])
def test_peano_curve_is_face_continuous(dim, level):
    cells = stt.peano_cells(level, dim)
    assert len(cells) == 3 ** (dim * level)
    assert len(set(cells)) == len(cells)
    a = np.array(cells)
    step = np.abs(np.diff(a, axis=0))
    # consecutive cells share a (d-1)-face: exactly one coordinate differs, by one
    assert np.all(step.sum(axis=1) == 1)


def test_peano_level1_serpentine():
    # Peano's map on a 3x3 grid: axis 0 major, axis 1 reversed on odd columns
    expect = [(0, 0), (0, 1), (0, 2), (1, 2), (1, 1), (1, 0), (2, 0), (2, 1), (2, 2)]
    assert stt.peano_cells(1, 2) == expect


@pytest.mark.parametrize("dim,level", [(2, 2), (2, 4), (3, 2), (3, 3)])
def test_uniform_tables_brute_force(dim, level):
    tree = stt.Spacetree(dim, level)
    for lv_i in range(level + 1):
        lv = tree.levels[lv_i]
        n = 3**lv_i
        c = lv.coords[lv.valid]
        # every position of [0, n)^d appears exactly once
        assert len(c) == n**dim
        assert len({tuple(x) for x in c}) == n**dim
        # flags: boundary iff a zero coordinate; DoFs = (n-1)^d interior vertices
        bnd = np.any(c == 0, axis=1)
        assert np.array_equal((lv.vflags[lv.valid] & stt.BOUNDARY) != 0, bnd)
        assert lv.dof.sum() == (n - 1) ** dim
        # refined vertices: interior and all adjacent cells refined (all, below max level)
        ref = (lv.vflags & stt.REFINED) != 0
        assert ref.sum() == (lv.dof.sum() if lv_i < level else 0)
        # neighbour symmetry
        offs = stt.offsets(dim)
        opp = {tuple(o): j for j, o in enumerate(offs)}
        for s in np.nonzero(lv.valid)[0][:: max(1, lv.n_slots // 200)]:
            for j, o in enumerate(offs):
                t = lv.nbr[s, j]
                inside = np.all((lv.coords[s] + o >= 0) & (lv.coords[s] + o < n))
                assert (t >= 0) == inside
                if t >= 0:
                    assert np.array_equal(lv.coords[t], lv.coords[s] + o)
                    assert lv.nbr[t, opp[tuple(-o)]] == s
        # Peano order of bricks: consecutive brick roots are face neighbours
        if lv.n_bricks > 1:
            st = np.abs(np.diff(lv.brick_roots, axis=0)).sum(axis=1)
            assert np.all(st == 1)


def test_adaptive_flags_brute_force():
    dim, L = 2, 3
    m1 = np.zeros((3, 3), bool)
    m1[1, 1] = m1[2, 1] = True
    m2 = np.zeros((9, 9), bool)
    m2[4, 4] = True
    tree = stt.Spacetree(dim, L, {1: m1, 2: m2})
    for lv_i in range(L + 1):
        lv = tree.levels[lv_i]
        cells = tree.cells[lv_i]
        refined = tree.refined[lv_i]
        n = 3**lv_i
        for s in np.nonzero(lv.valid)[0]:
            x = lv.coords[s]
            adj = [tuple(x - np.array(e)) for e in [(0, 0), (1, 0), (0, 1), (1, 1)]]
            adj = [a for a in adj if all(0 <= v < n for v in a)]
            na = sum(cells[a] for a in adj)
            nr = sum(refined[a] for a in adj)
            f = lv.vflags[s]
            assert bool(f & stt.EXISTS) == (na > 0)
            if na == 0:
                continue
            bnd = bool(np.any(x == 0))
            assert bool(f & stt.BOUNDARY) == bnd
            if not bnd:
                assert bool(f & stt.HANGING) == (na < 4)
                assert bool(f & stt.REFINED) == (na == 4 and nr == 4)
    # hanging weights: sum to one where every parent exists, d-linear interpolant
    idx, w = tree.hanging_map(3)
    lv = tree.levels[3]
    hang = np.nonzero(lv.vflags & stt.HANGING)[0]
    assert len(hang) > 0
    for s in hang:
        assert abs(w[s].sum() - 1.0) < 1e-15
        # the interpolant reproduces a linear function of position
        xc = tree.levels[2].coords
        val = sum(w[s, j] * (xc[idx[s, j]] @ [0.3, 0.7]) for j in range(4) if idx[s, j] >= 0)
        assert abs(val - (lv.coords[s] / 3.0) @ [0.3, 0.7]) < 1e-13


# --------------------------------------------------------------------------- A2 stencils
def test_element_matrix_closed_forms():
    K2 = fem.element_matrix(2, 0.37)
    ham = lambda a, b: bin(a ^ b).count("1")
    table2 = {0: 2 / 3, 1: -1 / 6, 2: -1 / 3}
    for a in range(4):
        for b in range(4):
            assert abs(K2[a, b] - table2[ham(a, b)]) < 1e-15
    h = 1 / 27
    K3 = fem.element_matrix(3, h)
    table3 = {0: 1 / 3, 1: 0.0, 2: -1 / 12, 3: -1 / 12}
    for a in range(8):
        for b in range(8):
            assert abs(K3[a, b] - h * table3[ham(a, b)]) < 1e-15 * h * 10


def test_assembled_stencil_constant_eps():
    for dim, L in [(2, 2), (3, 2)]:
        tree = stt.Spacetree(dim, L)
        A = fem.assemble(tree, L, syn.constant_eps(L, dim))
        st = fem.stencils(tree, L, A)
        lv = tree.levels[L]
        s = lv.slot_of([4] * dim)
        offs = stt.offsets(dim)
        h = lv.h
        for j, o in enumerate(offs):
            k = int(np.abs(o).sum())
            if dim == 2:
                expect = 8 / 3 if k == 0 else -1 / 3
            else:
                expect = h * {0: 8 / 3, 1: 0.0, 2: -1 / 6, 3: -1 / 12}[k]
            assert abs(st[s, j] - expect) < 1e-14


def test_full_operator_rows_sum_to_zero():
    rng = np.random.default_rng(5)
    for dim, L in [(2, 3), (3, 2)]:
        tree = stt.Spacetree(dim, L)
        eps = rng.uniform(0.1, 10, size=(3**L,) * dim)
        A = fem.assemble(tree, L, eps)
        lv = tree.levels[L]
        # vertices whose whole 3^d neighbourhood has slots (the upper boundary x = 3^l has none)
        interior = np.all((lv.coords > 0) & (lv.coords < lv.n - 1), axis=1) & lv.valid
        rs = np.asarray(A.sum(axis=1)).ravel()[interior]
        assert np.abs(rs).max() < 1e-13


def _frac(t):
    return float(Fraction(t))


def test_stencil_split_matches_paper():
    # for eps = 1 the cell-wise pieces of the FEM stencil are the paper's split
    tree = stt.Spacetree(2, 2)
    st = fem.stencils(tree, 2, fem.assemble(tree, 2, syn.constant_eps(2, 2)))
    lv = tree.levels[2]
    v = lv.slot_of([4, 4])
    K = fem.element_matrix(2, 1.0)
    cs = stt.corners(2)
    offs = stt.offsets(2)
    with open(os.path.join(GOLDEN, "stencil_split_2d.txt")) as f:
        lines = [ln for ln in f if ln.startswith("cell")]
    total = np.zeros(9)
    for ln in lines:
        head, facs = ln.split(":")
        cell = np.array([int(t) for t in head.split()[1:]])
        facs = np.array([_frac(t) for t in facs.split()])
        corner_v = -cell  # position of the vertex inside that cell
        piece = np.zeros(9)
        for j, o in enumerate(offs):
            corner_n = corner_v + o
            if np.all((corner_n >= 0) & (corner_n <= 1)):
                a = int(np.nonzero((cs == corner_v).all(axis=1))[0][0])
                b = int(np.nonzero((cs == corner_n).all(axis=1))[0][0])
                piece[j] = K[a, b]
        assert np.allclose(piece, facs * st[v], atol=1e-15)
        total += piece
    assert np.allclose(total, st[v], atol=1e-15)


# --------------------------------------------------------------------------- A8 BoxMG
def test_boxmg_1d_worked_example():
    with open(os.path.join(GOLDEN, "boxmg_1d_worked_example.txt")) as f:
        rows = [ln.split() for ln in f if not ln.startswith("#")]
    sten = np.array([float(t) for t in rows[0][1:]])
    p_expect = np.array([float(t) for t in rows[1][1:]])
    s = np.tile(sten, (4, 1))
    assert np.allclose(boxmg.solve_corner(s, [0], 1), p_expect, atol=1e-15)
    # the right coarse vertex, through mirroring, gets the mirrored values
    assert np.allclose(boxmg.solve_corner(s, [1], 1), p_expect, atol=1e-15)


def test_boxmg_2d_system_matrix_matches_appendix():
    rng = np.random.default_rng(0)
    s = rng.standard_normal((16, 9))
    C = boxmg.system_matrix(s, 2)
    with open(os.path.join(GOLDEN, "boxmg_2d_C_matrix.txt")) as f:
        rows = [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 9
    for ln in rows:
        head, body = ln.split(":", 1)
        v = int(head[2:])
        i = (v % 4) + 3 * (v // 4)  # oracle rows are lexicographic over reference positions
        cells = [c.strip() for c in body.split("|")]
        assert len(cells) == 9
        for j, c in enumerate(cells):
            if c == "0":
                val = 0.0
            elif c == "1":
                val = 1.0
            else:
                val = 0.0
                for term in c.split("+"):
                    vi, sj = term[1:].split(",")
                    val += s[int(vi), int(sj)]
            assert abs(C[i, j] - val) < 1e-14, (i, j)


def test_boxmg_constant_eps_gives_dlinear():
    with_expect = np.array([1, 2 / 3, 1 / 3, 2 / 3, 4 / 9, 2 / 9, 1 / 3, 2 / 9, 1 / 9])
    s = np.tile(np.array([-1, -1, -1, -1, 8, -1, -1, -1, -1]) / 3.0, (16, 1))
    for e in stt.corners(2):
        assert np.allclose(boxmg.solve_corner(s, e, 2), with_expect, atol=1e-15)
    for dim, L in [(2, 3), (3, 2)]:
        tree = stt.Spacetree(dim, L)
        st = fem.stencils(tree, L, fem.assemble(tree, L, syn.constant_eps(L, dim)))
        Pb = boxmg.prolongation(tree, L, st, "boxmg")
        Pd = boxmg.prolongation(tree, L, None, "dlinear")
        assert abs(Pb - Pd).max() < 1e-14


def test_boxmg_partition_of_unity_random_eps():
    rng = np.random.default_rng(3)
    for dim, L in [(2, 3), (3, 2)]:
        tree = stt.Spacetree(dim, L)
        eps = np.exp(rng.standard_normal((3**L,) * dim) * 2)
        st = fem.stencils(tree, L, fem.assemble(tree, L, eps))
        P = boxmg.prolongation(tree, L, st, "boxmg")
        fine = tree.levels[L]
        x = fine.coords
        # fine DoFs inside patches whose 2^d corners are all interior coarse vertices
        c = x // 3
        ok = fine.valid & np.all(c >= 1, axis=1) & np.all(c + 1 <= 3 ** (L - 1) - 1, axis=1)
        rs = np.asarray(P.sum(axis=1)).ravel()
        assert np.abs(rs[ok] - 1).max() < 1e-12
        # entries computed by several patches agree (mirroring consistency)
        r, cc, v = boxmg.prolongation(tree, L, st, "boxmg", return_raw=True)
        key = r * tree.levels[L - 1].n_slots + cc
        order = np.argsort(key, kind="stable")
        ks, vs = key[order], v[order]
        same = ks[1:] == ks[:-1]
        assert same.any()
        assert np.abs(vs[1:][same] - vs[:-1][same]).max() < 1e-13


# --------------------------------------------------------------------------- A9 / A10 Galerkin
@pytest.mark.parametrize("dim,L", [(2, 4), (3, 3)])
def test_galerkin_constant_eps_has_zero_deltas(dim, L):
    tree = stt.Spacetree(dim, L)
    H = multigrid.Hierarchy(tree, {L: syn.constant_eps(L, dim)})
    for lv in range(1, L):
        scale = np.abs(H.ops[lv].st).max()
        assert np.abs(H.ops[lv].a_hat).max() < 1e-14 * scale * 10
        assert np.abs(H.ops[lv + 1].p_hat).max() < 1e-14 * 10


def test_galerkin_dlinear_equals_coarse_fem_for_coarse_piecewise_eps():
    # eps constant on every coarse cell: the coarse FE space is nested in the fine one
    # and d-linear P is exact on it, so R A P equals the coarse FE matrix.
    rng = np.random.default_rng(11)
    for dim, L in [(2, 3), (3, 2)]:
        tree = stt.Spacetree(dim, L)
        ec = rng.uniform(0.5, 5.0, size=(3 ** (L - 1),) * dim)
        ef = ec
        for ax in range(dim):
            ef = np.repeat(ef, 3, axis=ax)
        Af = fem.restrict_to_dofs(fem.assemble(tree, L, ef), tree.levels[L].dof)
        P = boxmg.prolongation(tree, L, None, "dlinear")
        Ag = galerkin.galerkin(Af, P)
        Ac = fem.restrict_to_dofs(fem.assemble(tree, L - 1, ec), tree.levels[L - 1].dof)
        assert abs(Ag - Ac).max() < 1e-13 * abs(Ac).max()


def test_galerkin_is_symmetric_and_positive_diagonal():
    tree = stt.Spacetree(2, 4)
    H = multigrid.Hierarchy(tree, {4: syn.checkerboard_eps(4, 2, seed=0)})
    for lv in range(1, 4):
        A = H.ops[lv].A
        assert abs(A - A.T).max() < 1e-13 * abs(A).max()
        assert np.all(H.ops[lv].diag[H.ops[lv].dof] > 0)


# --------------------------------------------------------------------------- A3-A12 solver
def test_jacobi_sweep_closed_form():
    tree = stt.Spacetree(2, 2)
    H = multigrid.Hierarchy(tree, {2: syn.constant_eps(2, 2)}, transfer="dlinear", coarse="redisc",
                            omega=0.6)
    b = tree.vertices_to_slots(2, np.ones((10, 10)))
    u1 = H.smooth(2, np.zeros_like(b), b, 1)
    lv = tree.levels[2]
    assert np.allclose(u1[lv.dof], 0.6 * 1.0 / (8 / 3), atol=1e-15)
    # second sweep at a vertex two away from the boundary: neighbours all equal c
    c = 0.6 * 3 / 8
    u2 = H.smooth(2, u1, b, 1)
    s = lv.slot_of([4, 4])
    assert abs(u2[s] - (c + 0.6 * (1.0 - 0.0) / (8 / 3))) < 1e-15


def test_sin_discretisation_error_is_second_order():
    errs = []
    for L in (3, 4):
        tree = stt.Spacetree(2, L)
        H = multigrid.Hierarchy(tree, {L: syn.constant_eps(L, 2)}, transfer="dlinear", coarse="redisc")
        b = tree.vertices_to_slots(L, syn.sin_load(L, 2))
        u = H.direct(b)
        ue = tree.vertices_to_slots(L, syn.sin_solution(L, 2))
        errs.append(np.abs(u - ue).max())
    assert 7.0 < errs[0] / errs[1] < 11.0


@pytest.mark.parametrize("dim,L", [(2, 2), (2, 3), (3, 2)])
def test_vcycle_solve_matches_dense_solve(dim, L):
    tree = stt.Spacetree(dim, L)
    H = multigrid.Hierarchy(tree, {L: syn.checkerboard_eps(L, dim, seed=1, tiles=3, values=(1.0, 0.1))})
    b = tree.vertices_to_slots(L, syn.uniform_load(L, dim, 7))
    u, hist = H.solve(b, 1e-13, 300)
    o = H.ops[L]
    idx = np.nonzero(o.dof)[0]
    ud = np.zeros_like(b)
    ud[idx] = np.linalg.solve(o.A[idx][:, idx].toarray(), b[idx])
    assert np.linalg.norm(u - ud) <= 1e-10 * np.linalg.norm(ud)


def test_level_independent_contraction_and_cycle_count():
    rates, cycles = [], []
    for L in (3, 4, 5):
        tree = stt.Spacetree(2, L)
        H = multigrid.Hierarchy(tree, {L: syn.constant_eps(L, 2)}, transfer="dlinear", coarse="redisc",
                                omega=0.6)
        b = tree.vertices_to_slots(L, syn.sin_load(L, 2))
        _, h = H.solve(b, 1e-8, 60)
        rates.append(np.median(h[-4:] / h[-5:-1]))
        cycles.append(len(h) - 1)
    assert max(rates) < 0.4 and max(rates) - min(rates) < 0.08
    # the paper reports 10-15 multiplicative cycles with an exact coarse solve on `sin`
    assert all(10 <= c <= 20 for c in cycles)


# --------------------------------------------------------------------------- codec
def test_codec_rounding_bit_patterns():
    vals = np.array([1.0, 1 / 3, -0.1, 1 + 2**-8, 1 + 3 * 2**-8, 2.0**-130, 0.0])
    bf = codec.to_bits(codec.round_to_format(vals, "bf16"), "bf16")
    assert list(bf) == [0x3F80, 0x3EAB, 0xBDCD, 0x3F80, 0x3F82, 0x0008, 0x0000]
    hf = codec.to_bits(codec.round_to_format(np.array([1.0, 1 / 3, -0.1, 2.0**-24, 1 + 2**-11]), "fp16"), "fp16")
    assert list(hf) == [0x3C00, 0x3555, 0xAE66, 0x0001, 0x3C00]


def test_codec_against_library_conversions():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    x = rng.standard_normal(20000) * np.exp(rng.uniform(-30, 0, 20000))
    # numpy's float64 -> float16 conversion rounds once to nearest even
    assert np.array_equal(codec.to_bits(codec.round_to_format(x, "fp16"), "fp16"),
                          x.astype(np.float16).view(np.uint16))
    # for FP32-representable inputs one rounding to bf16 is torch's float32 -> bfloat16
    x32 = x.astype(np.float32).astype(np.float64)
    tb = torch.from_numpy(x32.astype(np.float32)).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(codec.to_bits(codec.round_to_format(x32, "bf16"), "bf16"), tb)


def test_codec_roundtrip_error_bound():
    rng = np.random.default_rng(4)
    d = rng.standard_normal((500, 9)) * np.exp(rng.uniform(-5, 5, (500, 1)))
    d[3] = 0.0
    for fmt, u in (("bf16", 2.0**-8), ("fp16", 2.0**-11)):
        q, s = codec.encode(d, fmt)
        back = codec.decode(q, s, fmt).astype(np.float64)
        m = np.abs(d).max(axis=1, keepdims=True)
        assert np.all(np.abs(back - d) <= (u + 2.0**-23) * 1.01 * m + 1e-300)
        assert np.all(back[3] == 0) and s[3] == 0


def test_jump_coefficient_recipe():
    # eps by cell centre: 1 for x_1 < 0.5, 0.1 beyond; on 3^L cells the jump falls inside
    # the middle column, which takes the value of its centre (x_1 = 0.5 exactly: 0.1)
    import synthetic as syn

    e = syn.jump_eps(2, 2)
    assert e.shape == (9, 9)
    assert np.all(e[:4] == 1.0) and np.all(e[4:] == 0.1)
    assert np.all(syn.unit_load(2, 2) == 1.0 / 81)
