"""Host-side parity of the C-ABI library with the oracle (no GPU needed).

The grid builder (mg_create_grid / mg_grid_tables) is plain host C++; its level
tables must equal the oracle's independently computed ones bit for bit.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import spacetree as stt
import synthetic as syn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def mg():
    import paper_1607_00648_gb300 as mgpkg
    from paper_1607_00648_gb300 import build

    if not os.path.exists(mgpkg._lib.LIB_PATH):
        build.build()
    mgpkg.load()
    return mgpkg


def test_library_exports_every_declared_symbol(mg):
    header = open(os.path.join(ROOT, "include", "mg.h")).read()
    declared = set(re.findall(r"^\s*(?:mg_status|void|const char\*)\s+(mg_\w+)\s*\(", header, re.M))
    assert len(declared) >= 20
    lib = ctypes.CDLL(mg._lib.LIB_PATH)
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert declared <= set(mg._lib.symbols())


def _compare_level(g, tree, level):
    t = g.tables(level)
    lv = tree.levels[level]
    inf = g.info(level)
    assert inf.n_slots == lv.n_slots and inf.n_bricks == lv.n_bricks
    assert inf.brick_edge == lv.B and inf.slots_per_brick == lv.S
    assert inf.n_dofs == int(lv.dof.sum())
    assert np.array_equal(t["coords"], lv.coords)
    assert np.array_equal(t["vflags"], lv.vflags)
    assert np.array_equal(t["cflags"], lv.cflags)
    assert np.array_equal(t["nbr"], lv.nbr)
    assert np.array_equal(t["cell_vertices"], lv.cell_vertices)
    assert np.array_equal(t["brick_roots"], lv.brick_roots)
    assert np.array_equal(t["brick_nbr"], lv.brick_nbr)
    assert np.array_equal(t["parent"], tree.parent_map(level))
    assert np.array_equal(t["child"], tree.child_map(level))
    hi, hw = tree.hanging_map(level)
    assert np.array_equal(t["hang_idx"], hi)
    assert np.array_equal(t["hang_w"].view(np.uint64), hw.view(np.uint64))


@pytest.mark.parametrize("dim,L", [(2, 3), (2, 4), (3, 2), (3, 3)])
def test_uniform_tables_bit_exact(mg, dim, L):
    g = mg.Grid(dim, L)
    tree = stt.Spacetree(dim, L)
    for level in range(L + 1):
        _compare_level(g, tree, level)


def test_adaptive_tables_bit_exact_2d(mg):
    m1 = np.zeros((3, 3), bool)
    m1[1, 1] = m1[2, 1] = m1[0, 0] = True
    m2 = np.zeros((9, 9), bool)
    m2[4, 4] = m2[3, 4] = m2[0, 1] = True
    masks = {1: m1, 2: m2}
    g = mg.Grid(2, 3, masks)
    tree = stt.Spacetree(2, 3, masks)
    for level in range(4):
        _compare_level(g, tree, level)


def test_adaptive_tables_bit_exact_3d_shell(mg):
    # the sphere-shell refinement of the adaptive 3D workload, one level lower
    masks = {2: syn.sphere_shell_mask(2, 3)}
    g = mg.Grid(3, 3, masks)
    tree = stt.Spacetree(3, 3, masks)
    assert tree.levels[3].vflags.astype(bool).any()
    for level in range(4):
        _compare_level(g, tree, level)


def test_invalid_arguments_are_rejected(mg):
    with pytest.raises(mg.MgError):
        mg.Grid(4, 2)
    with pytest.raises(mg.MgError):
        mg.Grid(2, 0)
    g = mg.Grid(2, 2)
    with pytest.raises(mg.MgError):
        g.info(5)


def test_adaptive_hierarchy_shape_is_checked_before_any_device_work(mg):
    # the composite hierarchy needs levels 0 .. L-2 refined everywhere; both checks
    # come before any allocation, so they run without a GPU
    m1 = np.zeros((3, 3), bool)
    m1[1, 1] = True
    g = mg.Grid(2, 3, {1: m1})  # level 1 refined in part
    with pytest.raises(mg.MgError) as e:
        mg.Hierarchy(g)
    assert e.value.status == 10  # MG_ERR_UNSUPPORTED
    g2 = mg.Grid(2, 3, {2: syn.sphere_shell_mask(2, 2)})
    with pytest.raises(mg.MgError) as e:
        mg.Hierarchy(g2, coarsest_level=2)  # the coarsest level must lie below level L-1
    assert e.value.status == 1  # MG_ERR_INVALID_ARG


def test_option_validation_needs_no_gpu(mg):
    # mg_hier_create checks its options before touching the device
    g = mg.Grid(2, 3)
    bad = [dict(smoother="block", gs_sweeps=0), dict(smoother="block", gs_sweeps=65), dict(smoother=2),
           dict(cycle="additive", precision="mixed_bf16"), dict(cycle="additive", smoother="block"),
           dict(cycle=2), dict(precision=4), dict(precision="mixed_bpa", eps_mf=-1.0),
           dict(precision="mixed_bpa", eps_mf=float("nan")), dict(coarsest_level=3), dict(omega=0.0)]
    for kw in bad:
        with pytest.raises(mg.MgError):
            mg.Hierarchy(g, **kw)
    ga = mg.Grid(2, 4, {3: syn.sphere_shell_mask(3, 2, radius=0.3, centre=(0.5, 0.5))})
    with pytest.raises(mg.MgError):
        mg.Hierarchy(ga, cycle="additive")


def test_footprints_of_the_storage_modes(mg):
    # device bytes planned per mode: the bpa streams are held at their worst case (8 bytes
    # per entry plus an 8-byte record per slot and operator, against 2 bytes + a 4-byte
    # scale for BF16, and for A_hat 2 more bytes per entry: the low halves of promoted
    # vertices); the additive cycle adds two vectors per level and injection maps, BPX
    # one more vector per coarse level
    g = mg.Grid(2, 5)
    base = mg.hier_footprint(g)
    bf16 = mg.hier_footprint(g, precision="mixed_bf16")
    bpa = mg.hier_footprint(g, precision="mixed_bpa")
    coarse = sum(g.info(lv).n_slots for lv in range(1, 5))
    assert bpa - bf16 == coarse * (9 * 4 + 25 * 6 + 2 * 4)
    add = mg.hier_footprint(g, cycle="additive")
    allv = sum(g.info(lv).n_slots for lv in range(1, 6))
    assert add - base == allv * 16 + coarse * 4
    assert mg.hier_footprint(g, cycle="bpx") - add == coarse * 8
    assert mg.hier_footprint(g, smoother="block") == base
