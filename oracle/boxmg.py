"""BoxMG operator-dependent prolongation (oracle; test infrastructure only).

Sect. 4.4 and App. C of the paper: per coarse cell (a patch of 3^d fine cells,
4^d fine vertices) and per corner coarse vertex, the 3^d entries of that
vertex's P stencil inside the patch solve one linear system C(s) p = f.  The
corner is first mirrored onto the reference corner (the bottom-left vertex),
the system is assembled there and solved, and the result is mirrored back.

Rows of C(s), unknowns p at reference positions r in {0,1,2}^d:
* the c-point r = 0 gets the row p = 1 (f = 1), everything else f = 0;
* a point r with Z = {axes with r_i = 0} not empty lies on a line (d = 2) or an
  edge / face (d = 3) through the corner: its stencil is collapsed by summing
  over the axes in Z, and it couples only to unknowns with the same zero axes;
* interior points (Z empty) use their full stencil;
* unknowns at reference coordinate 3 (the neighbouring coarse vertex) are 0.
For d = 2 this is exactly the 9 x 9 matrix printed in App. C (with the garbled
sixth row read as s_{5,0} ... s_{5,8}), and for d = 1 the 3 x 3 system of the
1D worked example.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .spacetree import Spacetree, corners, offsets


def reference_positions(dim: int) -> np.ndarray:
    """Unknown positions {0,1,2}^d, lexicographic with x fastest."""
    return offsets(dim, 1) + 1


def patch_positions(dim: int) -> np.ndarray:
    """Patch vertices {0,1,2,3}^d, lexicographic with x fastest (index i = x + 4y + 16z)."""
    k = np.arange(4**dim)
    return np.stack([(k // 4**i) % 4 for i in range(dim)], axis=1)


def system_matrix(s_ref: np.ndarray, dim: int) -> np.ndarray:
    """C(s) for stencils already in the reference orientation.

    s_ref: (..., 4^d, 3^d) stencils of the patch vertices (patch lex order,
    stencil offsets lex in {-1,0,1}^d).  Returns (..., 3^d, 3^d).
    """
    R = reference_positions(dim)
    O = offsets(dim, 1)
    nr = len(R)
    batch = s_ref.shape[:-2]
    C = np.zeros(batch + (nr, nr))
    pos_index = {tuple(r): j for j, r in enumerate(R)}
    for j, r in enumerate(R):
        if not np.any(r):
            C[..., j, j] = 1.0
            continue
        zero_axes = r == 0
        patch_vertex = int(sum(int(r[i]) * 4**i for i in range(dim)))
        for k, o in enumerate(O):
            t = r + np.where(zero_axes, 0, o)
            if np.any(t == 3):
                continue
            C[..., j, pos_index[tuple(t)]] += s_ref[..., patch_vertex, k]
    return C


def mirror_patch_stencils(s_patch: np.ndarray, corner: np.ndarray, dim: int) -> np.ndarray:
    """Reorder patch stencils so that ``corner`` becomes the reference (bottom-left) corner.

    Reference patch vertex r sits at actual patch position a_i = r_i or 3 - r_i
    (mirrored axes are those with corner_i = 1); stencil offsets flip sign on
    mirrored axes.
    """
    P = patch_positions(dim)
    O = offsets(dim, 1)
    flip = np.asarray(corner).astype(bool)
    a = np.where(flip, 3 - P, P)
    a_index = (a * (4 ** np.arange(dim))).sum(axis=1)
    o_act = np.where(flip, -O, O)
    o_index = ((o_act + 1) * (3 ** np.arange(dim))).sum(axis=1)
    return s_patch[..., a_index[:, None], o_index[None, :]]


def solve_corner(s_patch: np.ndarray, corner, dim: int) -> np.ndarray:
    """P entries of one corner vertex inside one (or a batch of) patch(es).

    Returns p[..., r] for reference positions r; the actual fine position of
    entry r is corner*3 mirrored: a_i = r_i or 3 - r_i.
    """
    s_ref = mirror_patch_stencils(s_patch, np.asarray(corner), dim)
    C = system_matrix(s_ref, dim)
    f = np.zeros(C.shape[:-1])
    f[..., 0] = 1.0
    return np.linalg.solve(C, f[..., None])[..., 0]


def dlinear_weight(o: np.ndarray) -> np.ndarray:
    """d-linear interpolation weight for fine offsets o in [-2, 2]^d from a coarse vertex (coarsening by 3)."""
    w1 = {0: 1.0, 1: 2.0 / 3.0, 2: 1.0 / 3.0}
    o = np.atleast_2d(o)
    out = np.ones(len(o))
    for i in range(o.shape[1]):
        out = out * np.array([w1[abs(int(v))] if abs(int(v)) <= 2 else 0.0 for v in o[:, i]])
    return out


def prolongation(tree: Spacetree, fine_level: int, fine_stencils: np.ndarray | None,
                 kind: str = "boxmg", return_raw: bool = False):
    """P from level fine_level-1 (columns, coarse slots) to fine_level (rows, fine slots).

    ``kind='dlinear'`` gives d-linear interpolation; ``kind='boxmg'`` solves
    C(s) p = f per refined coarse cell and corner with the fine 3^d stencils
    ``fine_stencils`` (slot x offset).  Only coarse DoF columns and fine DoF
    rows are filled.
    """
    d = tree.dim
    fine = tree.levels[fine_level]
    coarse = tree.levels[fine_level - 1]
    patch = patch_positions(d)
    R = reference_positions(d)
    rows, cols, vals = [], [], []
    ref_cells = np.argwhere(tree.refined[fine_level - 1])
    for e in corners(d):
        X = ref_cells + e
        inside = np.all(X < coarse.n, axis=1)
        Xs = np.full(len(X), -1, dtype=np.int64)
        Xs[inside] = coarse.pos2slot[tuple(X[inside].T)]
        keep = Xs >= 0
        keep[keep] &= coarse.dof[Xs[keep]]
        C0 = ref_cells[keep]
        cs = Xs[keep]
        if len(C0) == 0:
            continue
        # actual fine positions of the reference unknowns
        a = np.where(e.astype(bool), 3 - R, R)  # (3^d, d)
        fpos = 3 * C0[:, None, :] + a[None, :, :]
        fslot = fine.pos2slot[tuple(np.moveaxis(fpos, -1, 0))]
        if kind == "dlinear":
            off = fpos - 3 * (C0 + e)[:, None, :]
            p = dlinear_weight(off.reshape(-1, d)).reshape(len(C0), -1)
        else:
            ppos = 3 * C0[:, None, :] + patch[None, :, :]
            inside_p = np.all(ppos < fine.n, axis=2)
            pslot = np.full(ppos.shape[:2], -1, dtype=np.int64)
            pslot[inside_p] = fine.pos2slot[tuple(ppos[inside_p].T)]
            s_patch = np.where(pslot[..., None] >= 0, fine_stencils[np.maximum(pslot, 0)], 0.0)
            p = solve_corner(s_patch, e, d)
        ok = (fslot >= 0)
        ok &= np.where(fslot >= 0, fine.dof[np.maximum(fslot, 0)], False)
        rows.append(fslot[ok])
        cols.append(np.broadcast_to(cs[:, None], fslot.shape)[ok])
        vals.append(p[ok])
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    if return_raw:
        return r, c, v
    # entries shared by neighbouring patches (lines / faces through the corner) are
    # computed by each of them; keep one value per (fine, coarse) pair
    key = r * coarse.n_slots + c
    _, first = np.unique(key, return_index=True)
    return sp.csr_matrix((v[first], (r[first], c[first])), shape=(fine.n_slots, coarse.n_slots))


def stencil_of_P(tree: Spacetree, fine_level: int, P: sp.spmatrix) -> np.ndarray:
    """5^d view of P per coarse slot: out[X, k] = P[fine(3X + o_k), X], offsets o in [-2,2]^d lex."""
    d = tree.dim
    fine = tree.levels[fine_level]
    coarse = tree.levels[fine_level - 1]
    O = offsets(d, 2)
    Pr = P.tocsr()
    out = np.zeros((coarse.n_slots, len(O)))
    xs = np.nonzero(coarse.dof)[0]
    base = 3 * coarse.coords[xs]
    for k, o in enumerate(O):
        y = base + o
        inside = np.all((y >= 0) & (y < fine.n), axis=1)
        f = np.full(len(xs), -1, dtype=np.int64)
        f[inside] = fine.pos2slot[tuple(y[inside].T)]
        ok = f >= 0
        out[xs[ok], k] = np.asarray(Pr[f[ok], xs[ok]]).ravel()
    return out
