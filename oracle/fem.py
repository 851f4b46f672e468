"""d-linear finite-element operators on spacetree levels (oracle; test infrastructure only).

Sect. 4 of the paper: the operator of -div(eps grad u) discretised with
d-linear shape functions gives 3^d-point stencils; a stencil splits additively
over the 2^d cells adjacent to its vertex (eq. "03_solver:stencils").  Here the
element matrix is the plain definition K_ij = int_cell grad phi_i . grad phi_j,
integrated by tensor Gauss-Legendre quadrature (exact for these polynomials),
and level operators are assembled cell by cell into scipy sparse matrices.

eps is a scalar per cell, or a diagonal tensor (eps_1, ..., eps_d) per cell (eq. (1)
allows a diagonal diffusion tensor; the paper's `checkerboard` benchmark sets eps_i
by the coordinate x_i): a coordinate array with a trailing axis of length d.  The
tensor case uses the directional element matrices K^(i)_ab = int d_i phi_a d_i phi_b,
whose sum is K.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

from .spacetree import CELL_EXISTS, Spacetree, corners, offsets


def element_matrix(dim: int, h: float) -> np.ndarray:
    """K_ij = int over a cube of side h of grad phi_i . grad phi_j (corners lex, x fastest).

    phi_e(xi) = prod_i (xi_i if e_i else 1 - xi_i) on the reference cube; the
    chain rule gives grad_x = grad_xi / h and dx = h^d dxi, so K scales as h^(d-2).
    """
    return sum(directional_element_matrices(dim, h))


def directional_element_matrices(dim: int, h: float) -> list[np.ndarray]:
    """[K^(i)] with K^(i)_ab = int over a cube of side h of d_i phi_a d_i phi_b (same
    quadrature and scaling as ``element_matrix``)."""
    gp, gw = np.polynomial.legendre.leggauss(2)
    gp = 0.5 * (gp + 1.0)
    gw = 0.5 * gw
    cs = corners(dim)
    K = [np.zeros((len(cs), len(cs))) for _ in range(dim)]
    for q in itertools.product(range(2), repeat=dim):
        xi = np.array([gp[i] for i in q])
        wq = np.prod([gw[i] for i in q])
        grads = np.zeros((len(cs), dim))
        for a, e in enumerate(cs):
            for i in range(dim):
                g = 1.0 if e[i] else -1.0
                for j in range(dim):
                    if j != i:
                        g *= xi[j] if e[j] else 1.0 - xi[j]
                grads[a, i] = g
        for i in range(dim):
            K[i] += wq * np.outer(grads[:, i], grads[:, i])
    return [k * h ** (dim - 2) for k in K]


def coarse_eps(tree: Spacetree, leaf_eps: dict[int, np.ndarray]) -> dict[int, np.ndarray]:
    """Cell coefficients on every level, as coordinate arrays.

    Leaf cells take the given values; a refined cell takes the arithmetic mean
    of its 3^d children (the build's reading where the paper leaves the coarse
    rediscretisation coefficient open, Sect. 4.3 / Sect. 5).
    """
    d = tree.dim
    tail = next(iter(leaf_eps.values())).shape[d:]  # () scalar, (d,) diagonal tensor
    ext = (slice(None),) * d + (None,) * len(tail)
    out: dict[int, np.ndarray] = {}
    for lv in range(tree.max_level, -1, -1):
        n = 3**lv
        e = np.zeros((n,) * d + tail)
        if lv in leaf_eps:
            e = np.where((tree.cells[lv] & ~tree.refined[lv])[ext], leaf_eps[lv], 0.0)
        if lv < tree.max_level:
            child = out[lv + 1]
            shape = []
            for _ in range(d):
                shape += [n, 3]
            mean = child.reshape(shape + list(tail)).mean(axis=tuple(range(1, 2 * d, 2)))
            e = np.where(tree.refined[lv][ext], mean, e)
        out[lv] = e
    return out


def assemble(tree: Spacetree, level: int, eps_cells: np.ndarray) -> sp.csr_matrix:
    """Full level operator over all slots (boundary and hanging rows included).

    Sums eps_c K_c over every existing level-l cell c into the rows and columns
    of its 2^d corner slots.  ``eps_cells`` is a coordinate array of the level.
    """
    lv = tree.levels[level]
    d = tree.dim
    tensor = eps_cells.ndim == d + 1
    K = directional_element_matrices(d, lv.h) if tensor else element_matrix(d, lv.h)
    rows, cols, vals = [], [], []
    cell_slots = np.nonzero((lv.cflags & CELL_EXISTS) != 0)[0]
    cv = lv.cell_vertices[cell_slots]
    ec = eps_cells[tuple(lv.coords[cell_slots].T)]
    for a in range(2**d):
        for b in range(2**d):
            ok = (cv[:, a] >= 0) & (cv[:, b] >= 0)
            rows.append(cv[ok, a])
            cols.append(cv[ok, b])
            if tensor:
                vals.append(sum(ec[ok, i] * K[i][a, b] for i in range(d)))
            else:
                vals.append(ec[ok] * K[a, b])
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(lv.n_slots, lv.n_slots))
    return A.tocsr()


def restrict_to_dofs(A: sp.spmatrix, dof_rows: np.ndarray, dof_cols: np.ndarray | None = None) -> sp.csr_matrix:
    """Zero every row / column that is not a degree of freedom (Dirichlet elimination)."""
    if dof_cols is None:
        dof_cols = dof_rows
    Dr = sp.diags(dof_rows.astype(np.float64))
    Dc = sp.diags(dof_cols.astype(np.float64))
    return (Dr @ A @ Dc).tocsr()


def stencils(tree: Spacetree, level: int, A: sp.spmatrix) -> np.ndarray:
    """3^d stencil view of a full operator: st[v, k] = A[v, nbr(v, k)] (0 where nbr = -1)."""
    lv = tree.levels[level]
    A = A.tocsr()
    st = np.zeros(lv.nbr.shape)
    for k in range(lv.nbr.shape[1]):
        col = lv.nbr[:, k]
        ok = col >= 0
        rows = np.nonzero(ok)[0]
        st[rows, k] = np.asarray(A[rows, col[ok]]).ravel()
    return st


def stencils_to_matrix(tree: Spacetree, level: int, st: np.ndarray, dof_only: bool = True) -> sp.csr_matrix:
    """Inverse of :func:`stencils`: rows of DoF slots, columns restricted to DoF slots."""
    lv = tree.levels[level]
    rows, cols, vals = [], [], []
    for k in range(lv.nbr.shape[1]):
        col = lv.nbr[:, k]
        ok = col >= 0
        if dof_only:
            ok &= lv.dof & np.where(col >= 0, lv.dof[np.maximum(col, 0)], False)
        rows.append(np.nonzero(ok)[0])
        cols.append(col[ok])
        vals.append(st[ok, k])
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(lv.n_slots, lv.n_slots)).tocsr()


def offsets_radius1(dim: int) -> np.ndarray:
    return offsets(dim, 1)
