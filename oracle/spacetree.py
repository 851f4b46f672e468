"""Spacetree flattening into level arrays (oracle; test infrastructure only).

Follows Sect. 3 of the paper (k = 3 spacetree, cell levels, hanging / refined /
unrefined vertices) and App. A (depth-first traversal = Peano curve).  The
level layout is the build's reading of the SFC order:

* bricks: the level-l descendants of one level-(l-m) cell, m = min(l, 3) in 2D
  and min(l, 2) in 3D, so a brick is 27^2 or 9^3 cells (smaller on coarse levels);
* bricks are ordered along the Peano curve of their root cells;
* inside a brick, vertex slots are lexicographic (x fastest), padded to a
  multiple of 32 slots; slot k of brick b is vertex brick_origin + lex(k);
* a cell shares the slot of its lower-left corner vertex;
* a brick is allocated iff it, or a brick at root offset -e (e in {0,1}^d),
  holds an existing level-l cell (so every corner of an existing cell has a slot).

Everything is computed here by literal recursion / brute force, independently
of the CUDA library's host builder.
"""
from __future__ import annotations

import itertools

import numpy as np

EXISTS, BOUNDARY, HANGING, REFINED = 1, 2, 4, 8
CELL_EXISTS, CELL_REFINED = 1, 2
SLOT_ALIGN = 32
_MAX_BRICK_DEPTH = {1: 3, 2: 3, 3: 2}


def brick_depth(level: int, dim: int) -> int:
    return min(level, _MAX_BRICK_DEPTH[dim])


def slots_per_brick(level: int, dim: int) -> int:
    nb = (3 ** brick_depth(level, dim)) ** dim
    return ((nb + SLOT_ALIGN - 1) // SLOT_ALIGN) * SLOT_ALIGN


def peano_cells(level: int, dim: int) -> list[tuple[int, ...]]:
    """All cells of a complete level in Peano order, by recursive descent.

    The Peano index has ternary digits t_1 t_2 ... (d digits per level, axis 0
    first).  A digit of axis i maps to the coordinate digit t or 2 - t, the
    latter iff the sum of all earlier digits of the other axes is odd (Peano's
    classic serpentine map; depth-first order for k = 3, Sect. 3 / App. A).
    """
    order: list[tuple[int, ...]] = []

    def descend(pos: int, coords: list[int], sums: list[int]) -> None:
        if pos == level * dim:
            order.append(tuple(coords))
            return
        axis = pos % dim
        others = sum(sums) - sums[axis]
        for t in range(3):
            a = t if others % 2 == 0 else 2 - t
            c = list(coords)
            c[axis] = 3 * c[axis] + a
            s = list(sums)
            s[axis] += t
            descend(pos + 1, c, s)

    descend(0, [0] * dim, [0] * dim)
    return order


def offsets(dim: int, radius: int = 1) -> np.ndarray:
    """Offsets in [-radius, radius]^d, lexicographic with x fastest."""
    rng = range(-radius, radius + 1)
    return np.array([tuple(reversed(t)) for t in itertools.product(rng, repeat=dim)], dtype=np.int64)


def corners(dim: int) -> np.ndarray:
    """Cell corner offsets e in {0,1}^d, lexicographic with x fastest."""
    return np.array([tuple(reversed(t)) for t in itertools.product((0, 1), repeat=dim)], dtype=np.int64)


def _upsample(a: np.ndarray) -> np.ndarray:
    for ax in range(a.ndim):
        a = np.repeat(a, 3, axis=ax)
    return a


class Level:
    """Tables of one level of the spacetree (see module docstring for the layout)."""

    def __init__(self, grid: "Spacetree", level: int):
        d = grid.dim
        self.level, self.dim = level, d
        n = 3**level
        self.n = n
        self.h = 1.0 / n
        m = brick_depth(level, d)
        B = 3**m
        self.B = B
        self.S = slots_per_brick(level, d)
        nb_axis = 3 ** (level - m)
        cells = grid.cells[level]
        refined = grid.refined[level]

        # bricks holding existing cells, then the allocation rule
        shape = []
        for _ in range(d):
            shape += [nb_axis, B]
        has = cells.reshape(shape).any(axis=tuple(range(1, 2 * d, 2)))
        alloc = np.zeros_like(has)
        for e in corners(d):
            src = tuple(slice(0, nb_axis - e[i]) for i in range(d))
            dst = tuple(slice(e[i], nb_axis) for i in range(d))
            alloc[dst] |= has[src]
        roots = [c for c in peano_cells(level - m, d) if alloc[c]]
        self.brick_roots = np.array(roots, dtype=np.int64).reshape(-1, d)
        self.n_bricks = len(roots)
        brick_rank = np.full((nb_axis,) * d, -1, dtype=np.int64)
        for i, r in enumerate(roots):
            brick_rank[r] = i
        self.n_slots = self.n_bricks * self.S

        nloc = B**d
        k = np.arange(nloc)
        local = np.stack([(k // B**i) % B for i in range(d)], axis=1)
        coords = np.full((self.n_slots, d), -1, dtype=np.int64)
        pos2slot = np.full((n,) * d, -1, dtype=np.int64)
        for i, r in enumerate(roots):
            g = np.asarray(r) * B + local
            coords[i * self.S: i * self.S + nloc] = g
            pos2slot[tuple(g.T)] = i * self.S + k
        self.coords = coords
        self.pos2slot = pos2slot
        valid = coords[:, 0] >= 0
        self.valid = valid

        # vertex flags (Sect. 3: hanging / refined / unrefined)
        cpad = np.pad(cells, 1)
        rpad = np.pad(refined, 1)
        n_adj = np.zeros(self.n_slots, dtype=np.int64)
        n_ref = np.zeros(self.n_slots, dtype=np.int64)
        xv = coords[valid]
        for e in corners(d):
            idx = tuple((xv[:, i] - e[i] + 1) for i in range(d))
            n_adj[valid] += cpad[idx]
            n_ref[valid] += rpad[idx]
        full = 2**d
        vflags = np.zeros(self.n_slots, dtype=np.uint8)
        exists = n_adj > 0
        boundary = exists & valid & np.any(np.where(valid[:, None], coords == 0, False), axis=1)
        interior = exists & ~boundary
        hanging = interior & (n_adj < full)
        refd = interior & (n_adj == full) & (n_ref == full)
        vflags[exists] |= EXISTS
        vflags[boundary] |= BOUNDARY
        vflags[hanging] |= HANGING
        vflags[refd] |= REFINED
        self.vflags = vflags
        self.dof = interior & ~hanging

        cflags = np.zeros(self.n_slots, dtype=np.uint8)
        cidx = tuple(xv[:, i] for i in range(d))
        cflags[valid] |= np.where(cells[cidx], CELL_EXISTS, 0).astype(np.uint8)
        cflags[valid] |= np.where(refined[cidx], CELL_REFINED, 0).astype(np.uint8)
        self.cflags = cflags

        # neighbour table: slot of x + o, -1 if outside the domain or unallocated
        offs = offsets(d)
        nbr = np.full((self.n_slots, len(offs)), -1, dtype=np.int64)
        for j, o in enumerate(offs):
            y = xv + o
            inside = np.all((y >= 0) & (y < n), axis=1)
            col = np.full(len(xv), -1, dtype=np.int64)
            col[inside] = pos2slot[tuple(y[inside].T)]
            nbr[valid, j] = col
        self.nbr = nbr

        # per-cell vertex ids
        cv = np.full((self.n_slots, full), -1, dtype=np.int64)
        for j, e in enumerate(corners(d)):
            y = xv + e
            inside = np.all(y < n, axis=1)
            col = np.full(len(xv), -1, dtype=np.int64)
            col[inside] = pos2slot[tuple(y[inside].T)]
            cv[valid, j] = col
        self.cell_vertices = cv

        # brick neighbour table
        bn = np.full((self.n_bricks, len(offs)), -1, dtype=np.int64)
        for i, r in enumerate(roots):
            for j, o in enumerate(offs):
                q = np.asarray(r) + o
                if np.all((q >= 0) & (q < nb_axis)):
                    bn[i, j] = brick_rank[tuple(q)]
        self.brick_nbr = bn

    def slot_of(self, pos) -> int:
        pos = tuple(int(p) for p in pos)
        if any(p < 0 or p >= self.n for p in pos):
            return -1
        return int(self.pos2slot[pos])


class Spacetree:
    """k = 3 spacetree refined by per-level masks (Sect. 3).

    ``refine_masks[l]`` is a boolean array over the complete level l (shape
    (3^l,)*d); an existing cell refines iff its entry is set.  A level without
    a mask refines every existing cell, up to ``max_level``.
    """

    def __init__(self, dim: int, max_level: int, refine_masks: dict | None = None):
        self.dim, self.max_level = dim, max_level
        masks = refine_masks or {}
        self.cells = [np.ones((1,) * dim, dtype=bool)]
        self.refined = []
        for lv in range(max_level):
            mk = masks.get(lv)
            r = self.cells[lv] & (np.asarray(mk, dtype=bool) if mk is not None else True)
            self.refined.append(r)
            self.cells.append(_upsample(r))
        self.refined.append(np.zeros_like(self.cells[max_level]))
        self.levels = [Level(self, lv) for lv in range(max_level + 1)]

    # hanging-vertex interpolation map (Sect. 3, rule 2: d-linear interpolant of the coarser level)
    def hanging_map(self, level: int):
        lv = self.levels[level]
        d = self.dim
        full = 2**d
        idx = np.full((lv.n_slots, full), -1, dtype=np.int64)
        w = np.zeros((lv.n_slots, full), dtype=np.float64)
        if level == 0:
            return idx, w
        coarse = self.levels[level - 1]
        for s in np.nonzero(lv.vflags & HANGING)[0]:
            x = lv.coords[s]
            c = x // 3
            r = x % 3
            for j, e in enumerate(corners(d)):
                wt = 1.0
                for i in range(d):
                    f = (r[i] / 3.0) if e[i] else ((3 - r[i]) / 3.0)
                    wt = f if i == 0 else wt * f
                if wt == 0.0:
                    continue
                sl = coarse.slot_of(c + e)
                if sl >= 0:
                    idx[s, j] = sl
                    w[s, j] = wt
        return idx, w

    # injection map: fine slot -> coarse slot at the same position (Sect. 3, rule 1)
    def parent_map(self, level: int) -> np.ndarray:
        lv = self.levels[level]
        out = np.full(lv.n_slots, -1, dtype=np.int64)
        if level == 0:
            return out
        coarse = self.levels[level - 1]
        for s in np.nonzero(lv.valid)[0]:
            x = lv.coords[s]
            if np.all(x % 3 == 0):
                out[s] = coarse.slot_of(x // 3)
        return out

    def child_map(self, level: int) -> np.ndarray:
        lv = self.levels[level]
        out = np.full(lv.n_slots, -1, dtype=np.int64)
        if level == self.max_level:
            return out
        fine = self.levels[level + 1]
        for s in np.nonzero(lv.valid)[0]:
            out[s] = fine.slot_of(3 * lv.coords[s])
        return out

    # ---- field marshalling between coordinate arrays and slot vectors ----
    def cells_to_slots(self, level: int, field: np.ndarray) -> np.ndarray:
        lv = self.levels[level]
        out = np.zeros(lv.n_slots)
        v = lv.valid
        out[v] = field[tuple(lv.coords[v].T)]
        return out

    def vertices_to_slots(self, level: int, field: np.ndarray, mask_dof: bool = True) -> np.ndarray:
        lv = self.levels[level]
        out = np.zeros(lv.n_slots)
        v = lv.valid
        out[v] = field[tuple(lv.coords[v].T)]
        if mask_dof:
            out[~lv.dof] = 0.0
        return out

    def slots_to_vertices(self, level: int, vec: np.ndarray) -> np.ndarray:
        lv = self.levels[level]
        out = np.zeros((lv.n + 1,) * self.dim)
        v = lv.valid
        out[tuple(lv.coords[v].T)] = vec[v]
        return out
