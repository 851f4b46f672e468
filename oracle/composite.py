"""Adaptive composite grid: the system and its FAS cycle (oracle; test infrastructure only).

Sect. 3 of the paper (FAS on the hierarchical generating system): a refined
vertex holds the injected value of the finer vertex at its position (rule 1), a
hanging vertex holds the d-linear interpolant of the coarser level (rule 2), and
every level uses the same discretisation (rule 3).  For a spacetree that is
complete up to level T = L - 1 and refined to level L only in part, the
composite unknowns are the non-hanging level-L vertices and the unrefined level-T
vertices; their equations are

  (i)  at a level-L unknown: the level-L stencil applied with hanging neighbours
       interpolated from level T;
  (ii) at an unrefined level-T unknown: the level-T stencil applied with refined
       neighbours taking the injected level-L value.

Alg. 1's multiplicative cycle on this grid is the FAS two-level scheme below,
with the level-T coarse equation A_T (I u_L + e) = R r_L + A_T I u_L solved in
correction form by one V-cycle of the uniform levels T .. coarsest.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem, multigrid
from .boxmg import prolongation
from .spacetree import HANGING, REFINED, Spacetree


class Composite:
    def __init__(self, tree: Spacetree, leaf_eps: dict[int, np.ndarray], transfer: str = "boxmg",
                 coarse: str = "galerkin", omega: float = 0.6, nu1: int = 2, nu2: int = 2, coarsest: int = 1,
                 cycle: bool = True):
        """cycle=False builds the composite system only (fill, residual, matrix), not
        the transfer and the uniform sub-hierarchy that the cycle needs."""
        L = tree.max_level
        T = L - 1
        self.tree, self.L, self.T = tree, L, T
        self.omega, self.nu1, self.nu2 = omega, nu1, nu2
        d = tree.dim
        self.eps = fem.coarse_eps(tree, leaf_eps)
        fine, top = tree.levels[L], tree.levels[T]
        self.fine, self.top = fine, top
        self.A5 = fem.assemble(tree, L, self.eps[L]).tocsr()
        self.A4 = fem.restrict_to_dofs(fem.assemble(tree, T, self.eps[T]), top.dof)
        self.dof5 = fine.dof
        self.unref4 = top.dof & ((top.vflags & REFINED) == 0)
        self.ref4 = top.dof & ((top.vflags & REFINED) != 0)
        # hanging interpolation (level-L hanging slots from level-T slots)
        hi, hw = tree.hanging_map(L)
        rows, cols, vals = [], [], []
        for j in range(hi.shape[1]):
            ok = hi[:, j] >= 0
            rows.append(np.nonzero(ok)[0])
            cols.append(hi[ok, j])
            vals.append(hw[ok, j])
        self.Hmat = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                  shape=(fine.n_slots, top.n_slots))
        # injection: refined level-T slot <- level-L slot at the same position
        child = tree.child_map(T)
        ref = np.nonzero(self.ref4)[0]
        self.Inj = sp.csr_matrix((np.ones(len(ref)), (ref, child[ref])), shape=(top.n_slots, fine.n_slots))
        self.diag5 = np.where(self.dof5, self.A5.diagonal(), 1.0)
        if not cycle:
            return
        # d-linear transfer between the levels (the adaptive level has no BoxMG operator)
        self.P = prolongation(tree, L, None, "dlinear")
        # the uniform levels T .. coarsest as their own hierarchy
        self.sub = multigrid.Hierarchy(Spacetree(d, T), {T: self.eps[T]}, transfer=transfer, coarse=coarse,
                                       omega=omega, nu1=nu1, nu2=nu2, coarsest=coarsest)

    # --- the composite state: u5 (level-L slots), u4 (level-T slots) ---------------
    def fill(self, u5, u4):
        """Level-L values with hanging slots interpolated, level-T values with refined slots injected."""
        u5f = np.where(self.dof5, u5, 0.0) + self.Hmat @ np.where(self.unref4, u4, 0.0)
        u4f = np.where(self.unref4, u4, 0.0) + self.Inj @ np.where(self.dof5, u5, 0.0)
        return u5f, u4f

    def residual(self, u5, u4, b5, b4):
        u5f, u4f = self.fill(u5, u4)
        r5 = np.where(self.dof5, b5 - self.A5 @ u5f, 0.0)
        r4 = np.where(self.unref4, b4 - self.A4 @ u4f, 0.0)
        return r5, r4

    def smooth5(self, u5, u4, b5, nu):
        for _ in range(nu):
            u5f, _ = self.fill(u5, u4)
            r5 = b5 - self.A5 @ u5f
            u5 = np.where(self.dof5, u5 + self.omega * r5 / self.diag5, 0.0)
        return u5

    def cycle(self, u5, u4, b5, b4):
        """One composite FAS cycle (pre-smooth L, coarse correction on T..coarsest, post-smooth L)."""
        u5 = self.smooth5(u5, u4, b5, self.nu1)
        u5f, u4f = self.fill(u5, u4)
        r5 = np.where(self.dof5, b5 - self.A5 @ u5f, 0.0)
        # level-T correction right-hand side: R r_L on refined vertices, residual elsewhere
        r4 = np.where(self.ref4, self.P.T @ r5, np.where(self.unref4, b4 - self.A4 @ u4f, 0.0))
        e4 = self.sub.vcycle(np.zeros_like(r4), r4)
        u4 = np.where(self.unref4, u4 + e4, 0.0)
        u5 = np.where(self.dof5, u5 + self.P @ e4, 0.0)
        return self.smooth5(u5, u4, b5, self.nu2), u4

    def solve(self, b5, b4, rel_tol=1e-10, max_cycles=200):
        u5 = np.zeros_like(b5)
        u4 = np.zeros_like(b4)
        r5, r4 = self.residual(u5, u4, b5, b4)
        r0 = np.sqrt(r5 @ r5 + r4 @ r4)
        hist = [r0]
        for _ in range(max_cycles):
            if hist[-1] <= rel_tol * r0:
                break
            u5, u4 = self.cycle(u5, u4, b5, b4)
            r5, r4 = self.residual(u5, u4, b5, b4)
            hist.append(np.sqrt(r5 @ r5 + r4 @ r4))
        return u5, u4, np.array(hist)

    def matrix(self):
        """The composite system over x = (level-L unknowns, unrefined level-T unknowns)."""
        i5 = np.nonzero(self.dof5)[0]
        i4 = np.nonzero(self.unref4)[0]
        n = len(i5) + len(i4)
        E5 = sp.csr_matrix((np.ones(len(i5)), (i5, np.arange(len(i5)))), shape=(self.fine.n_slots, n))
        E4 = sp.csr_matrix((np.ones(len(i4)), (i4, len(i5) + np.arange(len(i4)))), shape=(self.top.n_slots, n))
        U5 = E5 + self.Hmat @ E4
        U4 = E4 + self.Inj @ E5
        M = sp.vstack([(self.A5 @ U5)[i5], (self.A4 @ U4)[i4]]).tocsr()
        return M, i5, i4

    def direct(self, b5, b4):
        M, i5, i4 = self.matrix()
        x = spla.spsolve(M.tocsc(), np.concatenate([b5[i5], b4[i4]]))
        u5 = np.zeros_like(b5)
        u4 = np.zeros_like(b4)
        u5[i5] = x[: len(i5)]
        u4[i4] = x[len(i5):]
        return u5, u4
