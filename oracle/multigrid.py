"""Multigrid hierarchy, smoother, transfers, V-cycle and solve (oracle; test infrastructure only).

Sect. 4.1 / Alg. 1 of the paper: multiplicative V(mu_pre, mu_post) cycles with
omega-damped point Jacobi, u <- u + omega diag(A)^-1 (b - A u).  On a uniform
grid with Galerkin coarse operators the FAS / HTMG coarse equation of Sect. 3
reduces exactly to the correction scheme A_{l-1} e = R r, so the textbook
recursive V-cycle written here is the paper's method.  The coarsest level is
solved directly (dense FP64), as in the paper's exact coarse-grid variants.

Hierarchy options:
* transfer = 'dlinear' | 'boxmg' (Sect. 4.4)
* coarse   = 'redisc'  | 'galerkin' (Sect. 4.3)
* smoother = 'jacobi'  | 'block' (Sect. 4.2: block Jacobi, Gauss-Seidel sweeps on the
  iota vertices of every 3^d patch, then damped Jacobi on the c and gamma vertices)
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import boxmg, fem, galerkin
from .spacetree import Spacetree


@dataclass
class LevelOps:
    A: sp.csr_matrix            # operator over DoF rows/cols (slot numbering)
    st: np.ndarray              # full 3^d stencils (slot x offset)
    st_redisc: np.ndarray       # rediscretised 3^d stencils from the level's cell eps
    diag: np.ndarray            # diagonal per slot (1 on non-DoF slots)
    dof: np.ndarray
    P: sp.csr_matrix | None = None      # prolongation from level l-1 to l
    a_hat: np.ndarray | None = None     # A - A_redisc (coarse levels)
    p_hat: np.ndarray | None = None     # P - P_dlin, 5^d per slot of level l-1 (stored on this object for transfer l-1 -> l)
    extra: dict = field(default_factory=dict)


# Dynamic coarsest level (Sect. 4.3): the paper starts from the coarsest level 1 and
# raises it (a) at once when a Galerkin computation gives a coarse stencil that is not
# diagonally dominant or has a non-positive diagonal, (b) between two cycles when the
# residual stagnates or grows.  Readings: dominance is checked on the operator over the
# unknowns (entries towards Dirichlet vertices multiply 0), with a relative rounding
# allowance; (a) makes the coarsest level the one above the finest failing level; (b)
# raises it by one level after a cycle whose residual contraction exceeds STALL.
AUDIT_REL = 1e-12
STALL = 0.95


def audit_rows(A: sp.csr_matrix, dof: np.ndarray) -> np.ndarray:
    """Per slot: True where a DoF row of A (over DoF columns) has a non-positive
    diagonal or sum |off-diagonal| > (1 + AUDIT_REL) |diagonal| (not diagonally dominant)."""
    A = A.tocsr()
    diag = np.asarray(A.diagonal())
    absum = np.asarray(abs(A).sum(axis=1)).ravel()
    off = absum - np.abs(diag)
    fail = (diag <= 0.0) | (off > (1.0 + AUDIT_REL) * np.abs(diag))
    return fail & dof


def raised_coarsest(failing_levels, coarsest: int) -> int:
    """Rule (a): one level above the finest level whose audit failed (or unchanged)."""
    return max([coarsest] + [lv + 1 for lv in failing_levels])


def stalled(hist) -> bool:
    """Rule (b): the last cycle contracted the residual by less than a factor 1/STALL."""
    return len(hist) >= 2 and hist[-2] > 0 and hist[-1] > STALL * hist[-2]


class Hierarchy:
    """Operators of a uniform spacetree hierarchy (levels ``coarsest`` .. max_level).

    dynamic_coarsest: apply the Sect. 4.3 rules above, with the coarsest level kept at
    most max_coarse_dofs unknowns (it is solved directly); a raise beyond that, or to the
    finest level, raises ValueError (no admissible coarsest level)."""

    def __init__(self, tree: Spacetree, leaf_eps: dict[int, np.ndarray], transfer: str = "boxmg",
                 coarse: str = "galerkin", omega: float = 0.6, nu1: int = 2, nu2: int = 2,
                 coarsest: int = 1, smoother: str = "jacobi", gs_sweeps: int = 1,
                 dynamic_coarsest: bool = False, max_coarse_dofs: int = 1024):
        self.tree, self.omega, self.nu1, self.nu2, self.coarsest = tree, omega, nu1, nu2, coarsest
        self.smoother, self.gs_sweeps = smoother, gs_sweeps
        self.transfer, self.coarse = transfer, coarse
        L = tree.max_level
        self.L = L
        self.eps = fem.coarse_eps(tree, leaf_eps)
        self.ops: dict[int, LevelOps] = {}
        for lv in range(L, coarsest - 1, -1):
            level = tree.levels[lv]
            A_full = fem.assemble(tree, lv, self.eps[lv])
            st_r = fem.stencils(tree, lv, A_full)
            if lv == L or coarse == "redisc":
                A = fem.restrict_to_dofs(A_full, level.dof)
                st = st_r
                a_hat = None if lv == L else np.zeros_like(st_r)
            else:
                fine = self.ops[lv + 1]
                A = galerkin.galerkin(fine.A, fine.P)
                st = galerkin.full_coarse_stencils(tree, lv, A, st_r)
                a_hat = galerkin.a_delta(st, st_r, level.dof)
            diag = np.asarray(A.diagonal()).copy()
            diag[~level.dof] = 1.0
            ops = LevelOps(A=A, st=st, st_redisc=st_r, diag=diag, dof=level.dof, a_hat=a_hat)
            self.ops[lv] = ops
            if lv > coarsest:
                ops.P = boxmg.prolongation(tree, lv, st, kind=transfer)
                ops.p_hat = galerkin.p_delta(tree, lv, ops.P)
        self.dynamic, self.max_coarse_dofs = dynamic_coarsest, max_coarse_dofs
        if dynamic_coarsest:
            failing = [lv for lv in range(coarsest, L) if audit_rows(self.ops[lv].A, self.ops[lv].dof).any()]
            self.failing_levels = failing
            self.set_coarsest(raised_coarsest(failing, coarsest))
            self.setup_coarsest = self.coarsest
        else:
            self.set_coarsest(coarsest)

    def set_coarsest(self, c: int) -> None:
        """Solve level c directly from now on (levels below it are left out)."""
        if c >= self.L or int(self.ops[c].dof.sum()) > self.max_coarse_dofs and self.dynamic:
            raise ValueError(f"no admissible coarsest level: level {c} of {self.L}")
        self.coarsest = c
        o = self.ops[c]
        idx = np.nonzero(o.dof)[0]
        self._coarse_idx = idx
        self._coarse_dense = o.A[idx][:, idx].toarray()

    # --- single steps -----------------------------------------------------
    def smooth(self, lv: int, u: np.ndarray, b: np.ndarray, nu: int) -> np.ndarray:
        """nu smoothing steps: omega-damped Jacobi sweeps (Alg. 1 smoothing update), or
        block Jacobi steps (Sect. 4.2) with smoother='block'."""
        if self.smoother == "block":
            return self.block_smooth(lv, u, b, nu)
        o = self.ops[lv]
        u = u.copy()
        for _ in range(nu):
            r = b - o.A @ u
            u = u + np.where(o.dof, self.omega * r / o.diag, 0.0)
        return u

    def iota_vertices(self, lv: int) -> np.ndarray:
        """Slots of the iota DoFs of level lv (Sect. 4.2: vertices inside a 3^d patch, i.e.
        inside a level lv-1 cell: no coordinate a multiple of 3), patch by patch, within a
        patch in lexicographic order of the position (x fastest)."""
        o = self.ops[lv]
        c = self.tree.levels[lv].coords
        iota = o.dof & (c[:, 0] >= 0) & np.all(c % 3 != 0, axis=1)
        idx = np.nonzero(iota)[0]
        key = sorted(range(len(idx)), key=lambda j: (tuple((c[idx[j]] // 3)[::-1]), tuple(c[idx[j]][::-1])))
        return idx[key]

    def block_smooth(self, lv: int, u: np.ndarray, b: np.ndarray, nu: int) -> np.ndarray:
        """nu block Jacobi steps (Sect. 4.2).  Reading of the paper: a step first runs
        gs_sweeps Gauss-Seidel sweeps over the iota vertices of every patch (each vertex
        in turn: u_v += (b_v - (A u)_v) / A_vv with the current values), then one
        omega-damped Jacobi update of the c and gamma DoFs from the values the
        Gauss-Seidel sweeps left.  Patches share no iota vertex and no iota vertex is
        a neighbour of another patch's, so the patch order does not matter."""
        o = self.ops[lv]
        A = o.A.tocsr()
        order = self.iota_vertices(lv)
        not_iota = o.dof.copy()
        not_iota[order] = False
        u = u.copy()
        for _ in range(nu):
            for _s in range(self.gs_sweeps):
                for i in order:
                    lo, hi = A.indptr[i], A.indptr[i + 1]
                    r = b[i] - A.data[lo:hi] @ u[A.indices[lo:hi]]
                    u[i] += r / o.diag[i]
            r = b - A @ u
            u = u + np.where(not_iota, self.omega * r / o.diag, 0.0)
        return u

    def residual(self, lv: int, u: np.ndarray, b: np.ndarray) -> np.ndarray:
        o = self.ops[lv]
        return np.where(o.dof, b - o.A @ u, 0.0)

    def restrict(self, lv: int, r: np.ndarray) -> np.ndarray:
        """b_{l-1} = R r_l with R = P^T."""
        return self.ops[lv].P.T @ r

    def prolong(self, lv: int, e: np.ndarray) -> np.ndarray:
        """P e_{l-1} on level l."""
        return self.ops[lv].P @ e

    def coarse_solve(self, b: np.ndarray) -> np.ndarray:
        u = np.zeros_like(b)
        u[self._coarse_idx] = np.linalg.solve(self._coarse_dense, b[self._coarse_idx])
        return u

    # --- cycles -----------------------------------------------------------
    def vcycle(self, u: np.ndarray, b: np.ndarray, lv: int | None = None) -> np.ndarray:
        lv = self.L if lv is None else lv
        if lv == self.coarsest:
            return self.coarse_solve(b)
        u = self.smooth(lv, u, b, self.nu1)
        r = self.residual(lv, u, b)
        bc = self.restrict(lv, r)
        ec = self.vcycle(np.zeros_like(bc), bc, lv - 1)
        u = u + np.where(self.ops[lv].dof, self.prolong(lv, ec), 0.0)
        return self.smooth(lv, u, b, self.nu2)

    def solve(self, b: np.ndarray, rel_tol: float = 1e-10, max_cycles: int = 100):
        """V-cycles from u = 0 until ||r||_2 / ||r_0||_2 <= rel_tol; returns (u, history).
        With the dynamic coarsest level every solve starts from the level of rule (a)."""
        if self.dynamic and self.coarsest != self.setup_coarsest:
            self.set_coarsest(self.setup_coarsest)
        u = np.zeros_like(b)
        r0 = np.linalg.norm(self.residual(self.L, u, b))
        hist = [r0]
        for _ in range(max_cycles):
            if hist[-1] <= rel_tol * r0:
                break
            u = self.vcycle(u, b)
            hist.append(np.linalg.norm(self.residual(self.L, u, b)))
            if self.dynamic and stalled(hist) and self.coarsest + 1 < self.L and \
                    int(self.ops[self.coarsest + 1].dof.sum()) <= self.max_coarse_dofs:
                self.set_coarsest(self.coarsest + 1)  # rule (b), before the next cycle
        return u, np.array(hist)

    # --- additive multigrid (Alg. 2) --------------------------------------
    def inject(self, lv: int, u_fine: np.ndarray) -> np.ndarray:
        """I: a level lv-1 DoF takes the level-lv value at the same position (Sect. 3, rule 1)."""
        ch = self.tree.child_map(lv - 1)
        ok = self.ops[lv - 1].dof & (ch >= 0)
        out = np.zeros(ch.size)
        out[ok] = u_fine[ch[ok]]
        return out

    def additive_traversal(self, u: dict, d: dict, b: np.ndarray) -> None:
        """One grid traversal of the additive multigrid of Alg. 2, in place on the level
        iterates u[l] (u[L] is the solution) and corrections d[l], levels coarsest .. L.

        Coarse to fine (the descent): d_l += P d_{l-1} and u_l += P d_{l-1} (the coarse
        corrections of the previous traversal), the hierarchical surplus
        uh_l = u_l - P u_{l-1}, and the coarse right-hand sides cleared.  Fine to coarse
        (the ascent): r_l = b_l - A_l u_l, rh_l = b_l - A_l uh_l, d_l = omega D_l^-1 r_l,
        u_l += d_l, then u_{l-1} = I u_l and b_{l-1} = R rh_l.  Every level, the coarsest
        included, is smoothed; nothing is solved exactly."""
        L, c = self.L, self.coarsest
        uh, bb = {}, {}
        for lv in range(c, L + 1):
            dof = self.ops[lv].dof
            if lv > c:
                pd = np.where(dof, self.prolong(lv, d[lv - 1]), 0.0)
                d[lv] = d[lv] + pd
                u[lv] = u[lv] + pd
                uh[lv] = u[lv] - np.where(dof, self.prolong(lv, u[lv - 1]), 0.0)
            else:
                uh[lv] = u[lv].copy()
            bb[lv] = b if lv == L else np.zeros_like(u[lv])
        for lv in range(L, c - 1, -1):
            o = self.ops[lv]
            r = self.residual(lv, u[lv], bb[lv])
            rh = self.residual(lv, uh[lv], bb[lv])
            d[lv] = np.where(o.dof, self.omega * r / o.diag, 0.0)
            u[lv] = u[lv] + d[lv]
            if lv > c:
                u[lv - 1] = self.inject(lv, u[lv])
                bb[lv - 1] = np.where(self.ops[lv - 1].dof, self.restrict(lv, rh), 0.0)

    def c_points(self, lv: int) -> np.ndarray:
        """Slots of level lv that coincide with a level lv-1 vertex (every coordinate a
        multiple of 3): the c-points of Sect. 4.2 / Alg. 3."""
        c = self.tree.levels[lv].coords
        return (c[:, 0] >= 0) & np.all(c % 3 == 0, axis=1)

    def bpx_traversal(self, u: dict, d: dict, i: dict, b: np.ndarray) -> None:
        """One grid traversal of the BPX variant of Alg. 3, in place on u[l], d[l] and the
        injected skipped updates i[l].

        Reading of the paper: as Alg. 2, except that (a) on every level above the
        coarsest the c-points skip their own Jacobi update (u_l += d_l off the c-points
        only); their corrections are injected to the coarser level, i_{l-1} = I d_l, and
        then zeroed (d_l = 0 at c-points); (b) the descent applies P d_{l-1} at c-points
        and P d_{l-1} - P i_{l-1} elsewhere, to d_l and u_l; (c) the coarse iterates are
        not overwritten by injection (the printed surplus line lacks its u, read as
        uh_l = u_l - P u_{l-1}).  The coarsest level has no c-points."""
        L, c = self.L, self.coarsest
        uh, bb = {}, {}
        for lv in range(c, L + 1):
            dof = self.ops[lv].dof
            if lv > c:
                cp = self.c_points(lv)
                corr = (np.where(dof, self.prolong(lv, d[lv - 1]), 0.0)
                        - np.where(dof & ~cp, self.prolong(lv, i[lv - 1]), 0.0))
                d[lv] = d[lv] + corr
                u[lv] = u[lv] + corr
                uh[lv] = u[lv] - np.where(dof, self.prolong(lv, u[lv - 1]), 0.0)
            else:
                uh[lv] = u[lv].copy()
            bb[lv] = b if lv == L else np.zeros_like(u[lv])
        for lv in range(L, c - 1, -1):
            o = self.ops[lv]
            r = self.residual(lv, u[lv], bb[lv])
            rh = self.residual(lv, uh[lv], bb[lv])
            d[lv] = np.where(o.dof, self.omega * r / o.diag, 0.0)
            cp = self.c_points(lv) if lv > c else np.zeros_like(o.dof)
            u[lv] = u[lv] + np.where(cp, 0.0, d[lv])
            if lv > c:
                bb[lv - 1] = np.where(self.ops[lv - 1].dof, self.restrict(lv, rh), 0.0)
                i[lv - 1] = self.inject(lv, d[lv])
                d[lv] = np.where(cp, 0.0, d[lv])

    def bpx_solve(self, b: np.ndarray, rel_tol: float = 1e-10, max_cycles: int = 100):
        """BPX traversals from u = 0 until ||b - A u_L||_2 / ||b||_2 <= rel_tol."""
        L = self.L
        u = {lv: np.zeros(self.ops[lv].dof.size) for lv in range(self.coarsest, L + 1)}
        d = {lv: np.zeros_like(u[lv]) for lv in u}
        i = {lv: np.zeros_like(u[lv]) for lv in u}
        r0 = np.linalg.norm(self.residual(L, u[L], b))
        hist = [r0]
        for _ in range(max_cycles):
            if hist[-1] <= rel_tol * r0:
                break
            self.bpx_traversal(u, d, i, b)
            hist.append(np.linalg.norm(self.residual(L, u[L], b)))
        return u[L], np.array(hist)

    def additive_solve(self, b: np.ndarray, rel_tol: float = 1e-10, max_cycles: int = 100):
        """Additive traversals from u = 0 until ||b - A u_L||_2 / ||b||_2 <= rel_tol;
        returns (u_L, history of relative residuals)."""
        L = self.L
        u = {lv: np.zeros(self.ops[lv].dof.size) for lv in range(self.coarsest, L + 1)}
        d = {lv: np.zeros_like(u[lv]) for lv in u}
        r0 = np.linalg.norm(self.residual(L, u[L], b))
        hist = [r0]
        for _ in range(max_cycles):
            if hist[-1] <= rel_tol * r0:
                break
            self.additive_traversal(u, d, b)
            hist.append(np.linalg.norm(self.residual(L, u[L], b)))
        return u[L], np.array(hist)

    def direct(self, b: np.ndarray) -> np.ndarray:
        """Exact discrete solution of the finest level (sparse direct solve)."""
        o = self.ops[self.L]
        idx = np.nonzero(o.dof)[0]
        u = np.zeros_like(b)
        u[idx] = spla.spsolve(o.A[idx][:, idx].tocsc(), b[idx])
        return u
