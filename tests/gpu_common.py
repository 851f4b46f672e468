"""Shared fixtures of the GPU parity tests: build a case on both sides from the same seeded inputs."""
from __future__ import annotations

import os

import numpy as np

from oracle import multigrid
from oracle import spacetree as stt
import synthetic as syn

# Unit roundoff of FP64.
U64 = 2.0 ** -53

# Parity bound of multi-step FP64 outputs (V-cycles, block steps, traversals, solves)
# against the oracle, as an infinity-norm relative difference:
#     |gpu - oracle|_inf / |oracle|_inf  <=  U64 * (C1 + C2 * F),
# F the cancellation factor of the hierarchy (Case.amplification: the largest
# sum|terms| / |sum| over the coarse Galerkin diagonals; 1 without Galerkin operators).
# Two correct FP64 evaluations of a Galerkin entry differ by up to a small multiple of
# U64 * sum|terms| (Higham's bound for a sum), i.e. U64 * F relative to the diagonal,
# and a cycle's coarse corrections inherit that perturbation (the C2 F term); the
# smoothing and transfer arithmetic itself adds a few hundred roundings (the C1 term).
# Measured on the GPU (err / U64 of every check is recorded and printed at the end of
# the session): the C1 term, largest where F is small, reaches 1969 u (a 3D V-cycle on
# the sphere coefficient, F = 68) and 1351 u (the 3D solve); with heavy cancellation the
# error follows 0.02-0.05 F (2D checkerboard, F = 7.2e5 at level 4 and 5.8e7 at level 6).
# The constants keep a margin of at least 6x over every measured error.  On the
# composite grid the two-level FAS cycle amplifies rounding beyond F (measured 10,700 u
# per cycle and 42,700 u per solve at F = 118), so it has its own C1.
BOUNDS = {
    "cycle": (2.0 ** 14, 0.25),
    "solve": (2.0 ** 14, 0.5),
    # float-float finest sweeps: their roundings are 2^-46 instead of 2^-53 (the C1 term
    # grows by 2^7); the Galerkin setup stays FP64 (same C2 F term)
    "ff_cycle": (2.0 ** 21, 0.25),
    "ff_solve": (2.0 ** 21, 0.5),
    "ff_composite_solve": (2.0 ** 26, 0.0),
    "composite_cycle": (2.0 ** 17, 0.0),
    "composite_solve": (2.0 ** 19, 0.0),
}
# residual histories (relative residuals, down to 1e-10) of two correct solves: the
# residual b - A u cancels, so each carries an absolute rounding of order 1e-16 |b|;
# measured: within 4e-9 relative plus 1.2e-13 absolute (the 2D composite solve's tail)
HIST_RTOL, HIST_ATOL = 4e-9, 5e-13

# (check, err / U64, F, bound / U64) of every comparison of the session
OBSERVED: list = []


def parity_bound(amp: float, kind: str) -> float:
    c1, c2 = BOUNDS[kind]
    return U64 * (c1 + c2 * max(float(amp), 1.0))


def parity_check(name: str, err: float, amp: float, kind: str) -> None:
    """Record err / U64 and assert err <= U64 (C1 + C2 F) for the kind of output."""
    bound = parity_bound(amp, kind)
    OBSERVED.append((name, float(err) / U64, float(amp), bound / U64))
    assert err <= bound, f"{name}: err {err:.3e} = {err / U64:.1f} u > bound {bound / U64:.1f} u (F = {amp:.3e})"


def lib():
    import paper_1607_00648_gb300 as mg
    from paper_1607_00648_gb300 import build

    if not os.path.exists(mg._lib.LIB_PATH):
        build.build()
    mg.load()
    return mg


def eps_field(kind: str, L: int, dim: int, seed: int = 0) -> np.ndarray:
    if kind == "const":
        return syn.constant_eps(L, dim)
    if kind == "checker":
        return syn.checkerboard_eps(L, dim, seed=seed, tiles=9 if L >= 2 else 3)
    if kind == "checker3":
        return syn.checkerboard_eps(L, dim, seed=seed, tiles=3)
    if kind == "sphere":
        return syn.sphere_eps(L, dim)
    if kind == "jump":
        return syn.jump_eps(L, dim)
    if kind == "grf":
        return syn.lognormal_grf_eps(L, dim, sigma=2.0, seed=1000 + seed)
    raise ValueError(kind)


class Case:
    """One problem on the CPU oracle and on the GPU library, same slot numbering."""

    def __init__(self, dim, L, eps_kind="checker", transfer="boxmg", coarse="galerkin", precision="fp64",
                 seed=0, omega=0.6, nu1=2, nu2=2, load="uniform", oracle=True, persistent=0, eps_mf=None,
                 smoother="jacobi", gs_sweeps=1, ff_sweeps=0):
        import torch

        self.mg = lib()
        self.torch = torch
        self.dim, self.L = dim, L
        self.eps = eps_field(eps_kind, L, dim, seed)
        self.grid = self.mg.Grid(dim, L)
        extra = {} if eps_mf is None else {"eps_mf": eps_mf}
        if smoother != "jacobi":
            extra.update(smoother=smoother, gs_sweeps=gs_sweeps)
        if ff_sweeps:
            extra.update(ff_sweeps=ff_sweeps)
        self.H = self.mg.Hierarchy(self.grid, transfer=transfer, coarse=coarse, precision=precision,
                                   omega=omega, nu1=nu1, nu2=nu2, persistent=persistent, **extra)
        eps_cat = self.grid.cells_to_concat({L: self.eps})
        self.eps_dev = torch.from_numpy(eps_cat).cuda()
        self.H.setup(self.eps_dev)
        torch.cuda.synchronize()
        self.tree = stt.Spacetree(dim, L) if oracle else None
        self.O = (multigrid.Hierarchy(self.tree, {L: self.eps}, transfer=transfer, coarse=coarse, omega=omega,
                                      nu1=nu1, nu2=nu2, smoother=smoother, gs_sweeps=gs_sweeps)
                  if oracle else None)
        if load == "sin":
            bf = syn.sin_load(L, dim)
        elif load == "unit":
            bf = syn.unit_load(L, dim)
        else:
            bf = syn.uniform_load(L, dim, seed + 1)
        self.b = self.grid.to_slots(L, bf)
        self.b_dev = torch.from_numpy(self.b).cuda()

    def n(self, level):
        return self.grid.info(level).n_slots

    def dof(self, level):
        return self.grid.dof_mask(level)

    def dev(self, a):
        return self.torch.from_numpy(np.ascontiguousarray(a)).cuda()

    def host(self, t):
        self.torch.cuda.synchronize()
        return t.cpu().numpy()

    def abs_scale(self, level):
        """Per-entry magnitude scale of the floating-point sums behind a level's stencils.

        S_L = |A_L| on the finest level and S_{l-1} = |P|^T S_l |P| below (Galerkin):
        the forward error of a sum is bounded by (number of terms) * u * sum |terms|
        (Higham), so two correct FP64 evaluations of an entry differ by at most a small
        multiple of u * S.  Returned in the 3^d stencil view (slot x offset).
        """
        from oracle import fem

        if not hasattr(self, "_S"):
            S = {self.L: abs(self.O.ops[self.L].A)}
            for lv in range(self.L - 1, 0, -1):
                if self.O.coarse == "galerkin":
                    P = abs(self.O.ops[lv + 1].P)
                    S[lv] = (P.T @ S[lv + 1] @ P).tocsr()
                else:
                    S[lv] = abs(self.O.ops[lv].A)
            self._S = S
        st = np.maximum(fem.stencils(self.tree, level, self._S[level]), np.abs(self.O.ops[level].st))
        # floor: 1e-4 of the row's scale (the oracle's quadrature leaves ~1e-17 where the
        # element matrix has exact zeros, e.g. 3D face neighbours)
        return np.maximum(st, 1e-4 * st.max(axis=1, keepdims=True))

    def amplification(self):
        """Largest cancellation factor sum|terms| / |sum| of a coarse Galerkin diagonal."""
        if not hasattr(self, "_amp"):
            amp = 1.0
            for lv in range(1, self.L):
                S = self.abs_scale(lv)
                dof = self.dof(lv)
                c = 3**self.dim // 2
                amp = max(amp, float((S[dof, c] / np.abs(self.O.ops[lv].st[dof, c])).max()))
            self._amp = amp
        return self._amp

    def random_vec(self, level, seed):
        rng = np.random.default_rng(seed)
        v = rng.standard_normal(self.n(level))
        v[~self.dof(level)] = 0.0
        return v


def rel_inf(a, b):
    """max |a - b| / max |b| (infinity-norm relative error)."""
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def rowwise_rel(a, b):
    """max over rows of max |a - b| / max |b| within the row."""
    den = np.abs(b).max(axis=1)
    den = np.where(den > 0, den, 1.0)
    return (np.abs(a - b).max(axis=1) / den).max()


def galerkin_amplification(O, tree, L, dim):
    """Case.amplification for an oracle hierarchy O over `tree` with finest level L."""
    from oracle import fem

    S = {L: abs(O.ops[L].A)}
    amp = 1.0
    c = 3**dim // 2
    for lv in range(L - 1, 0, -1):
        S[lv] = (abs(O.ops[lv + 1].P).T @ S[lv + 1] @ abs(O.ops[lv + 1].P)).tocsr() if O.coarse == "galerkin" \
            else abs(O.ops[lv].A)
        st = fem.stencils(tree, lv, S[lv])
        dof = tree.levels[lv].dof
        amp = max(amp, float((st[dof, c] / np.abs(O.ops[lv].st[dof, c])).max()))
    return amp


_FULL: dict = {}


def full_size_checker_solve():
    """2D level 6 (529,984 DoFs), seeded 9x9 checkerboard {1, 1e-4}, BoxMG + Galerkin, FP64:
    the Case and the oracle's solve to a 1e-10 drop (computed once per session)."""
    if "c" not in _FULL:
        c = Case(2, 6, "checker")
        ref, hist = c.O.solve(c.b, 1e-10, 400)
        _FULL.update(c=c, ref=ref, hist=hist)
    return _FULL["c"], _FULL["ref"], _FULL["hist"]
