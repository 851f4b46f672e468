"""Galerkin coarse operators and hierarchical deltas (oracle; test infrastructure only).

Sect. 4.3: A_{l-1} = R A_l P with R = P^T (Sect. 4.4: R follows from R^T = P
unless stated otherwise), computed here by plain scipy sparse products over the
degrees of freedom.  Sect. 5: only the hierarchical differences
A_hat = A - A_rediscretised and P_hat = P - P_d-linear are stored.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fem
from .boxmg import dlinear_weight, stencil_of_P
from .spacetree import Spacetree, offsets


def galerkin(A_fine_dof: sp.spmatrix, P: sp.spmatrix) -> sp.csr_matrix:
    """R A P with R = P^T (plain definition)."""
    return (P.T @ A_fine_dof @ P).tocsr()


def full_coarse_stencils(tree: Spacetree, level: int, A_gal_dof: sp.spmatrix,
                         st_redisc: np.ndarray) -> np.ndarray:
    """3^d stencils of a Galerkin level: Galerkin entries where the neighbour is a
    DoF, rediscretised entries where it points to a non-DoF slot (boundary)."""
    lv = tree.levels[level]
    st_gal = fem.stencils(tree, level, A_gal_dof)
    nbr_dof = np.where(lv.nbr >= 0, lv.dof[np.maximum(lv.nbr, 0)], False)
    use_gal = nbr_dof & lv.dof[:, None]
    return np.where(use_gal, st_gal, st_redisc)


def a_delta(st_full: np.ndarray, st_redisc: np.ndarray, dof: np.ndarray) -> np.ndarray:
    """A_hat = A - A_rediscretised per DoF slot (Sect. 5)."""
    return np.where(dof[:, None], st_full - st_redisc, 0.0)


def p_delta(tree: Spacetree, fine_level: int, P: sp.spmatrix) -> np.ndarray:
    """P_hat = P - P_d-linear as a 5^d stencil per coarse DoF slot (Sect. 5)."""
    d = tree.dim
    coarse = tree.levels[fine_level - 1]
    Pst = stencil_of_P(tree, fine_level, P)
    w = dlinear_weight(offsets(d, 2))
    return np.where(coarse.dof[:, None], Pst - w[None, :], 0.0)
