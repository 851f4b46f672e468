"""Seeded synthetic inputs for the multigrid workloads.

This module is shared by the CPU oracle and by the CUDA path's callers (tests,
bench).  It holds no multigrid arithmetic: it only produces coefficient fields,
load vectors and refinement masks on integer grid coordinates, plus request
streams.  Arrays are indexed ``[x, y]`` or ``[x, y, z]`` (axis i = coordinate
i), cell arrays have ``3**level`` entries per axis (cell with lower-left corner
at that index), vertex arrays ``3**level + 1`` entries per axis.

Workloads follow the benchmark table of the paper (Sect. 7, Table
"parameters": ``sin`` with f = d*pi^2 * prod sin(pi x_i), zero Dirichlet data)
and the seeded recipes of the design notes (checkerboard, Gaussian random
field, sphere shell, Poisson arrivals).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "sin_load",
    "uniform_load",
    "checkerboard_eps",
    "constant_eps",
    "jump_eps",
    "unit_load",
    "lognormal_grf_eps",
    "sphere_shell_mask",
    "sphere_eps",
    "batch_problem_sizes",
    "poisson_arrivals",
]


def _vertex_coords(level: int, dim: int) -> list[np.ndarray]:
    n = 3**level
    x = np.arange(n + 1, dtype=np.float64) / n
    return np.meshgrid(*([x] * dim), indexing="ij")


def sin_load(level: int, dim: int) -> np.ndarray:
    """Lumped load b_v = h^d f(x_v) of the ``sin`` benchmark, f = d pi^2 prod sin(pi x_i).

    The exact solution of -Laplace(u) = f with zero Dirichlet data is prod sin(pi x_i).
    """
    h = 3.0**-level
    xs = _vertex_coords(level, dim)
    f = dim * math.pi**2 * np.prod([np.sin(math.pi * x) for x in xs], axis=0)
    return (h**dim) * f


def sin_solution(level: int, dim: int) -> np.ndarray:
    xs = _vertex_coords(level, dim)
    return np.prod([np.sin(math.pi * x) for x in xs], axis=0)


def uniform_load(level: int, dim: int, seed: int) -> np.ndarray:
    """Lumped load b_v = h^d f_v with f_v ~ U[-1, 1] drawn per vertex."""
    rng = np.random.default_rng(seed)
    n = 3**level + 1
    f = rng.uniform(-1.0, 1.0, size=(n,) * dim)
    return (3.0**-level) ** dim * f


def constant_eps(level: int, dim: int, value: float = 1.0) -> np.ndarray:
    return np.full((3**level,) * dim, float(value))


def jump_eps(level: int, dim: int, low: float = 1.0, high: float = 0.1) -> np.ndarray:
    """The paper's `jump` coefficient: `low` where the cell centre has x_1 < 0.5, else `high`."""
    n = 3**level
    xc = (np.arange(n) + 0.5) / n
    col = np.where(xc < 0.5, low, high)
    shape = [1] * dim
    shape[0] = n
    return np.broadcast_to(col.reshape(shape), (n,) * dim).astype(np.float64).copy()


def axis_checkerboard_eps(level: int, dim: int, low: float = 1.0, high: float = 0.1) -> np.ndarray:
    """The paper's `checkerboard` coefficient, a diagonal tensor per cell: eps_i = `low`
    where the cell centre has x_i < 0.5, else `high`.  Shape (3^level,)*dim + (dim,)."""
    n = 3**level
    xc = (np.arange(n) + 0.5) / n
    col = np.where(xc < 0.5, low, high)
    out = np.empty((n,) * dim + (dim,))
    for i in range(dim):
        shape = [1] * dim
        shape[i] = n
        out[..., i] = np.broadcast_to(col.reshape(shape), (n,) * dim)
    return out


def unit_load(level: int, dim: int) -> np.ndarray:
    """Lumped load b_v = h^d f with f = 1 (the paper's `jump` and `checkerboard` right-hand side)."""
    n = 3**level + 1
    return np.full((n,) * dim, (3.0**-level) ** dim)


def checkerboard_eps(level: int, dim: int, seed=0, tiles: int = 9,
                     values=(1.0, 1e-4)) -> np.ndarray:
    """Piecewise constant eps on ``tiles**dim`` tiles aligned with the grid.

    seed='alt' gives the deterministic alternating pattern; an integer seed
    draws each tile independently (p = 1/2) from ``default_rng(seed)``.
    """
    n = 3**level
    if n % tiles:
        raise ValueError("tiles must divide the cell count per axis")
    if seed == "alt":
        idx = np.indices((tiles,) * dim).sum(axis=0) % 2
    else:
        idx = np.random.default_rng(seed).integers(0, 2, size=(tiles,) * dim)
    tile_vals = np.where(idx == 0, values[0], values[1]).astype(np.float64)
    per = n // tiles
    out = tile_vals
    for ax in range(dim):
        out = np.repeat(out, per, axis=ax)
    return out


def lognormal_grf_eps(level: int, dim: int, sigma: float, seed: int,
                      corr_len: float = 0.1) -> np.ndarray:
    """eps = exp(sigma g), g a Gaussian random field with covariance exp(-r^2/(2 lambda^2)).

    Synthesised by FFT on the cell-centre grid padded x2 (periodic), normalised
    to unit sample variance, then rounded to FP32-representable doubles so
    that FP64 and FP32 consumers see the same coefficients.
    """
    n = 3**level
    m = 2 * n
    rng = np.random.default_rng(seed)
    freqs = np.fft.fftfreq(m, d=1.0 / n)  # cycles per unit length
    ks = np.meshgrid(*([freqs] * dim), indexing="ij")
    k2 = sum(k * k for k in ks)
    # spectral density of the squared-exponential kernel (up to a constant)
    spec = np.exp(-2.0 * (math.pi**2) * (corr_len**2) * k2)
    noise = rng.standard_normal((m,) * dim)
    field = np.fft.ifftn(np.fft.fftn(noise) * np.sqrt(spec)).real
    g = field[tuple(slice(0, n) for _ in range(dim))]
    g = (g - g.mean()) / g.std()
    eps = np.exp(sigma * g)
    return eps.astype(np.float32).astype(np.float64)


def lognormal_grf_eps_torch(level: int, dim: int, sigma: float, seed: int, corr_len: float = 0.1,
                            device: str = "cuda"):
    """The same recipe as lognormal_grf_eps, generated on a GPU with torch.fft (for
    fields too large to synthesise quickly on the host); returns an FP64 torch tensor
    indexed [x, y(, z)].  Its random stream is torch's, not numpy's."""
    import torch

    n = 3**level
    m = 2 * n
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    freqs = torch.fft.fftfreq(m, d=1.0 / n, device=device, dtype=torch.float64)
    ks = torch.meshgrid(*([freqs] * dim), indexing="ij")
    k2 = sum(k * k for k in ks)
    spec = torch.exp(-2.0 * (math.pi**2) * (corr_len**2) * k2)
    noise = torch.randn((m,) * dim, generator=gen, device=device, dtype=torch.float64)
    field = torch.fft.ifftn(torch.fft.fftn(noise) * torch.sqrt(spec)).real
    g = field[tuple(slice(0, n) for _ in range(dim))]
    g = (g - g.mean()) / g.std()
    return torch.exp(sigma * g).float().double()


def sphere_shell_mask(level: int, dim: int = 3, radius: float = 0.3,
                      centre=(0.5, 0.5, 0.5)) -> np.ndarray:
    """Refinement mask on a uniform level: cells whose box grown by one cell meets |x-c| = r."""
    n = 3**level
    h = 1.0 / n
    lo = (np.arange(n) - 1) * h
    hi = (np.arange(n) + 2) * h
    c = centre[:dim]
    # nearest and farthest distance from the centre to the grown box, per axis
    near_ax, far_ax = [], []
    for ax in range(dim):
        near = np.maximum(np.maximum(lo - c[ax], c[ax] - hi), 0.0)
        far = np.maximum(np.abs(lo - c[ax]), np.abs(hi - c[ax]))
        near_ax.append(near)
        far_ax.append(far)
    grids_n = np.meshgrid(*near_ax, indexing="ij")
    grids_f = np.meshgrid(*far_ax, indexing="ij")
    dn = np.sqrt(sum(g * g for g in grids_n))
    df = np.sqrt(sum(g * g for g in grids_f))
    return (dn <= radius) & (df >= radius)


def sphere_eps(level: int, dim: int = 3, radius: float = 0.3, inside: float = 1e3,
               outside: float = 1.0, centre=(0.5, 0.5, 0.5)) -> np.ndarray:
    """eps per cell: ``inside`` where the cell centre lies inside the sphere."""
    n = 3**level
    x = (np.arange(n) + 0.5) / n
    xs = np.meshgrid(*([x] * dim), indexing="ij")
    r2 = sum((xs[i] - centre[i]) ** 2 for i in range(dim))
    return np.where(r2 < radius * radius, inside, outside).astype(np.float64)


def batch_problem_sizes(n_problems: int, seed: int, exponents=(3, 4, 5, 6)) -> np.ndarray:
    """Edge exponents m (edge = 3^m cells) drawn uniformly over ``exponents``."""
    rng = np.random.default_rng(seed)
    return rng.choice(np.asarray(exponents), size=n_problems)


def poisson_arrivals(n_requests: int, rate_per_s: float, seed: int,
                     edges=(3, 4, 5), weights=(6, 3, 1)):
    """Arrival times (s) with exponential gaps and per-request edge exponents."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=n_requests)
    w = np.asarray(weights, dtype=np.float64)
    ex = rng.choice(np.asarray(edges), size=n_requests, p=w / w.sum())
    return np.cumsum(gaps), ex
