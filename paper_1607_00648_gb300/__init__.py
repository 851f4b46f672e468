"""GB300-native quasi-matrix-free hybrid multigrid (arXiv:1607.00648 hot path).

Python face of libmg.so: every compute step runs in the library's CUDA kernels;
this package only marshals arguments (numpy / torch tensors -> pointers).
PyTorch provides device memory and streams.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import MgError, Options, SolveStats, check, load

__all__ = ["Batch", "Server", "Grid", "Hierarchy", "MgError", "bpa_decode", "bpa_encode", "default_options",
           "encode_deltas", "encode_deltas_promote", "load", "probe_fp64_fma"]

TRANSFER = {"dlinear": 0, "boxmg": 1}
COARSE = {"redisc": 0, "galerkin": 1}
PRECISION = {"fp64": 0, "mixed_bf16": 1, "mixed_fp16": 2, "mixed_bpa": 3}
SMOOTHER = {"jacobi": 0, "block": 1}
CYCLE = {"v": 0, "additive": 1, "bpx": 2}


def _stream_ptr(stream) -> C.c_void_p:
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dptr(t) -> C.c_void_p:
    return C.c_void_p(t.data_ptr())


class Grid:
    """Flattened k = 3 spacetree (mg_create_grid); host object."""

    def __init__(self, dim: int, max_level: int, refine_masks: dict | None = None):
        lib = load()
        self.dim, self.max_level = dim, max_level
        self._masks = []
        arr = None
        if refine_masks:
            arr = (_lib._U8P * max_level)()
            for lv in range(max_level):
                m = refine_masks.get(lv)
                if m is None:
                    arr[lv] = C.cast(None, _lib._U8P)
                else:
                    # lexicographic with x fastest == numpy [x, y(, z)] array in Fortran order
                    mb = np.asfortranarray(np.asarray(m, dtype=np.uint8)).ravel(order="F").copy()
                    self._masks.append(mb)
                    arr[lv] = _lib._ptr(mb, C.c_uint8)
        h = C.c_void_p()
        check(lib.mg_create_grid(dim, max_level, arr, C.byref(h)), "mg_create_grid")
        self._h = h
        self._tables: dict = {}

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            load().mg_destroy_grid(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def info(self, level: int) -> _lib.LevelInfo:
        inf = _lib.LevelInfo()
        check(load().mg_grid_info(self._h, level, C.byref(inf)), "mg_grid_info")
        return inf

    def tables(self, level: int) -> dict:
        if level in self._tables:
            return self._tables[level]
        inf = self.info(level)
        n, d = inf.n_slots, self.dim
        t = {
            "coords": np.empty((n, d), np.int32), "vflags": np.empty(n, np.uint8),
            "cflags": np.empty(n, np.uint8), "nbr": np.empty((n, 3**d), np.int32),
            "cell_vertices": np.empty((n, 2**d), np.int32), "hang_idx": np.empty((n, 2**d), np.int32),
            "hang_w": np.empty((n, 2**d), np.float64), "parent": np.empty(n, np.int32),
            "child": np.empty(n, np.int32), "brick_roots": np.empty((inf.n_bricks, d), np.int32),
            "brick_nbr": np.empty((inf.n_bricks, 3**d), np.int32),
        }
        P = _lib._ptr
        check(load().mg_grid_tables(
            self._h, level, P(t["coords"], C.c_int32), P(t["vflags"], C.c_uint8), P(t["cflags"], C.c_uint8),
            P(t["nbr"], C.c_int32), P(t["cell_vertices"], C.c_int32), P(t["hang_idx"], C.c_int32),
            P(t["hang_w"], C.c_double), P(t["parent"], C.c_int32), P(t["child"], C.c_int32),
            P(t["brick_roots"], C.c_int32), P(t["brick_nbr"], C.c_int32)), "mg_grid_tables")
        self._tables[level] = t
        return t

    def n_slots_total(self) -> int:
        inf = self.info(self.max_level)
        return int(inf.slot_offset + inf.n_slots)

    # ---- marshalling between coordinate arrays and the library's slot order ----
    def dof_mask(self, level: int) -> np.ndarray:
        f = self.tables(level)["vflags"]
        return ((f & _lib.V_EXISTS) != 0) & ((f & (_lib.V_BOUNDARY | _lib.V_HANGING)) == 0)

    def to_slots(self, level: int, field: np.ndarray, dof_only: bool = True) -> np.ndarray:
        c = self.tables(level)["coords"]
        ok = c[:, 0] >= 0
        out = np.zeros(len(c))
        out[ok] = field[tuple(c[ok].T)]
        if dof_only:
            out[~self.dof_mask(level)] = 0.0
        return out

    def cells_to_concat(self, leaf_eps: dict) -> np.ndarray:
        """Level-concatenated cell-slot array from per-level coordinate arrays of leaf cells."""
        out = np.zeros(self.n_slots_total())
        for lv, field in leaf_eps.items():
            inf = self.info(lv)
            out[inf.slot_offset: inf.slot_offset + inf.n_slots] = self.to_slots(lv, field, dof_only=False)
        return out


def default_options(**kw) -> Options:
    o = Options()
    load().mg_default_options(C.byref(o))
    for k, v in kw.items():
        if k == "transfer":
            v = TRANSFER[v] if isinstance(v, str) else v
        elif k == "coarse":
            v = COARSE[v] if isinstance(v, str) else v
        elif k == "precision":
            v = PRECISION[v] if isinstance(v, str) else v
        elif k == "smoother":
            v = SMOOTHER[v] if isinstance(v, str) else v
        elif k == "cycle":
            v = CYCLE[v] if isinstance(v, str) else v
        setattr(o, k, v)
    return o


def hier_footprint(grid, **options) -> int:
    """Device bytes a hierarchy of this grid and options would hold."""
    o = default_options(**options)
    n = C.c_size_t()
    check(load().mg_hier_footprint(grid.handle, C.byref(o), C.byref(n)), "mg_hier_footprint")
    return n.value


class Hierarchy:
    """Device-resident multigrid hierarchy of a grid (mg_hier_create / mg_setup / solvers)."""

    def __init__(self, grid: Grid, **options):
        self.grid = grid
        self.options = default_options(**options)
        h = C.c_void_p()
        check(load().mg_hier_create(grid.handle, C.byref(self.options), C.byref(h)), "mg_hier_create")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            load().mg_destroy_hier(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def setup(self, eps, stream=None):
        check(load().mg_setup(self._h, _dptr(eps), _stream_ptr(stream)), "mg_setup")

    def setup_tensor(self, eps_axes, stream=None):
        """mg_setup_tensor: eps_axes (d * n,) device FP64, one level-concatenated array per axis."""
        check(load().mg_setup_tensor(self._h, _dptr(eps_axes), _stream_ptr(stream)), "mg_setup_tensor")

    def smooth(self, level, u, b, nu, stream=None):
        check(load().mg_smooth(self._h, level, _dptr(u), _dptr(b), nu, _stream_ptr(stream)), "mg_smooth")

    def residual(self, level, u, b, r, want_norm=False, stream=None):
        n2 = C.c_double(0.0)
        check(load().mg_residual(self._h, level, _dptr(u), _dptr(b), _dptr(r),
                                 C.byref(n2) if want_norm else None, _stream_ptr(stream)), "mg_residual")
        return n2.value if want_norm else None

    def smooth_f32(self, level, u, b, nu, stream=None):
        check(load().mg_smooth_f32(self._h, level, _dptr(u), _dptr(b), nu, _stream_ptr(stream)), "mg_smooth_f32")

    def residual_f32(self, level, u, b, r, want_norm=False, stream=None):
        n2 = C.c_double(0.0)
        check(load().mg_residual_f32(self._h, level, _dptr(u), _dptr(b), _dptr(r),
                                     C.byref(n2) if want_norm else None, _stream_ptr(stream)), "mg_residual_f32")
        return n2.value if want_norm else None

    def vcycle_f32(self, u, b, stream=None):
        check(load().mg_vcycle_f32(self._h, _dptr(u), _dptr(b), _stream_ptr(stream)), "mg_vcycle_f32")

    def restrict(self, fine_level, r_fine, b_coarse, stream=None):
        check(load().mg_restrict(self._h, fine_level, _dptr(r_fine), _dptr(b_coarse), _stream_ptr(stream)),
              "mg_restrict")

    def prolong(self, fine_level, e_coarse, u_fine, stream=None):
        check(load().mg_prolong(self._h, fine_level, _dptr(e_coarse), _dptr(u_fine), _stream_ptr(stream)),
              "mg_prolong")

    def interpolate_hanging(self, level, u_coarse, u_fine, stream=None):
        check(load().mg_interpolate_hanging(self._h, level, _dptr(u_coarse), _dptr(u_fine), _stream_ptr(stream)),
              "mg_interpolate_hanging")

    def autotune(self, stream=None) -> dict:
        """Time each level's smoother per slab depth and keep the fastest (mg_autotune);
        returns {level: (fp64 depth, fp32 depth)} with 0 where a type was not tuned."""
        L = self.grid.max_level
        chosen = (C.c_int32 * (2 * (L + 1)))()
        check(load().mg_autotune(self._h, chosen, _stream_ptr(stream)), "mg_autotune")
        return {lv: (chosen[2 * lv], chosen[2 * lv + 1]) for lv in range(self.options.coarsest_level, L + 1)}

    def vcycle(self, u, b, stream=None):
        check(load().mg_vcycle(self._h, _dptr(u), _dptr(b), _stream_ptr(stream)), "mg_vcycle")

    def solve(self, u, b, rel_tol=1e-10, max_cycles=500, stream=None, history=256, raise_on_fail=True):
        st = SolveStats()
        hist = np.zeros(history)
        st.history = hist.ctypes.data_as(C.POINTER(C.c_double))
        st.history_capacity = history
        status = load().mg_solve(self._h, _dptr(u), _dptr(b), rel_tol, max_cycles, C.byref(st),
                                 _stream_ptr(stream))
        if raise_on_fail:
            check(status, "mg_solve")
        return {"status": status, "cycles": st.cycles, "outer_steps": st.outer_steps,
                "rel_residual": st.rel_residual, "r0_norm": st.r0_norm, "solve_ms": st.solve_ms,
                "history": hist[: st.history_len].copy()}

    def get_stencils(self, level, out, stream=None):
        check(load().mg_get_stencils(self._h, level, _dptr(out), _stream_ptr(stream)), "mg_get_stencils")

    def get_deltas(self, level, a_hat=None, p_hat=None, stream=None):
        check(load().mg_get_deltas(self._h, level, _dptr(a_hat) if a_hat is not None else None,
                                   _dptr(p_hat) if p_hat is not None else None, _stream_ptr(stream)),
              "mg_get_deltas")

    def get_codes(self, level, a_codes=None, a_scale=None, p_codes=None, p_scale=None, stream=None):
        f = lambda t: _dptr(t) if t is not None else None
        check(load().mg_get_codes(self._h, level, f(a_codes), f(a_scale), f(p_codes), f(p_scale),
                                  _stream_ptr(stream)), "mg_get_codes")

    def coarsest(self) -> int:
        """The level this hierarchy solves directly (after the dynamic rule, if enabled)."""
        c = C.c_int32()
        check(load().mg_get_coarsest(self._h, C.byref(c)), "mg_get_coarsest")
        return int(c.value)

    def get_code_lo(self, level, a_lo, stream=None):
        check(load().mg_get_code_lo(self._h, level, _dptr(a_lo), _stream_ptr(stream)), "mg_get_code_lo")

    def get_bpa(self, level, a_rec=None, a_stream=None, p_rec=None, p_stream=None, stream=None):
        """Copies of a bpa hierarchy's records / byte streams of a coarse level; returns the
        streams' lengths (a_bytes, p_bytes).  Synchronises."""
        f = lambda t: _dptr(t) if t is not None else None
        ab, pb = C.c_uint64(), C.c_uint64()
        check(load().mg_get_bpa(self._h, level, f(a_rec), f(a_stream), f(p_rec), f(p_stream), C.byref(ab),
                                C.byref(pb), _stream_ptr(stream)), "mg_get_bpa")
        return ab.value, pb.value


class Batch:
    """Many set-up hierarchies solved together (mg_batch_create / mg_batch_solve)."""

    def __init__(self, hierarchies):
        self.hiers = list(hierarchies)  # keep the handles alive as long as the batch
        arr = (C.c_void_p * len(self.hiers))(*[h.handle.value for h in self.hiers])
        h = C.c_void_p()
        check(load().mg_batch_create(len(self.hiers), arr, C.byref(h)), "mg_batch_create")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            load().mg_batch_destroy(h)
            self._h = None

    def setup(self, eps_list, stream=None):
        n = len(self.hiers)
        ea = (C.c_void_p * n)(*[e.data_ptr() for e in eps_list])
        check(load().mg_batch_setup(self._h, ea, _stream_ptr(stream)), "mg_batch_setup")

    def solve(self, us, bs, rel_tol=1e-10, max_cycles=500, stream=None, raise_on_fail=True):
        n = len(self.hiers)
        ua = (C.c_void_p * n)(*[u.data_ptr() for u in us])
        ba = (C.c_void_p * n)(*[b.data_ptr() for b in bs])
        st = (SolveStats * n)()
        status = load().mg_batch_solve(self._h, ua, ba, rel_tol, max_cycles, st, _stream_ptr(stream))
        if raise_on_fail:
            check(status, "mg_batch_solve")
        return status, [{"cycles": s.cycles, "outer_steps": s.outer_steps, "rel_residual": s.rel_residual,
                         "r0_norm": s.r0_norm, "solve_ms": s.solve_ms} for s in st]


class Server:
    """Continuous-batching solve server (mg_server_*): submit requests, poll results."""

    def __init__(self, hbm_budget_bytes: int, **options):
        self.options = default_options(**options)
        h = C.c_void_p()
        check(load().mg_server_create(int(hbm_budget_bytes), C.byref(self.options), C.byref(h)), "mg_server_create")
        self._h = h
        self._keep = {}

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            load().mg_server_destroy(h)
            self._h = None

    def __del__(self):
        self.close()

    def submit(self, grid, eps, b, u, rel_tol=1e-8, max_cycles=500) -> int:
        req = _lib.Request(grid.handle.value, eps.data_ptr(), b.data_ptr(), u.data_ptr(), rel_tol, max_cycles, 0)
        t = C.c_uint64()
        check(load().mg_server_submit(self._h, C.byref(req), C.byref(t)), "mg_server_submit")
        self._keep[t.value] = (grid, eps, b, u)
        return t.value

    def poll(self, ticket: int, wait: bool = False):
        done = C.c_int(0)
        st = SolveStats()
        status = load().mg_server_poll(self._h, ticket, 1 if wait else 0, C.byref(done), C.byref(st))
        if not done.value:
            return None
        self._keep.pop(ticket, None)
        return {"status": status, "cycles": st.cycles, "rel_residual": st.rel_residual, "r0_norm": st.r0_norm,
                "latency_ms": st.solve_ms}

    def info(self):
        q, r, b = C.c_int64(), C.c_int64(), C.c_size_t()
        check(load().mg_server_info(self._h, C.byref(q), C.byref(r), C.byref(b)), "mg_server_info")
        return {"queued": q.value, "running": r.value, "bytes_in_use": b.value}


def encode_deltas_promote(delta, diag, codes, lo, scale, fmt: int, stream=None):
    """Rows of delta (n, k) FP64 with their reconstructed diagonals diag (n,) ->
    codes, lo (n, k) int16 views of uint16, scale (n,) float32 (sign = promotion flag)."""
    n, k = delta.shape
    check(load().mg_encode_deltas_promote(n, k, _dptr(delta), _dptr(diag), fmt, _dptr(codes), _dptr(lo),
                                          _dptr(scale), _stream_ptr(stream)), "mg_encode_deltas_promote")


def encode_deltas(delta, codes, scale, fmt: int, stream=None):
    n, k = delta.shape
    check(load().mg_encode_deltas(n, k, _dptr(delta), fmt, _dptr(codes), _dptr(scale), _stream_ptr(stream)),
          "mg_encode_deltas")


def bpa_encode(x, eps_mf: float, rec, stream_bytes, total, status=None, stream=None):
    """Rows of x (n, k) FP64 -> records rec (n,) int64 view of uint64, bytes (n*k*8,) uint8,
    total (1,) int64: the stream length; status (1,) int32, nullable."""
    n, k = x.shape
    check(load().mg_bpa_encode(n, k, _dptr(x), float(eps_mf), _dptr(rec), _dptr(stream_bytes), _dptr(total),
                               _dptr(status) if status is not None else None, _stream_ptr(stream)),
          "mg_bpa_encode")


def bpa_decode(rec, stream_bytes, out, stream=None):
    """Decode into out (n, k): FP64 (exact) or FP32 (as the FP32 cycle kernels decode)."""
    n, k = out.shape
    fp32 = 1 if out.element_size() == 4 else 0
    check(load().mg_bpa_decode(n, k, _dptr(rec), _dptr(stream_bytes), fp32, _dptr(out), _stream_ptr(stream)),
          "mg_bpa_decode")


def probe_fp64_fma(n_ctas: int, iters: int, sink, stream=None) -> int:
    """Enqueue the FP64 fma-rate probe (mg_probe_fp64_fma); returns the launch's flops."""
    fl = C.c_int64()
    check(load().mg_probe_fp64_fma(int(n_ctas), int(iters), _dptr(sink), C.byref(fl), _stream_ptr(stream)),
          "mg_probe_fp64_fma")
    return int(fl.value)
