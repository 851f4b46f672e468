"""ctypes binding of libmg.so (argument marshalling only; every step runs in the library)."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmg.so")

MG_OK = 0
STATUS_NAMES = {
    0: "MG_OK", 1: "MG_ERR_INVALID_ARG", 2: "MG_ERR_OOM", 3: "MG_ERR_CUDA", 4: "MG_ERR_NOT_CONVERGED",
    5: "MG_ERR_DIVERGED", 6: "MG_ERR_NONFINITE", 7: "MG_ERR_INDEFINITE_COARSE", 8: "MG_ERR_TIMEOUT",
    9: "MG_ERR_BUDGET", 10: "MG_ERR_UNSUPPORTED",
}

V_EXISTS, V_BOUNDARY, V_HANGING, V_REFINED = 1, 2, 4, 8
C_EXISTS, C_REFINED = 1, 2


class MgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class LevelInfo(C.Structure):
    _fields_ = [("level", C.c_int32), ("dim", C.c_int32), ("brick_edge", C.c_int32),
                ("slots_per_brick", C.c_int32), ("n_bricks", C.c_int64), ("n_slots", C.c_int64),
                ("n_dofs", C.c_int64), ("n_cells", C.c_int64), ("n_hanging", C.c_int64),
                ("slot_offset", C.c_int64), ("h", C.c_double)]


class Options(C.Structure):
    _fields_ = [("transfer", C.c_int32), ("coarse", C.c_int32), ("precision", C.c_int32),
                ("nu1", C.c_int32), ("nu2", C.c_int32), ("omega", C.c_double),
                ("coarsest_level", C.c_int32), ("inner_cycles", C.c_int32), ("use_graphs", C.c_int32),
                ("persistent", C.c_int32), ("eps_mf", C.c_double), ("smoother", C.c_int32),
                ("gs_sweeps", C.c_int32), ("cycle", C.c_int32), ("dynamic_coarsest", C.c_int32),
                ("tensor_coefficients", C.c_int32), ("ff_sweeps", C.c_int32)]


class SolveStats(C.Structure):
    _fields_ = [("cycles", C.c_int32), ("outer_steps", C.c_int32), ("rel_residual", C.c_double),
                ("r0_norm", C.c_double), ("solve_ms", C.c_double), ("history", C.POINTER(C.c_double)),
                ("history_capacity", C.c_int32), ("history_len", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("grid", C.c_void_p), ("eps", C.c_void_p), ("b", C.c_void_p), ("u", C.c_void_p),
                ("rel_tol", C.c_double), ("max_cycles", C.c_int32), ("reserved", C.c_int32)]


_P = C.c_void_p
_I32P = C.POINTER(C.c_int32)
_U8P = C.POINTER(C.c_uint8)
_F64P = C.POINTER(C.c_double)

_SIGS = {
    "mg_create_grid": (C.c_int, [C.c_int, C.c_int, C.POINTER(_U8P), C.POINTER(_P)]),
    "mg_grid_info": (C.c_int, [_P, C.c_int, C.POINTER(LevelInfo)]),
    "mg_grid_tables": (C.c_int, [_P, C.c_int, _I32P, _U8P, _U8P, _I32P, _I32P, _I32P, _F64P, _I32P, _I32P,
                                 _I32P, _I32P]),
    "mg_destroy_grid": (None, [_P]),
    "mg_default_options": (None, [C.POINTER(Options)]),
    "mg_hier_create": (C.c_int, [_P, C.POINTER(Options), C.POINTER(_P)]),
    "mg_hier_footprint": (C.c_int, [_P, C.POINTER(Options), C.POINTER(C.c_size_t)]),
    "mg_setup": (C.c_int, [_P, _P, _P]),
    "mg_setup_tensor": (C.c_int, [_P, _P, _P]),
    "mg_smooth": (C.c_int, [_P, C.c_int, _P, _P, C.c_int, _P]),
    "mg_residual": (C.c_int, [_P, C.c_int, _P, _P, _P, _F64P, _P]),
    "mg_smooth_f32": (C.c_int, [_P, C.c_int, _P, _P, C.c_int, _P]),
    "mg_residual_f32": (C.c_int, [_P, C.c_int, _P, _P, _P, _F64P, _P]),
    "mg_vcycle_f32": (C.c_int, [_P, _P, _P, _P]),
    "mg_residual_norm_noalloc": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, _P]),
    "mg_restrict": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "mg_prolong": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "mg_interpolate_hanging": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "mg_vcycle": (C.c_int, [_P, _P, _P, _P]),
    "mg_autotune": (C.c_int, [_P, C.POINTER(C.c_int32), _P]),
    "mg_solve": (C.c_int, [_P, _P, _P, C.c_double, C.c_int, C.POINTER(SolveStats), _P]),
    "mg_get_stencils": (C.c_int, [_P, C.c_int, _P, _P]),
    "mg_get_deltas": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "mg_get_codes": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, _P]),
    "mg_encode_deltas": (C.c_int, [C.c_int64, C.c_int, _P, C.c_int, _P, _P, _P]),
    "mg_encode_deltas_promote": (C.c_int, [C.c_int64, C.c_int, _P, _P, C.c_int, _P, _P, _P, _P]),
    "mg_get_code_lo": (C.c_int, [_P, C.c_int, _P, _P]),
    "mg_bpa_encode": (C.c_int, [C.c_int64, C.c_int32, _P, C.c_double, _P, _P, _P, _P, _P]),
    "mg_bpa_decode": (C.c_int, [C.c_int64, C.c_int32, _P, _P, C.c_int32, _P, _P]),
    "mg_get_bpa": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), _P]),
    "mg_batch_create": (C.c_int, [C.c_int, C.POINTER(_P), C.POINTER(_P)]),
    "mg_batch_solve": (C.c_int, [_P, C.POINTER(_P), C.POINTER(_P), C.c_double, C.c_int, C.POINTER(SolveStats), _P]),
    "mg_batch_setup": (C.c_int, [_P, C.POINTER(_P), _P]),
    "mg_batch_destroy": (None, [_P]),
    "mg_server_create": (C.c_int, [C.c_size_t, C.POINTER(Options), C.POINTER(_P)]),
    "mg_server_submit": (C.c_int, [_P, C.POINTER(Request), C.POINTER(C.c_uint64)]),
    "mg_server_poll": (C.c_int, [_P, C.c_uint64, C.c_int, C.POINTER(C.c_int), C.POINTER(SolveStats)]),
    "mg_server_info": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_size_t)]),
    "mg_server_destroy": (None, [_P]),
    "mg_get_coarsest": (C.c_int, [_P, C.POINTER(C.c_int32)]),
    "mg_destroy_hier": (None, [_P]),
    "mg_probe_fp64_fma": (C.c_int, [C.c_int64, C.c_int32, _P, C.POINTER(C.c_int64), _P]),
    "mg_last_error": (C.c_char_p, []),
    "mg_version": (C.c_char_p, []),
}

_lib = None


def load() -> C.CDLL:
    """Load libmg.so (built in-tree by ``paper_1607_00648_gb300.build``); fails loudly if missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1607_00648_gb300.build.build()")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def symbols() -> list[str]:
    return list(_SIGS)


def check(status: int, what: str = "") -> None:
    if status != MG_OK:
        msg = load().mg_last_error().decode(errors="replace")
        raise MgError(status, f"{what}: {msg}" if what else msg)


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))
