"""ctypes loader for libensemble_solve.so (the C ABI declared in include/ensemble_solve.h).

The library must have been built (``python -m paper_1711_10622_gb300.build`` or
``__graft_entry__.build()``); there is no fallback implementation.
"""

from __future__ import annotations

import ctypes
import os

from . import build as _build

ENS_OK, ENS_ERR_INVALID, ENS_ERR_OOM, ENS_ERR_CUDA, ENS_ERR_TIMEOUT, ENS_ERR_BUDGET, ENS_ERR_UNSUPPORTED = range(7)
STATUS_NAMES = {
    0: "ENS_OK",
    1: "ENS_ERR_INVALID",
    2: "ENS_ERR_OOM",
    3: "ENS_ERR_CUDA",
    4: "ENS_ERR_TIMEOUT",
    5: "ENS_ERR_BUDGET",
    6: "ENS_ERR_UNSUPPORTED",
}
ENS_F64, ENS_F32 = 0, 1
ENS_MATRIX_SINGULAR = 0x1
ENS_F64_AUTO, ENS_F64_NATIVE, ENS_F64_SPLIT, ENS_F64_HYBRID = 0, 1, 2, 3
COL_CONVERGED, COL_MAXITER, COL_BREAKDOWN, COL_NONFINITE, COL_INCOMPATIBLE = range(5)

_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_u32 = ctypes.c_uint32


ENS_PRECOND_NONE, ENS_PRECOND_CHEBYSHEV, ENS_PRECOND_AMG = 0, 1, 2
ENS_PREC_F64, ENS_PREC_MIXED = 0, 1


class SolveOpts(ctypes.Structure):
    """Mirror of ens_solve_opts (include/ensemble_solve.h)."""

    _fields_ = [
        ("max_iter", ctypes.c_int32),
        ("precond", ctypes.c_int32),
        ("cheb_steps", ctypes.c_int32),
        ("cheb_lo", ctypes.c_double),
        ("cheb_hi", ctypes.c_double),
        ("precision", ctypes.c_int32),
        ("inner_tol", ctypes.c_double),
        ("max_outer", ctypes.c_int32),
        ("inner_max_iter", ctypes.c_int32),
        ("check_every", ctypes.c_int32),
        ("x0_zero", ctypes.c_int32),
        ("use_graph", ctypes.c_int32),
        ("workspace", ctypes.c_void_p),
        ("workspace_bytes", ctypes.c_uint64),
    ]


class AmgOpts(ctypes.Structure):
    """Mirror of ens_amg_opts."""

    _fields_ = [
        ("theta", ctypes.c_double),
        ("max_levels", ctypes.c_int32),
        ("coarse_size", ctypes.c_int32),
        ("smooth_steps", ctypes.c_int32),
        ("coarse_steps", ctypes.c_int32),
        ("cheb_lo", ctypes.c_double),
        ("cheb_hi", ctypes.c_double),
    ]


class SolveStats(ctypes.Structure):
    """Mirror of ens_solve_stats."""

    _fields_ = [
        ("iters", ctypes.c_void_p),
        ("relres", ctypes.c_void_p),
        ("status", ctypes.c_void_p),
        ("outer", ctypes.c_void_p),
    ]


class BatchItem(ctypes.Structure):
    """Mirror of ens_batch_item."""

    _fields_ = [
        ("A", ctypes.c_void_p),
        ("m", ctypes.c_int32),
        ("B", ctypes.c_void_p),
        ("X", ctypes.c_void_p),
        ("tol", ctypes.c_void_p),
        ("stats", ctypes.POINTER(SolveStats)),
    ]


class EnsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None


def library_path() -> str:
    """The in-tree library, or the file named by ENSEMBLE_SOLVE_LIB (to load another build)."""
    return os.environ.get("ENSEMBLE_SOLVE_LIB") or _build.LIB


def lib():
    """Load libensemble_solve.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build it with `python -m paper_1711_10622_gb300.build` "
            "(there is no CPU fallback for the ensemble solver)"
        )
    L = ctypes.CDLL(path)
    sig = {
        "ens_create_matrix": (_i32, [_i64, _i64, _vp, _vp, _vp, _u32, _vp, ctypes.POINTER(_vp)]),
        "ens_destroy_matrix": (_i32, [_vp]),
        "ens_matrix_info": (_i32, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i32)]),
        "ens_set_f64_mode": (_i32, [_vp, _i32]),
        "ens_set_native_share": (_i32, [_vp, _i32]),
        "ens_set_untiled": (_i32, [_vp, _i32]),
        "ens_autotune": (
            _i32,
            [_vp, _i32, _i32, _vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_double)],
        ),
        "ens_gspmv": (_i32, [_vp, _i32, _i32, _vp, _vp, _vp]),
        "ens_tuned_variant": (_i32, [_vp, _i32, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
        "ens_gspmv_host": (_i32, [_vp, _i32, _i32, _vp, _vp, _vp]),
        "ens_gspmv_host_noalloc": (_i32, [_vp, _i32, _i32, _vp, _vp, _vp]),
        "ens_default_solve_opts": (None, [ctypes.POINTER(SolveOpts)]),
        "ens_solve_block": (
            _i32,
            [_vp, _i32, _vp, _vp, _vp, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveStats), _vp],
        ),
        "ens_solve_batch": (_i32, [_i32, ctypes.POINTER(BatchItem), ctypes.POINTER(SolveOpts), _vp]),
        "ens_solve_block_coupled": (
            _i32,
            [_vp, _i32, _vp, _vp, _vp, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveStats), _vp],
        ),
        "ens_create_grid": (_i32, [_i32, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_vp)]),
        "ens_destroy_grid": (_i32, [_vp]),
        "ens_grid_info": (_i32, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
        "ens_divergence": (_i32, [_vp, _i32, ctypes.c_double, _vp, _vp, _vp, _vp, _vp]),
        "ens_grad_correct": (_i32, [_vp, _i32, ctypes.c_double, _vp, _vp, _vp, _vp, _vp]),
        "ens_default_amg_opts": (None, [ctypes.POINTER(AmgOpts)]),
        "ens_amg_setup": (_i32, [_vp, ctypes.POINTER(AmgOpts), _vp]),
        "ens_amg_info": (_i32, [_vp, ctypes.POINTER(_i32), _vp, _vp]),
        "ens_amg_level": (_i32, [_vp, _i32, _vp, _vp, _vp, _vp]),
        "ens_amg_apply": (_i32, [_vp, _i32, _i32, _vp, _vp, _vp]),
        "ens_create_matrix_rect": (_i32, [_i64, _i64, _i64, _vp, _vp, _vp, _vp, ctypes.POINTER(_vp)]),
        "ens_matrix_shape": (_i32, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
        "ens_block_dots": (_i32, [_i64, _i32, _i32, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp, _vp]),
        "ens_block_lincomb": (_i32, [_i64, _i32, _i32, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp, _vp]),
        "ens_gather_rows": (_i32, [_i64, _i32, _vp, _vp, _vp, _vp]),
        "ens_last_error": (ctypes.c_char_p, []),
        "ens_last_workspace_bytes": (ctypes.c_uint64, []),
        "ens_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return _lib


def check(status: int):
    if status != ENS_OK:
        msg = lib().ens_last_error().decode(errors="replace")
        raise EnsError(status, msg)
