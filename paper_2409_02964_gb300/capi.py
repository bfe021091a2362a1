"""ctypes binding of the C ABI in ``include/lbm_vanse.h``, same names, argument
marshalling only. Every computation runs in the CUDA library; if the library is
missing this module raises instead of falling back to anything else."""
from __future__ import annotations

import ctypes
import os

from . import build as _build

LBM_OK, LBM_ERR_ARG, LBM_ERR_CUDA, LBM_ERR_OOM, LBM_ERR_DIVERGED, LBM_ERR_STATE, LBM_ERR_TIMEOUT = (
    0, -1, -2, -3, -4, -5, -6)
LBM_FP64, LBM_FP32, LBM_FP16, LBM_BF16 = 0, 1, 2, 3
LBM_BC_PERIODIC, LBM_BC_BOUNCEBACK = 0, 1
LBM_BASE_REST, LBM_BASE_MOMENTUM = 0, 1

NOALLOC_MAX_ROWS = 8192  # LBM_VANSE_NOALLOC_MAX_ROWS

STATUS_NAMES = {0: "LBM_OK", -1: "LBM_ERR_ARG", -2: "LBM_ERR_CUDA", -3: "LBM_ERR_OOM",
                -4: "LBM_ERR_DIVERGED", -5: "LBM_ERR_STATE", -6: "LBM_ERR_TIMEOUT"}

# every entry point of include/lbm_vanse.h
EXPORTS = [
    "lbm_vanse_default_params", "lbm_vanse_create", "lbm_vanse_set_void_fraction",
    "lbm_vanse_set_void_fraction_f32", "lbm_vanse_reduce_async", "lbm_vanse_step_sums",
    "lbm_vanse_set_body_force", "lbm_vanse_set_drag", "lbm_vanse_set_moving_wall", "lbm_vanse_set_solid_cells",
    "lbm_vanse_set_row_wait_limit", "lbm_vanse_state_bytes", "lbm_vanse_save_state", "lbm_vanse_load_state",
    "lbm_vanse_init_fields",
    "lbm_vanse_step", "lbm_vanse_macros",
    "lbm_vanse_get_populations", "lbm_vanse_set_populations", "lbm_vanse_reduce",
    "lbm_vanse_velocity_error", "lbm_vanse_reduce_noalloc", "lbm_vanse_sync", "lbm_vanse_step_count",
    "lbm_vanse_bytes_per_cell", "lbm_vanse_launch_shape", "lbm_vanse_last_error",
    "lbm_vanse_destroy",
    "lbm_vanse_batch_default_params", "lbm_vanse_batch_create", "lbm_vanse_batch_init",
    "lbm_vanse_batch_step", "lbm_vanse_batch_step_each", "lbm_vanse_batch_autotune",
    "lbm_vanse_batch_velocity_error", "lbm_vanse_batch_get_populations", "lbm_vanse_batch_cells",
    "lbm_vanse_batch_step_count", "lbm_vanse_batch_last_error", "lbm_vanse_batch_destroy",
    "lbm_vanse_outlet_momentum_grad",
    # include/lbm_vanse3d.h
    "lbm_vanse3d_default_params", "lbm_vanse3d_create", "lbm_vanse3d_destroy", "lbm_vanse3d_set_void_fraction",
    "lbm_vanse3d_set_body_force", "lbm_vanse3d_init_fields", "lbm_vanse3d_step", "lbm_vanse3d_sync",
    "lbm_vanse3d_get_populations", "lbm_vanse3d_set_populations", "lbm_vanse3d_macros", "lbm_vanse3d_reduce",
    "lbm_vanse3d_step_count", "lbm_vanse3d_last_error",
]


class lbm_vanse_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("tau_nu", ctypes.c_double),
        ("s_e", ctypes.c_double), ("s_eps", ctypes.c_double), ("s_q", ctypes.c_double),
        ("s_c", ctypes.c_double),
        ("kappa", ctypes.c_double), ("rho0", ctypes.c_double),
        ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int),
        ("storage", ctypes.c_int), ("model_b", ctypes.c_int),
        ("storage_scale_log2", ctypes.c_int), ("strip_rows", ctypes.c_int),
        ("eager", ctypes.c_int), ("kernel", ctypes.c_int), ("eq_order", ctypes.c_int),
        ("dev_base", ctypes.c_int),
    ]


class lbm_vanse3d_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("tau_nu", ctypes.c_double),
        ("s_e", ctypes.c_double), ("s_eps", ctypes.c_double), ("s_q", ctypes.c_double),
        ("s_pi", ctypes.c_double), ("s_m", ctypes.c_double),
        ("kappa", ctypes.c_double), ("rho0", ctypes.c_double),
        ("bc_y", ctypes.c_int), ("storage", ctypes.c_int),
    ]


class lbm_vanse_batch_lattice(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int), ("tau_nu", ctypes.c_double), ("amplitude", ctypes.c_double),
        ("period", ctypes.c_double), ("u0", ctypes.c_double),
    ]


class lbm_vanse_batch_params(ctypes.Structure):
    _fields_ = [
        ("storage", ctypes.c_int),
        ("s_e", ctypes.c_double), ("s_eps", ctypes.c_double), ("s_q", ctypes.c_double),
        ("kappa", ctypes.c_double), ("rho0", ctypes.c_double), ("phi0", ctypes.c_double),
        ("strip_rows", ctypes.c_int), ("eager", ctypes.c_int),
    ]


class lbm_vanse_adjoint_params(ctypes.Structure):
    _fields_ = [
        ("nsteps", ctypes.c_int), ("avg_steps", ctypes.c_int), ("checkpoint_every", ctypes.c_int),
        ("x_out", ctypes.c_int), ("gx", ctypes.c_double), ("gy", ctypes.c_double),
        ("dense_segments", ctypes.c_int),
    ]


class lbm_vanse_adjoint_stats(ctypes.Structure):
    _fields_ = [("forward_ms", ctypes.c_double), ("backward_ms", ctypes.c_double),
                ("device_bytes", ctypes.c_longlong), ("host_bytes", ctypes.c_longlong)]


_lib = None


def load(path: str | None = None):
    """Load liblbm_vanse.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = os.environ.get("LBM_VANSE_LIB") or _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not found at {path}")
    L = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    i = ctypes.c_int
    d = ctypes.c_double
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    pp = ctypes.POINTER(lbm_vanse_params)
    sig = {
        "lbm_vanse_default_params": (None, [pp]),
        "lbm_vanse_create": (i, [pp, vp, ctypes.POINTER(vp)]),
        "lbm_vanse_set_void_fraction": (i, [vp, vp, vp, i]),
        "lbm_vanse_set_void_fraction_f32": (i, [vp, vp, vp, i]),
        "lbm_vanse_reduce_async": (i, [vp, vp, i]),
        "lbm_vanse_step_sums": (i, [vp, vp, i]),
        "lbm_vanse_set_body_force": (i, [vp, d, d, vp, i]),
        "lbm_vanse_set_drag": (i, [vp, d, d, d, d]),
        "lbm_vanse_set_moving_wall": (i, [vp, i, d, d]),
        "lbm_vanse_set_solid_cells": (i, [vp, i]),
        "lbm_vanse_set_row_wait_limit": (i, [vp, ctypes.c_longlong]),
        "lbm_vanse_state_bytes": (ctypes.c_longlong, [vp]),
        "lbm_vanse_save_state": (i, [vp, vp, i]),
        "lbm_vanse_load_state": (i, [vp, vp, i]),
        "lbm_vanse_init_fields": (i, [vp, vp, vp, vp, i]),
        "lbm_vanse_step": (i, [vp, i]),
        "lbm_vanse_macros": (i, [vp, vp, vp, vp, vp, i]),
        "lbm_vanse_get_populations": (i, [vp, vp, i]),
        "lbm_vanse_set_populations": (i, [vp, vp, i]),
        "lbm_vanse_reduce": (i, [vp, dp, dp, dp]),
        "lbm_vanse_velocity_error": (i, [vp, vp, vp, i, dp, dp]),
        "lbm_vanse_reduce_noalloc": (i, [vp, vp]),
        "lbm_vanse_sync": (i, [vp]),
        "lbm_vanse_step_count": (ctypes.c_longlong, [vp]),
        "lbm_vanse_bytes_per_cell": (d, [vp]),
        "lbm_vanse_launch_shape": (i, [vp, ip, ip, ip, ip, ip, ip]),
        "lbm_vanse_last_error": (ctypes.c_char_p, [vp]),
        "lbm_vanse_destroy": (None, [vp]),
        "lbm_vanse_batch_default_params": (None, [ctypes.POINTER(lbm_vanse_batch_params)]),
        "lbm_vanse_batch_create": (i, [ctypes.POINTER(lbm_vanse_batch_lattice), i,
                                       ctypes.POINTER(lbm_vanse_batch_params), vp, ctypes.POINTER(vp)]),
        "lbm_vanse_batch_init": (i, [vp]),
        "lbm_vanse_batch_step": (i, [vp, i]),
        "lbm_vanse_batch_step_each": (i, [vp, i]),
        "lbm_vanse_batch_autotune": (i, [vp, i, ip]),
        "lbm_vanse_batch_velocity_error": (i, [vp, i, dp, dp]),
        "lbm_vanse_batch_get_populations": (i, [vp, i, vp, i]),
        "lbm_vanse_batch_cells": (ctypes.c_longlong, [vp]),
        "lbm_vanse_batch_step_count": (ctypes.c_longlong, [vp]),
        "lbm_vanse_batch_last_error": (ctypes.c_char_p, [vp]),
        "lbm_vanse_batch_destroy": (None, [vp]),
        "lbm_vanse_outlet_momentum_grad": (i, [pp, ctypes.POINTER(lbm_vanse_adjoint_params), vp, i, vp, dp, vp,
                                               ctypes.POINTER(lbm_vanse_adjoint_stats)]),
        "lbm_vanse3d_default_params": (None, [ctypes.POINTER(lbm_vanse3d_params)]),
        "lbm_vanse3d_create": (i, [ctypes.POINTER(lbm_vanse3d_params), vp, ctypes.POINTER(vp)]),
        "lbm_vanse3d_destroy": (None, [vp]),
        "lbm_vanse3d_set_void_fraction": (i, [vp, vp, vp, i]),
        "lbm_vanse3d_set_body_force": (i, [vp, d, d, d, vp, i]),
        "lbm_vanse3d_init_fields": (i, [vp, vp, vp, vp, vp, i]),
        "lbm_vanse3d_step": (i, [vp, i]),
        "lbm_vanse3d_sync": (i, [vp]),
        "lbm_vanse3d_get_populations": (i, [vp, vp, i]),
        "lbm_vanse3d_set_populations": (i, [vp, vp, i]),
        "lbm_vanse3d_macros": (i, [vp, vp, vp, i]),
        "lbm_vanse3d_reduce": (i, [vp, dp, dp]),
        "lbm_vanse3d_step_count": (ctypes.c_longlong, [vp]),
        "lbm_vanse3d_last_error": (ctypes.c_char_p, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def default_params() -> lbm_vanse_params:
    p = lbm_vanse_params()
    load().lbm_vanse_default_params(ctypes.byref(p))
    return p


def batch_default_params() -> lbm_vanse_batch_params:
    p = lbm_vanse_batch_params()
    load().lbm_vanse_batch_default_params(ctypes.byref(p))
    return p


def default_params3d() -> lbm_vanse3d_params:
    p = lbm_vanse3d_params()
    load().lbm_vanse3d_default_params(ctypes.byref(p))
    return p
