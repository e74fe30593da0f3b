"""ctypes declarations of ``include/sbg.h`` (argument marshalling only).

Loading fails loudly when ``libsbg.so`` is missing and cannot be built: there
is no CPU fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
# SBG_LIB_VARIANT=debug selects the debug build (libsbg_debug.so, compiled with
# SBG_DEBUG: index checks in the step kernels); the default is the release build
LIB_NAME = "libsbg_debug.so" if os.environ.get("SBG_LIB_VARIANT") == "debug" else "libsbg.so"
LIB_PATH = os.path.join(PKG, LIB_NAME)

SBG_OK = 0
SBG_ERR_INVALID_ARG = 1
SBG_ERR_OOM = 2
SBG_ERR_CUDA = 3
SBG_ERR_UNSTABLE_DT = 4
SBG_ERR_NONFINITE = 5
SBG_ERR_TIMEOUT = 6
SBG_ERR_NOT_CONVERGED = 7
SBG_ERR_BOUNDS = 8

SBG_F32, SBG_F64, SBG_F32X2, SBG_F32R = 0, 1, 2, 3
SBG_FACE_NOFLUX, SBG_FACE_DIRICHLET = 0, 1
SBG_KERNEL_AUTO, SBG_KERNEL_PLAIN, SBG_KERNEL_PIPELINED, SBG_KERNEL_PIPELINED_PREFETCH, SBG_KERNEL_PIPELINED_ASYNC = 0, 1, 2, 3, 4
SBG_KERNEL_STREAM = 5
SBG_KERNEL_WAVE, SBG_KERNEL_WAVE4 = 6, 7
SBG_ORDER_TILED, SBG_ORDER_PLANES = 0, 1

RED_MASS, RED_JIN, RED_JOUT, RED_RESIDUAL, RED_MIN, RED_MAX, RED_NONFINITE, RED_NACTIVE = range(8)
NRED = 8

c_void_p = ctypes.c_void_p
c_int32 = ctypes.c_int32
c_int64 = ctypes.c_int64
c_double = ctypes.c_double
c_float = ctypes.c_float


class BuildOpts(ctypes.Structure):
    _fields_ = [("block", c_int32), ("phi_on_device", c_int32), ("eps_mask", c_float),
                ("band_eps", c_float), ("order", c_int32)]


class RedistOpts(ctypes.Structure):
    _fields_ = [("cfl", c_double), ("max_iter", c_int64), ("tol", c_double), ("band", c_double),
                ("check_every", c_int32)]


class Params(ctypes.Structure):
    _fields_ = [("dx", c_double * 3), ("dt", c_double), ("nspecies", c_int32),
                ("face_type", c_int32 * 6), ("D", c_double * 2), ("decay", c_double * 2),
                ("k_surf", c_double), ("face_value", c_double * 6), ("allow_unstable", c_int32)]


class GridInfo(ctypes.Structure):
    _fields_ = [("dims", c_int64 * 3), ("block", c_int32), ("n_geoms", c_int32),
                ("n_blocks", c_int64), ("n_active", c_int64), ("n_band_blocks", c_int64),
                ("porosity", c_double), ("device_bytes", c_int64)]


# (name, restype, argtypes) for every entry point declared in include/sbg.h
SIGNATURES = [
    ("sbg_build", c_int32, [c_void_p, c_void_p, ctypes.POINTER(BuildOpts), c_void_p, ctypes.POINTER(c_void_p)]),
    ("sbg_build_batch", c_int32, [c_int32, c_void_p, c_void_p, ctypes.POINTER(BuildOpts), c_void_p,
                                  ctypes.POINTER(c_void_p)]),
    ("sbg_grid_info", c_int32, [c_void_p, ctypes.POINTER(GridInfo)]),
    ("sbg_grid_geometry_info", c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    ("sbg_grid_tables", c_int32, [c_void_p, c_void_p, c_void_p]),
    ("sbg_grid_destroy", None, [c_void_p]),
    ("sbg_grid_set_diffusivity", c_int32, [c_void_p, c_int32, c_void_p, c_int32, c_int32, c_void_p]),
    ("sbg_grid_set_diffusivity_sigmoid", c_int32, [c_void_p, c_int32, c_void_p, c_int32, c_double, c_double,
                                                   c_double, c_double, c_void_p]),
    ("sbg_grid_clear_diffusivity", c_int32, [c_void_p]),
    ("sbg_state_set_source", c_int32, [c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_int32, c_int32, c_void_p]),
    ("sbg_state_clear_source", c_int32, [c_void_p]),
    ("sbg_step_source", c_int32, [c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p]),
    ("sbg_redistance", c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_void_p,
                                 c_void_p, c_void_p]),
    ("sbg_reduce_async", c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    ("sbg_check_async", c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    ("sbg_reduce_box", c_int32, [c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("sbg_frap_curve", c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_int64,
                                 c_int32, c_void_p, c_void_p, c_void_p]),
    ("sbg_frap_fit", c_int32, [c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_int64, c_double, c_double,
                               c_void_p, c_void_p]),
    ("sbg_frap_recovery", c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_int64,
                                    c_int32, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("sbg_frap_effective_D", c_int32, [c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_int64, c_double, c_double,
                                       c_double, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("sbg_state_create", c_int32, [c_void_p, c_int32, c_int32, ctypes.POINTER(c_void_p)]),
    ("sbg_state_set", c_int32, [c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_int32, c_int32, c_void_p]),
    ("sbg_state_get", c_int32, [c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_int32, c_int32, c_void_p]),
    ("sbg_state_copy", c_int32, [c_void_p, c_void_p, c_void_p]),
    ("sbg_state_set_kernel", c_int32, [c_void_p, c_int32, c_int32]),
    ("sbg_state_destroy", None, [c_void_p]),
    ("sbg_step", c_int32, [c_void_p, c_void_p, ctypes.POINTER(Params), c_int64, c_void_p]),
    ("sbg_stability_limit", c_double, [ctypes.POINTER(Params), c_void_p, c_double]),
    ("sbg_reduce", c_int32, [c_void_p, c_void_p, ctypes.POINTER(Params), c_int32, c_void_p, c_void_p]),
    ("sbg_reduce_noalloc", c_int32, [c_void_p, c_void_p, ctypes.POINTER(Params), c_int32, c_int32, c_void_p,
                                     c_void_p]),
    ("sbg_effective_D", c_int32, [c_void_p, c_void_p, ctypes.POINTER(Params), c_int32, c_void_p, c_void_p,
                                  c_void_p, c_void_p]),
    ("sbg_run_to_steady", c_int32, [c_void_p, c_void_p, ctypes.POINTER(Params), c_double, c_int64, c_int64,
                                    c_void_p, c_void_p, c_void_p]),
    ("sbg_batch_run_to_steady", c_int32, [c_void_p, c_void_p, ctypes.POINTER(Params), c_double, c_int64, c_int64,
                                          c_void_p, c_void_p, c_void_p]),
    ("sbg_forward_record", c_int32, [c_void_p, c_void_p, ctypes.POINTER(Params), c_int64, c_int64, c_void_p,
                                     ctypes.POINTER(c_void_p)]),
    ("sbg_adjoint", c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("sbg_tape_info", c_int32, [c_void_p, c_void_p, c_void_p]),
    ("sbg_tape_destroy", None, [c_void_p]),
    ("sbg_last_error", ctypes.c_char_p, []),
    ("sbg_status_string", ctypes.c_char_p, [c_int32]),
    ("sbg_abi_version", c_int32, []),
    ("sbg_slab_partition", c_int32, [c_void_p, c_void_p, c_int32, c_float, c_int32, c_void_p]),
    ("sbg_state_get_xplane", c_int32, [c_void_p, c_void_p, c_int32, c_int32, c_int64, c_void_p, c_int32, c_int32,
                                       c_void_p]),
    ("sbg_state_set_xplane", c_int32, [c_void_p, c_void_p, c_int32, c_int32, c_int64, c_void_p, c_int32, c_int32,
                                       c_void_p]),
    ("sbg_debug_stall_stage", c_int32, [c_void_p, c_int64, c_int64]),
    ("sbg_debug_fail_alloc", c_int32, [c_int64]),
    ("sbg_debug_live_allocations", c_int32, [c_void_p, c_void_p]),
    ("sbg_debug_set_face", c_int32, [c_void_p, c_int64, c_int32, c_int32, c_void_p]),
    ("sbg_debug_wave_plan", c_int32, [c_void_p, c_int32, c_int32, c_int32, c_int32, c_int32, c_void_p, c_int64,
                                      c_void_p]),
]

_lib = None


def load(build_if_missing: bool = True):
    """Loads libsbg.so (building it with nvcc first when it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        from . import build as _build
        debug = LIB_NAME == "libsbg_debug.so"
        if _build.needs_build(debug):
            _build.build(debug=debug)
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("%s is missing: build it with `python -m paper_2304_11165_b300.build`" % LIB_NAME)
    lib = ctypes.CDLL(LIB_PATH)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class SbgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (status %d): %s" % (_status_name(status), status, msg))
        self.status = status


def _status_name(s):
    names = {0: "SBG_OK", 1: "SBG_ERR_INVALID_ARG", 2: "SBG_ERR_OOM", 3: "SBG_ERR_CUDA",
             4: "SBG_ERR_UNSTABLE_DT", 5: "SBG_ERR_NONFINITE", 6: "SBG_ERR_TIMEOUT",
             7: "SBG_ERR_NOT_CONVERGED", 8: "SBG_ERR_BOUNDS"}
    return names.get(s, "SBG_STATUS_%d" % s)


def check(status):
    if status != SBG_OK:
        raise SbgError(status, load().sbg_last_error().decode(errors="replace"))
    return status
