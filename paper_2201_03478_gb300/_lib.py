"""ctypes loader for libsidelobe.so (the C ABI declared in include/sidelobe.h).

The library is built in-tree by ``paper_2201_03478_gb300._build.build()``.  There
is no fallback: if the shared library is missing or fails to load, every entry
point raises.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

SL_OK, SL_ERR_ARG, SL_ERR_UNSUPPORTED, SL_ERR_NOMEM, SL_ERR_CUDA, SL_ERR_TIMEOUT = 0, -1, -2, -3, -4, -5
SL_FP64, SL_FP32, SL_TF32X3, SL_DF64 = 0, 1, 2, 4

STATUS_NAMES = {0: "SL_OK", -1: "SL_ERR_ARG", -2: "SL_ERR_UNSUPPORTED", -3: "SL_ERR_NOMEM",
                -4: "SL_ERR_CUDA", -5: "SL_ERR_TIMEOUT"}

# Symbols include/sidelobe.h declares (checked by the host tests).
EXPORTS = ["sidelobe_plan_create", "synth_spin_maps", "interp_tod", "convolve_tod", "convolve_tod_host", "adjoint_tod",
           "adjoint_interp",
           "adjoint_synth", "interp_tod_noalloc", "plan_destroy", "sl_plan_get_sizes", "sl_plan_set_stream", "sl_plan_sync",
           "sl_plan_enable_timing", "sl_plan_kernel_stats", "sl_plan_reserve", "sl_plan_set_tile_cols", "sl_plan_set_fft_tile", "sl_plan_set_contraction_pairs",
           "sl_batch_create", "sl_batch_run", "sl_batch_sync", "sl_batch_get_info", "sl_batch_destroy", "synth_spin_maps_multi",
           "sl_plan_selftest_timeout", "sl_orbital_moments", "orbital_dipole_tod", "synth_psi_cube", "interp_tod_psi",
           "sl_debug_check_status", "sl_measure_alu_peak", "sl_quad_factor", "sl_last_error"]
SL_BATCH_AUTOTUNE = 1
SL_BATCH_PERSISTENT = 2


class PlanDesc(ctypes.Structure):
    _fields_ = [("lmax", ctypes.c_int), ("kmax", ctypes.c_int), ("ncomp", ctypes.c_int),
                ("nrings", ctypes.c_int), ("ring_theta", ctypes.c_void_p), ("nphi", ctypes.c_int),
                ("interp_order", ctypes.c_int), ("precision", ctypes.c_int), ("device", ctypes.c_int),
                ("stream", ctypes.c_void_p)]


class PlanSizes(ctypes.Structure):
    _fields_ = [("nalm", ctypes.c_int64), ("sky_doubles", ctypes.c_int64), ("beam_doubles", ctypes.c_int64),
                ("maps_bytes", ctypes.c_int64), ("scratch_bytes", ctypes.c_int64), ("lsteps", ctypes.c_int64),
                ("tile_cols", ctypes.c_int64), ("fft_rings", ctypes.c_int64), ("fft_korders", ctypes.c_int64),
                ("contraction_pairs", ctypes.c_int64)]


class BatchItem(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("sky", ctypes.c_void_p), ("beam", ctypes.c_void_p),
                ("maps", ctypes.c_void_p), ("theta", ctypes.c_void_p), ("phi", ctypes.c_void_p),
                ("psi", ctypes.c_void_p), ("n", ctypes.c_int64), ("tod", ctypes.c_void_p)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("nitems", ctypes.c_int), ("nstreams", ctypes.c_int), ("tuned_ms", ctypes.c_double),
                ("serial_ms", ctypes.c_double), ("kernel_nodes", ctypes.c_int), ("graph_nodes", ctypes.c_int),
                ("persistent", ctypes.c_int)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class SidelobeError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_lib = None
_checked = False


def use_checked_build() -> None:
    """Select the bounds-checked library variant (libsidelobe_checked.so, built on
    demand) for this process; must come before the first call into the library."""
    global _checked
    if _lib is not None:
        raise RuntimeError("the library is already loaded")
    _checked = True


def load(build: bool = True) -> ctypes.CDLL:
    """Load (building first if stale) libsidelobe.so and declare the signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if _checked:
        path = _build.build(checked=True) if build else _build.LIB_CHECKED
    else:
        path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise OSError("libsidelobe.so not found at %s (run paper_2201_03478_gb300._build.build())" % path)
    lib = ctypes.CDLL(path)
    P, I, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    sig = {
        "sidelobe_plan_create": (I, [ctypes.POINTER(P), ctypes.POINTER(PlanDesc)]),
        "synth_spin_maps": (I, [P, P, P, P]),
        "synth_spin_maps_multi": (I, [P, I, P, P, P]),
        "interp_tod": (I, [P, P, P, P, P, I64, P]),
        "convolve_tod": (I, [P, P, P, P, P, P, P, I64, P]),
        "convolve_tod_host": (I, [P, P, P, P, P, P, I64, I, P]),
        "adjoint_tod": (I, [P, P, P, P, P, I64, P, P, P, P, I]),
        "adjoint_interp": (I, [P, P, P, P, P, I64, P]),
        "adjoint_synth": (I, [P, P, P, P, P, P, I]),
        "interp_tod_noalloc": (I, [P, P, P, P, P, I64, P]),
        "plan_destroy": (None, [P]),
        "sl_plan_get_sizes": (I, [P, ctypes.POINTER(PlanSizes)]),
        "sl_plan_set_stream": (I, [P, P]),
        "sl_plan_sync": (I, [P]),
        "sl_plan_selftest_timeout": (I, [P]),
        "sl_plan_enable_timing": (I, [P, I]),
        "sl_plan_kernel_stats": (I, [P, ctypes.POINTER(KernelStat), I, ctypes.POINTER(I), I]),
        "sl_plan_reserve": (I, [P, I64]),
        "sl_plan_set_tile_cols": (I, [P, I]),
        "sl_plan_set_fft_tile": (I, [P, I, I]),
        "sl_plan_set_contraction_pairs": (I, [P, I]),
        "sl_batch_create": (I, [ctypes.POINTER(P), ctypes.POINTER(BatchItem), I, P, I]),
        "sl_batch_run": (I, [P]),
        "sl_batch_sync": (I, [P]),
        "sl_batch_get_info": (I, [P, ctypes.POINTER(BatchInfo)]),
        "sl_batch_destroy": (None, [P]),
        "sl_orbital_moments": (I, [P, P, P]),
        "synth_psi_cube": (I, [P, P, I, P]),
        "interp_tod_psi": (I, [P, P, I, P, P, P, I64, P]),
        "orbital_dipole_tod": (I, [P, P, ctypes.c_double, ctypes.c_double, P, P, P, I64, P, P, I64, I, P, I]),
        "sl_debug_check_status": (ctypes.c_uint, []),
        "sl_measure_alu_peak": (I, [I, I, ctypes.POINTER(ctypes.c_double)]),
        "sl_quad_factor": (I, [ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
        "sl_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def check(status: int) -> None:
    if status != SL_OK:
        msg = load().sl_last_error()
        raise SidelobeError(status, msg.decode() if msg else "")
