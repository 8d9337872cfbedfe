"""ctypes declarations of the libarkcos C ABI (include/arkcos.h, include/arkcos_peaks.h).
Argument marshalling only."""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, ECUDA, EWORKSPACE, ETIMEOUT, EUNSUPPORTED = range(7)
FLAG_BASIC = 1
FLAG_NO_SHIFT_FIX = 2
FLAG_NO_POLE_FIX = 4
FLAG_3XTF32 = 8

_STATUS = {OK: "OK", EINVAL: "EINVAL", ENOMEM: "ENOMEM", ECUDA: "ECUDA",
           EWORKSPACE: "EWORKSPACE", ETIMEOUT: "ETIMEOUT", EUNSUPPORTED: "EUNSUPPORTED"}

# every symbol include/*.h declares
SYMBOLS = [
    "arkcos_create_grid_healpix", "arkcos_create_grid_ecp", "arkcos_destroy_grid",
    "arkcos_grid_info", "arkcos_set_kernel", "arkcos_kernel_update_knots",
    "arkcos_destroy_kernel", "arkcos_workspace_size", "arkcos_convolve",
    "arkcos_convolve_backward", "arkcos_convolve_static", "arkcos_batch_workspace_size",
    "arkcos_convolve_batch", "arkcos_autotune", "arkcos_set_launch_shape", "arkcos_host_workspace_size",
    "arkcos_convolve_host",
    "arkcos_ring_analysis",
    "arkcos_ring_synthesis",
    "arkcos_kernel_info", "arkcos_stage_timing", "arkcos_stage_report",
    "arkcos_sync_status", "arkcos_last_error", "arkcos_version",
    "arkcos_measure_peak", "arkcos_multi_workspace_size", "arkcos_convolve_multi",
]


class Job(ctypes.Structure):
    """arkcos_job (include/arkcos.h)."""
    _fields_ = [("grid", ctypes.c_void_p), ("kernels", ctypes.c_void_p), ("nkernels", ctypes.c_int64),
                ("map_in", ctypes.c_void_p), ("map_out", ctypes.c_void_p), ("nmaps", ctypes.c_int64),
                ("flags", ctypes.c_uint32)]


class ArkcosError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libarkcos.so (building it first if it is missing or stale and nvcc exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libarkcos.so is not built; run python -m paper_1104_0672_gb300.build")
        L = ctypes.CDLL(_build.LIB)
        I64, U32, VP, D = ctypes.c_int64, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_double
        PVP = ctypes.POINTER(ctypes.c_void_p)
        P64 = ctypes.POINTER(ctypes.c_int64)
        S = ctypes.c_int
        sig = {
            "arkcos_create_grid_healpix": ([I64, PVP], S),
            "arkcos_create_grid_ecp": ([I64, I64, PVP], S),
            "arkcos_destroy_grid": ([VP], S),
            "arkcos_grid_info": ([VP, P64, P64, P64], S),
            "arkcos_set_kernel": ([VP, VP, I64, D, U32, PVP], S),
            "arkcos_kernel_update_knots": ([VP, VP, ctypes.c_int, VP], S),
            "arkcos_destroy_kernel": ([VP], S),
            "arkcos_workspace_size": ([VP, VP, I64, I64, U32, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_size_t)], S),
            "arkcos_convolve": ([VP, VP, I64, VP, VP, I64, VP, ctypes.c_size_t, VP, U32], S),
            "arkcos_convolve_backward": ([VP, VP, I64, VP, VP, VP, VP, I64, VP, ctypes.c_size_t,
                                          VP, U32], S),
            "arkcos_convolve_static": ([VP, VP, I64, VP, VP, I64, VP, U32], S),
            "arkcos_batch_workspace_size": ([VP, I64, ctypes.POINTER(ctypes.c_size_t)], S),
            "arkcos_convolve_batch": ([VP, I64, VP, ctypes.c_size_t, VP], S),
            "arkcos_autotune": ([VP, VP, I64, VP, VP, I64, VP, ctypes.c_size_t, VP, U32, P64], S),
            "arkcos_set_launch_shape": ([VP, VP, I64, I64, U32, P64], S),
            "arkcos_host_workspace_size": ([VP, VP, I64, I64, I64, U32, ctypes.POINTER(ctypes.c_size_t)], S),
            "arkcos_convolve_host": ([VP, VP, I64, VP, VP, I64, I64, VP, ctypes.c_size_t, VP, U32], S),
            "arkcos_ring_analysis": ([VP, VP, VP, I64, VP], S),
            "arkcos_ring_synthesis": ([VP, VP, VP, I64, U32, VP], S),
            "arkcos_kernel_info": ([VP, P64, P64, P64], S),
            "arkcos_stage_timing": ([ctypes.c_int], S),
            "arkcos_stage_report": ([I64, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(D),
                                     P64, P64], S),
            "arkcos_sync_status": ([VP], S),
            "arkcos_last_error": ([], ctypes.c_char_p),
            "arkcos_version": ([], ctypes.c_char_p),
            "arkcos_measure_peak": ([ctypes.c_int, ctypes.POINTER(D), ctypes.POINTER(D), VP], S),
            "arkcos_multi_workspace_size": ([VP, VP, I64, I64, ctypes.c_int, U32, ctypes.POINTER(ctypes.c_size_t)], S),
            "arkcos_convolve_multi": ([VP, VP, I64, VP, VP, VP, I64, VP, ctypes.c_size_t, VP, U32], S),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
        return L


def check(status: int):
    if status != OK:
        msg = load().arkcos_last_error().decode(errors="replace")
        raise ArkcosError(status, msg)
