"""ctypes binding of libpointsht (include/pointsht.h): argument marshalling only.

The shared library is built in-tree by ``paper_2312_12285_gb300.build``.  If it
cannot be loaded, every call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpointsht.so")

OK, EINVAL, ERANGE, ENOMEM, ECUDA, EARCH, ETIMEOUT = range(7)
STATUS_NAMES = {OK: "OK", EINVAL: "EINVAL", ERANGE: "ERANGE", ENOMEM: "ENOMEM", ECUDA: "ECUDA", EARCH: "EARCH",
                ETIMEOUT: "ETIMEOUT"}
FP64, FP32, MIXED = 0, 1, 2
PRECISIONS = {"fp64": FP64, "fp32": FP32, "mixed": MIXED}

EXPORTS = (
    "pointsht_version", "pointsht_last_error", "pointsht_plan_create", "pointsht_plan_destroy",
    "pointsht_plan_lmax", "pointsht_plan_check", "pointsht_plan_set_timing_events", "pointsht_plan_set_tuning",
    "pointsht_plan_set_pole_threshold", "pointsht_plan_set_wait_probe", "pointsht_plan_set_skip_counters",
    "pointsht_plan_set_mixed_kernel",
    "pointsht_workspace_size",
    "pointsht_alm",
    "pointsht_shot_noise", "pointsht_combine", "pointsht_cl", "pointsht_cl_backward", "pointsht_bin",
    "pointsht_bin_backward", "pointsht_alm_backward", "pointsht_alm_noalloc",
    "pointsht_workspace_size_columns", "pointsht_alm_columns",
    "pointsht_workspace_size_interp", "pointsht_alm_interp",
    "pointsht_workspace_size_synthesis", "pointsht_synthesis",
    "pointsht_workspace_size_spin2", "pointsht_alm_spin2",
    "pointsht_workspace_size_coupling", "pointsht_coupling", "pointsht_coupling_binned",
    "pointsht_workspace_size_decouple", "pointsht_decouple", "pointsht_fkp_normalise",
)


class ShearCatalog(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("phi", ctypes.c_void_p), ("w", ctypes.c_void_p), ("g1", ctypes.c_void_p),
                ("g2", ctypes.c_void_p), ("n", ctypes.c_int64), ("field", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("coeff", ctypes.c_double)]


class Catalog(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("phi", ctypes.c_void_p), ("w", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("field", ctypes.c_int32), ("pad_", ctypes.c_int32), ("coeff", ctypes.c_double)]


class PointSHTError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lock = threading.Lock()
_lib = None


def load(build_if_missing: bool = True):
    """Load libpointsht.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            from . import build as _build
            if _build.needs_build():
                _build.build()
        lib = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, dp, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_size_t
        cp = ctypes.POINTER(Catalog)
        sig = {
            "pointsht_version": ([], ctypes.c_char_p),
            "pointsht_last_error": ([], ctypes.c_char_p),
            "pointsht_plan_create": ([i32, ctypes.POINTER(vp)], ctypes.c_int),
            "pointsht_plan_destroy": ([vp], None),
            "pointsht_plan_lmax": ([vp], i32),
            "pointsht_plan_check": ([vp], ctypes.c_int),
            "pointsht_plan_set_timing_events": ([vp, vp, vp], ctypes.c_int),
            "pointsht_plan_set_tuning": ([vp, i32, i32], ctypes.c_int),
            "pointsht_plan_set_pole_threshold": ([vp, ctypes.c_float], ctypes.c_int),
            "pointsht_plan_set_wait_probe": ([vp, i32], ctypes.c_int),
            "pointsht_plan_set_skip_counters": ([vp, vp], ctypes.c_int),
            "pointsht_plan_set_mixed_kernel": ([vp, i32], ctypes.c_int),
            "pointsht_workspace_size": ([vp, cp, i32, i32, ctypes.c_int], sz),
            "pointsht_alm": ([vp, cp, i32, i32, ctypes.c_int, dp, vp, sz, vp], ctypes.c_int),
            "pointsht_shot_noise": ([cp, i32, i32, ctypes.c_int, dp, vp, sz, vp], ctypes.c_int),
            "pointsht_combine": ([i32, dp, i32, dp, i32, dp, dp, dp, vp], ctypes.c_int),
            "pointsht_cl": ([i32, dp, i32, dp, dp, vp], ctypes.c_int),
            "pointsht_cl_backward": ([i32, dp, i32, dp, dp, dp, vp], ctypes.c_int),
            "pointsht_bin": ([i32, dp, i32, vp, i32, dp, vp], ctypes.c_int),
            "pointsht_bin_backward": ([i32, dp, i32, vp, i32, dp, vp], ctypes.c_int),
            "pointsht_alm_backward": ([vp, cp, i32, i32, ctypes.c_int, dp, dp, ctypes.POINTER(vp), vp, sz, vp],
                                      ctypes.c_int),
            "pointsht_alm_noalloc": ([vp, cp, i32, i32, ctypes.c_int, dp, vp], ctypes.c_int),
            "pointsht_workspace_size_columns": ([vp, i64, i32, ctypes.c_int], sz),
            "pointsht_alm_columns": ([vp, vp, vp, vp, i64, i32, ctypes.c_int, dp, vp, sz, vp], ctypes.c_int),
            "pointsht_workspace_size_interp": ([vp, cp, i32, i32, i32], sz),
            "pointsht_alm_interp": ([vp, cp, i32, i32, i32, dp, vp, sz, vp], ctypes.c_int),
            "pointsht_workspace_size_synthesis": ([vp, i64, ctypes.c_int], sz),
            "pointsht_synthesis": ([vp, vp, vp, i64, ctypes.c_int, dp, vp, vp, sz, vp], ctypes.c_int),
            "pointsht_workspace_size_spin2": ([vp, ctypes.POINTER(ShearCatalog), i32, i32], sz),
            "pointsht_alm_spin2": ([vp, ctypes.POINTER(ShearCatalog), i32, i32, dp, dp, vp, sz, vp], ctypes.c_int),
            "pointsht_workspace_size_coupling": ([i32], sz),
            "pointsht_coupling": ([i32, i32, dp, dp, vp, sz, vp], ctypes.c_int),
            "pointsht_coupling_binned": ([i32, dp, vp, i32, dp, dp, vp], ctypes.c_int),
            "pointsht_workspace_size_decouple": ([i32], sz),
            "pointsht_decouple": ([i32, i32, dp, dp, dp, i32, dp, dp, dp, vp, sz, vp], ctypes.c_int),
            "pointsht_fkp_normalise": ([i32, dp, i32, i32, dp, dp, i32, dp, dp, dp, vp], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def last_error() -> str:
    return load().pointsht_last_error().decode()


def check(status: int, what: str = ""):
    if status != OK:
        raise PointSHTError(status, f"{what}: {last_error()}" if what else last_error())


def catalog_array(entries):
    """entries: iterable of (x_ptr, phi_ptr, w_ptr, n, field, coeff) -> ctypes array."""
    entries = list(entries)
    arr = (Catalog * max(1, len(entries)))()
    for i, (x, p, w, n, f, c) in enumerate(entries):
        arr[i] = Catalog(x, p, w, int(n), int(f), 0, float(c))
    return arr, len(entries)
