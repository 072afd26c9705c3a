"""ctypes loader for libazint.so (the C ABI declared in include/azint.h).

The library is built in-tree by ``_build.build()``; there is no fallback: if it is missing
or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

AZ_OK = 0
ERRORS = {-1: "AZ_EINVAL", -2: "AZ_ESHAPE", -3: "AZ_ENOMEM", -4: "AZ_EOVERFLOW",
          -5: "AZ_ECUDA", -6: "AZ_EUNSUPPORTED", -7: "AZ_ETIMEOUT", -8: "AZ_ERANGE"}

UNIT_2TH_DEG, UNIT_Q_NM, UNIT_R_MM = 0, 1, 2
SPLIT_NONE, SPLIT_BBOX, SPLIT_FULL = 0, 1, 2
PREC_FP64, PREC_FP32_COMP = 0, 1
DTYPE_F32, DTYPE_U32, DTYPE_I32 = 0, 1, 2
WHERE_CORNERS, WHERE_CENTRES = 0, 1


class AzError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "AZ_E?"), code, message))
        self.code = code


class Info(ctypes.Structure):
    _fields_ = [("ny", ctypes.c_int32), ("nx", ctypes.c_int32), ("npt_rad", ctypes.c_int32),
                ("npt_azim", ctypes.c_int32), ("nrows", ctypes.c_int32), ("unit", ctypes.c_int32),
                ("split", ctypes.c_int32), ("n_unmasked", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("lo", ctypes.c_double), ("hi", ctypes.c_double), ("delta", ctypes.c_double),
                ("tile_h", ctypes.c_int32), ("tile_w", ctypes.c_int32),
                ("rows_per_warp", ctypes.c_int32), ("frames_per_pass", ctypes.c_int32),
                ("n_tiles", ctypes.c_int64), ("n_segments", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("copy_engine", ctypes.c_int32),
                ("n_items", ctypes.c_int32), ("layout", ctypes.c_int32),
                ("lut_width", ctypes.c_int64)]


class Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * 5), ("total_ms", ctypes.c_double * 5)]


PROFILE_KINDS = ("phase1_frames", "phase1_norm", "phase1_single", "phase2_finalize", "prep")

_lock = threading.Lock()
_lib = None

vp = ctypes.c_void_p
i32 = ctypes.c_int
f64 = ctypes.c_double
PP = ctypes.POINTER(ctypes.c_void_p)

SIGNATURES = {
    "az_geometry_create": ([f64] * 9 + [PP], i32),
    "az_geometry_destroy": ([vp], None),
    "az_geometry_rotation": ([vp, vp], i32),
    "az_geometry_positions": ([vp, i32, i32, i32, i32, vp, vp, vp], i32),
    "az_geometry_solid_angle": ([vp, i32, i32, vp, vp], i32),
    "az_geometry_polarization": ([vp, i32, i32, f64, vp, vp], i32),
    "az_csr_build": ([vp, i32, i32, i32, i32, i32, i32, vp, vp, PP], i32),
    "az_csr_build_from_positions": ([i32, i32, vp, vp, i32, i32, i32, vp, vp, PP], i32),
    "az_integrator_info": ([vp, ctypes.POINTER(Info)], i32),
    "az_csr_export": ([vp, vp, vp, vp], i32),
    "az_csr_import": ([i32, i32, i32, i32, i32, i32, vp, vp, vp, f64, f64, vp, PP], i32),
    "az_radial_axis": ([vp, vp], i32),
    "az_integrator_status": ([vp], i32),
    "az_integrator_destroy": ([vp], None),
    "az_integrate1d": ([vp, vp, i32, vp, vp, vp, vp, i32, vp, vp, vp, vp, vp], i32),
    "az_integrate2d": ([vp, vp, i32, vp, vp, vp, vp, i32, vp, vp, vp, vp, vp], i32),
    "az_integrate_noalloc": ([vp, vp, i32, vp, vp, vp, vp, i32, vp, vp, vp, vp, vp], i32),
    "az_integrate_batch": ([vp, vp, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp], i32),
    "az_integrate_batch_host": ([vp, vp, i32, i32, vp, vp, vp, vp, vp, vp, vp], i32),
    "az_set_corrections": ([vp, vp, vp, vp, vp, vp], i32),
    "az_integrate_batch_bound": ([vp, vp, i32, i32, vp, vp, vp, vp, vp], i32),
    "az_integrate_variance": ([vp, vp, i32, i32, vp, vp], i32),
    "az_integrate_batch_pixelnorm": ([vp, vp, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp], i32),
    "az_integrate_backward": ([vp, vp, vp, vp, vp, vp, i32, vp, vp, vp], i32),
    "az_multi_create": ([PP, i32, PP, i32, PP, PP, PP, PP, PP, PP, PP, PP, PP], i32),
    "az_multi_launch": ([vp, i32, vp], i32),
    "az_multi_destroy": ([vp], None),
    "az_autotune": ([vp, i32, vp, ctypes.POINTER(ctypes.c_double)], i32),
    "az_set_tuning": ([vp, i32, i32, i32, i32], i32),
    "az_lut_build": ([vp, i32, vp], i32),
    "az_lut_export": ([vp, vp, vp, vp, vp], i32),
    "az_integrate_lut": ([vp, vp, i32, vp, vp, vp, vp, i32, vp, vp, vp, vp, vp], i32),
    "az_set_layout": ([vp, i32], i32),
    "az_selftest_wait": ([i32, ctypes.c_int64, vp, vp], i32),
    "az_profile_enable": ([vp, i32], i32),
    "az_set_copy_engine": ([vp, i32], i32),
    "az_profile_read": ([vp, ctypes.POINTER(Profile)], i32),
    "az_last_error": ([], ctypes.c_char_p),
}


def library_path() -> str:
    return _build.LIB


def load(build: bool = True):
    """Load libazint.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("libazint.so is not built (%s); run __graft_entry__.build()" % path)
        lib = ctypes.CDLL(path)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def check(rc: int):
    if rc != AZ_OK:
        msg = load().az_last_error()
        raise AzError(rc, msg.decode() if msg else "")
    return rc
