"""ctypes declarations of libmuser.so (see include/muser.h).

Loading fails loudly: there is no fallback implementation of any call.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

MUSER_OK, MUSER_ERR_ARG, MUSER_ERR_CUDA, MUSER_ERR_TIMEOUT, MUSER_ERR_UNSUPPORTED, MUSER_ERR_WORKSPACE = range(6)
(ST_ALL_FLAGGED, ST_NONFINITE, ST_DROPPED, ST_GMM_DEGENERATE, ST_ITER_CAP, ST_BEAM_FIT, ST_TIMEOUT,
 ST_NO_DISK) = 1, 2, 4, 8, 16, 32, 64, 128
FORWARD, ADJOINT, REUSE_PLAN, GRAD_CHAIN, GRAD_ROWS_READY = 0, 1, 4, 8, 16
(CALL_GRID, CALL_DIRTY, CALL_GMM, CALL_CLEAN, CALL_RESTORE, CALL_IMAGE, CALL_DEGRID, CALL_CHI2, CALL_CENTER,
 CALL_STEER, CALL_GRAD) = range(1, 12)

_ERRNAMES = {1: "MUSER_ERR_ARG", 2: "MUSER_ERR_CUDA", 3: "MUSER_ERR_TIMEOUT", 4: "MUSER_ERR_UNSUPPORTED",
             5: "MUSER_ERR_WORKSPACE"}


class MuserError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("G", ctypes.c_int32), ("W", ctypes.c_int32), ("os", ctypes.c_int32),
                ("weight_mode", ctypes.c_int32), ("peak_mode", ctypes.c_int32), ("thr_mode", ctypes.c_int32),
                ("max_iter", ctypes.c_int32), ("gain", ctypes.c_float), ("gmm_bins", ctypes.c_int32),
                ("lat_rad", ctypes.c_double), ("batch_chunk", ctypes.c_int32), ("clean_kernel", ctypes.c_int32),
                ("w_planes", ctypes.c_int32), ("w_max", ctypes.c_float), ("w_support", ctypes.c_int32),
                ("clean_variant", ctypes.c_int32), ("steer_clip", ctypes.c_float), ("reserved", ctypes.c_int32 * 1)]


P = ctypes.c_void_p
I32, I64, F32, SZ = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_size_t
CFG = ctypes.POINTER(Config)

SIGNATURES = {
    "muser_version": (ctypes.c_char_p, []),
    "muser_last_error": (ctypes.c_char_p, []),
    "muser_launch_count": (ctypes.c_ulonglong, []),
    "muser_pixel_size": (I32, [P, I32, ctypes.c_double, I32, ctypes.c_double, P]),
    "muser_workspace_size": (SZ, [I32, I32, I64, CFG]),
    "muser_uvw": (I32, [P, I32, P, I32, P, P, I32, P, P, I32, P, P, P, CFG, P, P, P, P]),
    "muser_grid": (I32, [P, P, I32, I64, CFG, P, P, SZ, P, P]),
    "muser_dirty": (I32, [P, I32, CFG, P, P, P, SZ, P, P]),
    "muser_dirty_noalloc": (I32, [P, I32, CFG, P, P, P, P]),
    "muser_gmm": (I32, [P, I32, CFG, P, P, P, SZ, P, P]),
    "muser_clean": (I32, [P, P, I32, CFG, P, P, P, P, P, SZ, P, P]),
    "muser_restore": (I32, [P, P, P, P, P, I32, CFG, P, P, P, SZ, P, P]),
    "muser_image": (I32, [P, I32, P, I32, P, P, I32, P, P, I32, P, P, P, CFG, P, P, P, P, P, P, P, P, SZ, P, P]),
    "muser_image_events": (I32, [P, I32, P, I32, P, P, I32, P, P, I32, P, P, P, CFG, P, P, P, P, P, P, P, P, SZ, P,
                                 P, I32, P]),
    "muser_degrid": (I32, [I32, P, P, I64, P, CFG, P, SZ, P]),
    "muser_chi2": (I32, [P, P, P, I64, F32, P, P, P, SZ, P]),
    "muser_center": (I32, [P, P, P, P, I32, CFG, P, P, P, P, SZ, P, P]),
    "muser_steer": (I32, [P, P, I32, CFG, P, F32, P, P, P, SZ, P, P]),
    "muser_grad_step": (I32, [I32, P, P, I64, P, F32, F32, P, P, CFG, P, SZ, P]),
    "muser_normal_apply": (I32, [I32, P, P, P, I64, F32, CFG, P, SZ, P]),
    "muser_normalize": (I32, [P, I64, P, P, P]),
    "muser_lipschitz": (I32, [I32, P, P, I64, F32, I32, P, CFG, P, SZ, P]),
    "muser_axpy": (I32, [P, P, I64, F32, P, P]),
    "muser_selftest_wait": (I32, [ctypes.c_longlong, P, P]),
    "muser_autotune": (I32, [I32, P, P, I32, I64, CFG, P, P]),
    "muser_set_tuning": (I32, [I32, CFG, I32]),
}

_lib = None


def load(build_if_missing: bool = True):
    """The loaded library; builds it in-tree first when missing or stale."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        try:
            path = _build.build()
        except Exception as e:      # no compiler on this machine: use an existing build
            if not os.path.exists(path):
                raise ImportError(f"libmuser.so is missing and could not be built: {e}") from e
    if not os.path.exists(path):
        raise ImportError(f"libmuser.so not found at {path}; run `python -m paper_1712_06913_b300._build`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(rc: int):
    if rc != MUSER_OK:
        raise MuserError(rc, load().muser_last_error().decode())
