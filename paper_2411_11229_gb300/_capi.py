"""ctypes binding of libhweno.so with the names of include/hweno.h (argument marshalling only).

Every numerical step runs in the CUDA library; there is no host fallback.  Loading fails loudly
when the library is missing or cannot be built.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _make as _build

HWENO_ADVECTION, HWENO_BURGERS, HWENO_EULER = 0, 1, 2
HWENO_BC_PERIODIC, HWENO_BC_TRANSMISSIVE, HWENO_BC_REFLECTIVE, HWENO_BC_FIXED = 0, 1, 2, 3
HWENO_FLAG_V_WEIGHTED, HWENO_FLAG_CD2, HWENO_FLAG_R2, HWENO_FLAG_ALPHA_STEP, HWENO_FLAG_ALPHA_LOCAL = 1, 2, 4, 8, 16
HWENO_OK, HWENO_EINVAL, HWENO_ECUDA, HWENO_ENOMEM, HWENO_ENONPHYS, HWENO_ESTATE = 0, -1, -2, -3, -4, -5
HWENO_ETOOBIG = -6

# every entry point declared in include/hweno.h: name -> (restype, argtypes)
_D = ctypes.c_double
_P = ctypes.c_void_p
_I = ctypes.c_int
_H = ctypes.c_void_p
SIGNATURES = {
    "hweno_create": (_I, [_I, _I, ctypes.c_int64, ctypes.c_int64, _D, _D, _D, _I, ctypes.POINTER(_H)]),
    "hweno_create_ex": (_I, [_I, _I, ctypes.c_int64, ctypes.c_int64, _D, _D, _D, _P, ctypes.POINTER(_H)]),
    "hweno_set_params": (_I, [_H, _D, _D, _D, _D, _D, _D]),
    "hweno_run": (_I, [_H, _D, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "hweno_set_stream": (_I, [_H, _P]),
    "hweno_state_doubles": (ctypes.c_size_t, [_H]),
    "hweno_workspace_bytes": (ctypes.c_size_t, [_H]),
    "hweno_bind": (_I, [_H, _P, _P]),
    "hweno_rhs": (_I, [_H, _P, _P, _P]),
    "hweno_step": (_I, [_H, _D]),
    "hweno_steps": (_I, [_H, _D, _I]),
    "hweno_set_time": (_I, [_H, _D, _D]),
    "hweno_last_dt": (_I, [_H, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "hweno_max_wavespeed": (_I, [_H, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "hweno_sync": (_I, [_H]),
    "hweno_upload": (_I, [_H, _P]),
    "hweno_download": (_I, [_H, _P]),
    "hweno_set_profiling": (_I, [_H, _I]),
    "hweno_kernel_times": (_I, [_H, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_longlong)]),
    "hweno_selftest_rcp": (_I, [_P, _P, ctypes.c_int64, _P]),
    "hweno_selftest_fp64_peak": (_I, [_P, _I, _P, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "hweno_rhs_static": (_I, [_I, _I, ctypes.c_int64, ctypes.c_int64, _D, _D, _D, _I, _P, _P, _P, _P, _P]),
    "hweno_adjoint_workspace_bytes": (ctypes.c_size_t, [_H]),
    "hweno_step_record": (_I, [_H, _P]),
    "hweno_step_replay": (_I, [_H, _D, _P]),
    "hweno_adjoint_step": (_I, [_H, _P, _D, _P, _P, _P, _P]),
    "hweno_stage_vjp": (_I, [_H, _P, _P, _P, _P, _P, _P]),
    "hweno_adjoint_step_stages": (_I, [_H, _P, _P, _P, _D, _P, _P, _P, _P]),
    "hweno_step_replay_stages": (_I, [_H, _D, _P, _P, _P]),
    "hweno_step_stages": (_I, [_H, _D, _P, _P]),
    "hweno_pipeline_slot_bytes": (ctypes.c_size_t, [_H]),
    "hweno_pipeline": (_I, [_H, _I, ctypes.POINTER(_P), ctypes.POINTER(_P), _I, _I, _P]),
    "hweno_bounds_status": (ctypes.c_longlong, [ctypes.POINTER(ctypes.c_int)]),
    "hweno_bounds_selftest": (ctypes.c_longlong, []),
    "hweno_batch_create": (_I, [_I, _P, ctypes.POINTER(_H)]),
    "hweno_batch_set_stream": (_I, [_H, _P]),
    "hweno_batch_state_doubles": (ctypes.c_size_t, [_H]),
    "hweno_batch_state_offset": (ctypes.c_size_t, [_H, _I]),
    "hweno_batch_workspace_bytes": (ctypes.c_size_t, [_H]),
    "hweno_batch_bind": (_I, [_H, _P, _P]),
    "hweno_batch_set_time": (_I, [_H, _D]),
    "hweno_batch_step": (_I, [_H, _I]),
    "hweno_batch_step_plain": (_I, [_H, _I]),
    "hweno_batch_dts": (_I, [_H, ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "hweno_batch_tune": (_I, [_H, _P, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "hweno_batch_launch_count": (ctypes.c_longlong, [_H]),
    "hweno_batch_destroy": (None, [_H]),
    "hweno_destroy": (None, [_H]),
    "hweno_strerror": (ctypes.c_char_p, [_I]),
    "hweno_launch_count": (ctypes.c_longlong, [_H]),
}

class HwenoExt(ctypes.Structure):
    """hweno_ext of include/hweno.h"""
    _fields_ = [("flags", ctypes.c_int32), ("side", ctypes.c_int32 * 4), ("pad_", ctypes.c_int32),
                ("grav", ctypes.c_double), ("fixed", (ctypes.c_double * 4) * 4)]


class HwenoDesc(ctypes.Structure):
    """hweno_desc of include/hweno.h"""
    _fields_ = [("dim", ctypes.c_int), ("system", ctypes.c_int), ("bc", ctypes.c_int), ("pad_", ctypes.c_int),
                ("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("gamma", ctypes.c_double)]


_lock = threading.Lock()
_lib = None


def bounds_checked() -> bool:
    """True when HWENO_BOUNDS_CHECK=1 selects the bounds-checked library (libhweno_bounds.so)."""
    return os.environ.get("HWENO_BOUNDS_CHECK", "") == "1"


def load(build: bool = True):
    """Load libhweno.so (building it first if it is missing or stale), or the bounds-checked
    libhweno_bounds.so when the environment sets HWENO_BOUNDS_CHECK=1."""
    global _lib
    with _lock:
        if _lib is None:
            bc = bounds_checked()
            path = _build.build(bounds_check=bc) if build else _build.lib_path(bc)
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class HwenoError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = load().hweno_strerror(code).decode()
        super().__init__(f"{where}: {msg} ({code})")
        self.code = code


def check(code: int, where: str) -> None:
    if code != HWENO_OK:
        raise HwenoError(code, where)


def __getattr__(name):
    if name in SIGNATURES:
        return getattr(load(), name)
    raise AttributeError(name)
