"""ctypes declarations of libpsfsim's C ABI (include/psfsim.h, include/psfsim_fit.h,
include/psfsim_testing.h).

Argument marshalling only: every step of the method runs in the CUDA library.
Loading fails loudly when the library is missing; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpsfsim.so")

OK, ERR_ARG, ERR_RADII, ERR_WORKSPACE, ERR_CUDA, ERR_UNSUPPORTED, ERR_TIMEOUT = 0, -1, -2, -3, -4, -5, -6
FP32, SPLIT_BF16, BF16, FUSED, FP32_SYM, SPLIT_BF16_SYM = 0, 1, 2, 3, 4, 5
LINEAR, NEAREST = 0, 1
STATIC_SCRATCH_BYTES = 16 * 1024 * 1024

c_size_p = ctypes.POINTER(ctypes.c_size_t)
vp = ctypes.c_void_p
i32, i64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_double


class Info(ctypes.Structure):
    _fields_ = [("storage", ctypes.c_int32), ("interp", ctypes.c_int32), ("n", ctypes.c_int32),
                ("n_r", ctypes.c_int32), ("M", i64), ("K", i64), ("ld", i64), ("a_offset", i64),
                ("lo_offset", i64), ("scale_offset", i64), ("workspace_bytes", i64), ("K_stored", i64)]


class Job(ctypes.Structure):
    _fields_ = [("plan", vp), ("d_x", vp), ("d_y", vp), ("capacity", i32), ("d_count", vp)]


class Tuning(ctypes.Structure):
    _fields_ = [("chunk", i32), ("units_per_sm", i32), ("stages", i32)]


# name -> (restype, argtypes); every symbol include/*.h declares.
SIGNATURES = {
    "psfsim_status_string": (ctypes.c_char_p, [i32]),
    "psfsim_workspace_bytes": (i32, [i32, i32, i64, i32, c_size_p]),
    "psfsim_build": (i32, [vp, vp, i32, i32, f64, i32, f64, i32, i32, vp, ctypes.c_size_t, vp,
                           ctypes.POINTER(vp)]),
    "psfsim_build_points": (i32, [vp, vp, i32, i32, f64, vp, i64, i32, i32, vp, ctypes.c_size_t, vp,
                                  ctypes.POINTER(vp)]),
    "psfsim_info": (i32, [vp, ctypes.POINTER(Info)]),
    "psfsim_forward_scratch_bytes": (i32, [vp, i32, c_size_p]),
    "psfsim_adjoint_scratch_bytes": (i32, [vp, i32, c_size_p]),
    "psfsim_forward": (i32, [vp, vp, i32, vp, vp, ctypes.c_size_t, vp]),
    "psfsim_forward_sparse_scratch_bytes": (i32, [vp, i32, c_size_p]),
    "psfsim_forward_sparse": (i32, [vp, vp, i32, vp, vp, ctypes.c_size_t, vp]),
    "psfsim_adjoint": (i32, [vp, vp, i32, vp, vp, ctypes.c_size_t, vp]),
    "psfsim_forward_static": (i32, [vp, vp, i32, vp, vp]),
    "psfsim_forward_multi_scratch_bytes": (i32, [ctypes.POINTER(Job), i32, ctypes.POINTER(Tuning), c_size_p]),
    "psfsim_forward_multi": (i32, [ctypes.POINTER(Job), i32, ctypes.POINTER(Tuning), vp, ctypes.c_size_t, vp]),
    "psfsim_sync_status": (i32, [vp, vp]),
    "psfsim_reset_status": (i32, [vp, vp]),
    "psfsim_debug_forward_stall": (i32, [vp, vp, i32, vp, vp, ctypes.c_size_t, ctypes.c_uint64, i64, vp]),
    "psfsim_ring_chain_scratch_bytes": (i32, [i32, c_size_p]),
    "psfsim_loss_scratch_bytes": (i32, [i64, c_size_p]),
    "psfsim_ring_scene": (i32, [i32, f64, f64, vp, vp, vp]),
    "psfsim_ring_chain": (i32, [i32, f64, f64, vp, vp, vp, vp, ctypes.c_size_t, vp]),
    "psfsim_residual_loss": (i32, [vp, vp, i64, f64, vp, vp, vp, ctypes.c_size_t, vp]),
    "psfsim_ring_gradient_scratch_bytes": (i32, [vp, c_size_p]),
    "psfsim_ring_gradient": (i32, [vp, f64, vp, vp, f64, vp, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]),
    "psfsim_ring_forward_loss": (i32, [vp, f64, vp, vp, f64, vp, vp, vp, vp, ctypes.c_size_t, vp]),
    "psfsim_ring_adjoint_chain": (i32, [vp, f64, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]),
    "psfsim_free": (None, [vp]),
}

_lib = None


class PsfsimError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {status_string(code)} ({code})")


def load() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libpsfsim.so is not built ({LIB_PATH}); run __graft_entry__.build() "
                               "or python -m paper_2106_09122_gb300.build_lib")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def status_string(code: int) -> str:
    return load().psfsim_status_string(code).decode()


def check(code: int, what: str) -> None:
    if code != OK:
        raise PsfsimError(code, what)
