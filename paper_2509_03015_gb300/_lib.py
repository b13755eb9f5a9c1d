"""ctypes declarations of the C ABI in include/bdss.h (argument marshalling
only).  Loading fails loudly if the CUDA library has not been built: there is
no CPU fallback."""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libbdss.so")

BDSS_OK = 0
STATUS_NAMES = {
    0: "BDSS_OK", 1: "BDSS_ERR_INVALID_ARG", 2: "BDSS_ERR_NOT_SPD", 3: "BDSS_ERR_NOT_FACTORED",
    4: "BDSS_ERR_ALLOC", 5: "BDSS_ERR_CUDA", 6: "BDSS_ERR_TIMEOUT", 7: "BDSS_ERR_NO_CONVERGENCE",
    8: "BDSS_ERR_UNSUPPORTED", 9: "BDSS_ERR_GUARD",
}
PRECISIONS = {"fp64": 0, "fp32_ir": 1, "tf32_ir": 2}
OPTIONS = {"timeout_ms": 0, "persistent": 1, "max_refine": 2, "target_berr_e18": 3, "debug_skip_arrive": 4,
           "debug_guards": 5, "debug_corrupt_guard": 6, "refine_krylov": 7, "max_krylov_iters": 8,
           "kernel_timing": 9, "residual_emu": 10, "shift": 11, "nstar": 12,
           "schur_emu": 13, "small_cluster": 14}
KERNEL_CLASSES = ("factor", "schur_tc", "solve", "correction", "residual", "krylov", "slice")


class bdss_info(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int64), ("block", ctypes.c_int64), ("iters", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("backward_err", ctypes.c_double)]


# name -> (restype, argtypes); mirrors include/bdss.h
_vp = ctypes.c_void_p
_i64, _i32 = ctypes.c_int64, ctypes.c_int32
_info_p = ctypes.POINTER(bdss_info)
SIGNATURES = {
    "bdss_create": (_i32, [ctypes.POINTER(_vp), _i64, _i32, _i32, _i32, _vp]),
    "bdss_set_option": (_i32, [_vp, _i32, _i64]),
    "bdss_factor": (_i32, [_vp, _vp, _vp, _info_p]),
    "bdss_solve": (_i32, [_vp, _vp, _vp, _i32, _info_p]),
    "bdss_factor_solve": (_i32, [_vp, _vp, _vp, _vp, _vp, _i32, _info_p]),
    "bdss_logdet": (_i32, [_vp, ctypes.POINTER(ctypes.c_double)]),
    "bdss_last_launch_stats": (_i32, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "bdss_last_trace": (_i32, [_vp, ctypes.POINTER(_i64), _i32, ctypes.POINTER(_i32)]),
    "bdss_last_refine_stats": (_i32, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "bdss_get_launch_config": (_i32, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i64)]),
    "bdss_debug_fail_alloc": (_i32, [_i32]),
    "bdss_destroy": (_i32, [_vp]),
    "bdss_status_string": (ctypes.c_char_p, [_i32]),
    "bdss_last_cuda_error": (ctypes.c_char_p, []),
    "bdss_last_kernel_times": (_i32, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i64), _i32]),
    "bdss_residual": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "bdss_factor_shift": (_i32, [_vp, ctypes.POINTER(ctypes.c_double)]),
    "bdss_chunk_reduce": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _i32, _vp, _vp, _info_p]),
    "bdss_chunk_backsolve": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _i32, _vp]),
    "bdss_tc_selftest": (_i32, [ctypes.POINTER(ctypes.c_double)]),
    "bdss_adjoint_grads": (_i32, [_vp, _vp, _vp, _i32, _vp, _vp]),
    "bdss_batch_create": (_i32, [ctypes.POINTER(_vp), _i32, ctypes.POINTER(_i64), ctypes.POINTER(_i32), _i32, _vp]),
    "bdss_batch_set_inputs": (_i32, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                     ctypes.POINTER(_vp)]),
    "bdss_batch_launch": (_i32, [_vp, _i32]),
    "bdss_batch_wait": (_i32, [_vp, _info_p, ctypes.POINTER(ctypes.c_double)]),
    "bdss_batch_autotune": (_i32, [_vp, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "bdss_batch_destroy": (_i32, [_vp]),
    "bdss_factor_solve_batched": (_i32, [_i32, ctypes.POINTER(_i64), ctypes.POINTER(_i32), _i32,
                                         ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                         ctypes.POINTER(_vp), _vp, _info_p]),
    "bdss_factor_solve_noalloc": (_i32, [_i64, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _info_p]),
    "bdss_kalman_assemble": (_i32, [_i64, _i32, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
}

_lib = None


def load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is not built; run __graft_entry__.build() "
                               "(there is no CPU fallback)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class BDSSError(RuntimeError):
    def __init__(self, status, where, info=None):
        msg = load().bdss_status_string(status).decode()
        extra = ""
        if info is not None and status == 2:
            extra = f" (level {info.level}, block {info.block})"
        if status == 5:
            extra = f" ({load().bdss_last_cuda_error().decode()})"
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}{extra}")
        self.status = status
        self.info = info


def check(status, where, info=None):
    if status != BDSS_OK:
        raise BDSSError(status, where, info)
