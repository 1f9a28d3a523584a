"""ctypes declarations of libpdas (include/pdas.h, include/pdas_components.h,
include/pdas_batch.h, include/pdas_woodbury.h).

Loading fails loudly: there is no CPU fallback.  Build the library with
``python -m paper_1502_03543_gb300.build`` first.
"""
from __future__ import annotations

import ctypes
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libpdas.so")

# pdas_status
OK, OPTIMAL, OPTIMAL_EXACT, MAX_ITER, STALLED, ZERO_DIRECTION = 0, 1, 2, 3, 4, 5
ERR_ARG, ERR_NOT_INTERIOR, ERR_NOT_SPD, ERR_NONFINITE, ERR_TIMEOUT, ERR_CUDA, ERR_UNSUPPORTED = (-1, -2, -3, -4, -5,
                                                                                              -6, -7)
# pdas_form
FP64, TF32_IR, BF16_IR, FP32_IR = 0, 1, 2, 3
# pdas_dtype
A_F64, A_F32, A_BF16 = 0, 1, 2


class Options(ctypes.Structure):
    _fields_ = [
        ("form", ctypes.c_int),
        ("a_dtype", ctypes.c_int),
        ("max_iter", ctypes.c_int),
        ("refine_tol", ctypes.c_double),
        ("refine_max", ctypes.c_int),
        ("dspread_refactor", ctypes.c_double),
        ("stream", ctypes.c_void_p),
        ("splits", ctypes.c_int),
        ("stall_theta", ctypes.c_double),
        ("stall_count", ctypes.c_int),
        ("refine_be", ctypes.c_double),
        ("drop_tol", ctypes.c_double),
        ("drop_keep", ctypes.c_double),
        ("exact_passes", ctypes.c_int),
        ("infeasible", ctypes.c_int),
        ("fp64_tier_tc", ctypes.c_int),
        ("df_factor_floor", ctypes.c_double),
    ]


class IterInfo(ctypes.Structure):
    _fields_ = [
        ("psi", ctypes.c_double),
        ("theta", ctypes.c_double),
        ("rel_gap", ctypes.c_double),
        ("cx", ctypes.c_double),
        ("by", ctypes.c_double),
        ("xs", ctypes.c_double),
        ("dmax", ctypes.c_double),
        ("dmin", ctypes.c_double),
        ("refine_resid", ctypes.c_double),
        ("refine_sweeps", ctypes.c_int),
        ("used_fp64", ctypes.c_int),
        ("fp64_reason", ctypes.c_int),
        ("factor_columns", ctypes.c_int64),
        ("normal_form", ctypes.c_int),
        ("pres", ctypes.c_double),
        ("dres", ctypes.c_double),
        ("factor_form", ctypes.c_int),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


STAGES = ("rhs", "normal", "factor", "solve", "direction", "step", "fold")


class BatchOptions(ctypes.Structure):
    _fields_ = [
        ("alpha", ctypes.c_double),
        ("tol", ctypes.c_double),
        ("max_iter", ctypes.c_int),
        ("refine_tol", ctypes.c_double),
        ("refine_max", ctypes.c_int),
        ("autotune", ctypes.c_int),
        ("stream", ctypes.c_void_p),
    ]


class Profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 7), ("calls", ctypes.c_int64 * 7), ("launches", ctypes.c_int64)]

    def as_dict(self):
        return dict(ms={k: self.ms[i] for i, k in enumerate(STAGES)},
                    calls={k: int(self.calls[i]) for i, k in enumerate(STAGES)}, launches=int(self.launches))


_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_D = ctypes.c_double
_H = ctypes.c_void_p

SIGNATURES = {
    "pdas_default_options": ([ctypes.POINTER(Options)], None),
    "pdas_create": ([_I64, _I64, ctypes.POINTER(Options), ctypes.POINTER(_H)], _I),
    "pdas_step": ([_H, _P, _P, _P, _P, _P, _P, _D, ctypes.POINTER(IterInfo)], _I),
    "pdas_solve": ([_H, _P, _P, _P, _P, _P, _P, _D, _D, ctypes.POINTER(_I), ctypes.POINTER(_D)], _I),
    "pdas_backward": ([_H, _P, _P, _P, _P, _P, _P, _P, _P], _I),
    "pdas_destroy": ([_H], None),
    "pdas_status_str": ([_I], ctypes.c_char_p),
    "pdas_last_error_index": ([_H], _I64),
    "pdas_last_error_message": ([_H], ctypes.c_char_p),
    "pdas_set_wait_limit": ([_H, _I64], _I),
    "pdas_form_normal": ([_H, _P, _P, _P], _I),
    "pdas_copy_matrix": ([_H, _P, ctypes.POINTER(_I)], _I),
    "pdas_load_matrix": ([_H, _P, _I], _I),
    "pdas_factor": ([_H], _I),
    "pdas_factor_solve": ([_H, _P, _P], _I),
    "pdas_direction": ([_H, _P, _P, _P, _P, _P, _P, ctypes.POINTER(IterInfo)], _I),
    "pdas_direction_infeasible": ([_H] + [_P] * 9 + [ctypes.POINTER(IterInfo)], _I),
    "pdas_gemv": ([_H, _P, _P, _P], _I),
    "pdas_gemv_t": ([_H, _P, _P, _P], _I),
    "pdas_gemv_t_noalloc": ([_I64, _I64, _I, _P, _P, _P, _P], _I),
    "pdas_chol_tile_tasks": ([_I64, _I, _P, _I64], _I64),
    "pdas_batch_default_options": ([ctypes.POINTER(BatchOptions)], None),
    "pdas_batch_create": ([_I, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(BatchOptions), ctypes.POINTER(_H)],
                          _I),
    "pdas_batch_solve": ([_H, _P, _P, _P], _I),
    "pdas_batch_config": ([_H, _P, _P, _P, _I], _I),
    "pdas_batch_last_ms": ([_H], _D),
    "pdas_batch_diagnostics": ([_H, _P, _P, _P], _I),
    "pdas_batch_last_error_message": ([_H], ctypes.c_char_p),
    "pdas_batch_destroy": ([_H], None),
    "pdas_batch_backward": ([_H, _P, _P, _P, _P, _P], _I),
    "pdas_profile_enable": ([_H, _I], _I),
    "pdas_profile_read": ([_H, ctypes.POINTER(Profile)], _I),
    "pdas_woodbury_create": ([_I64, _I64, _I, _P, ctypes.POINTER(_H)], _I),
    "pdas_woodbury_prepare": ([_H, _P], _I),
    "pdas_woodbury_solve": ([_H, _P, _P, _P, _P, ctypes.POINTER(_D)], _I),
    "pdas_woodbury_last_error_message": ([_H], ctypes.c_char_p),
    "pdas_woodbury_destroy": ([_H], None),
}

_lib = None


def lib():
    """The loaded libpdas (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libpdas.so is not built (%s); run `python -m paper_1502_03543_gb300.build`"
                               % LIB_PATH)
        handle = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.argtypes = args
            fn.restype = res
        _lib = handle
    return _lib


def status_str(code: int) -> str:
    return lib().pdas_status_str(int(code)).decode()
