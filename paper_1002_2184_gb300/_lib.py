"""ctypes binding of libfasthaar.so (include/fasthaar.h).

Argument marshalling only: every computation happens inside the library's
CUDA kernels.  Loading fails loudly when the library has not been built;
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfasthaar.so")

# Status codes (fasthaar.h).
HAAR_OK = 0
HAAR_EINVAL = -1
HAAR_ESHAPE = -2
HAAR_EDTYPE = -3
HAAR_EALIAS = -4
HAAR_ECUDA = -5
HAAR_ETIMEOUT = -6
HAAR_EWORKSPACE = -7
HAAR_EQUEUE = -8

# Storage types.
HAAR_F32, HAAR_BF16, HAAR_F16, HAAR_U8, HAAR_F64 = 0, 1, 2, 3, 4

# Shrinkage rules of haar_denoise_1d / haar_denoise_2d.
HAAR_THRESH_SOFT, HAAR_THRESH_HARD = 0, 1

# Ragged work-unit shapes.
HAAR_UNIT_64x128, HAAR_UNIT_32x256, HAAR_UNIT_64x64, HAAR_UNIT_128x128 = 0, 1, 2, 3

# Workspace-size operation codes.
HAAR_OP_DWT_1D, HAAR_OP_IDWT_1D, HAAR_OP_DWT_2D, HAAR_OP_IDWT_2D = 0, 1, 2, 3


class HaarDesc(ctypes.Structure):
    _fields_ = [
        ("ptr", ctypes.c_void_p),
        ("dtype", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("batch", ctypes.c_int64),
        ("h", ctypes.c_int64),
        ("w", ctypes.c_int64),
        ("batch_stride", ctypes.c_int64),
        ("row_stride", ctypes.c_int64),
    ]


class HaarDesc3(ctypes.Structure):
    _fields_ = [
        ("ptr", ctypes.c_void_p),
        ("dtype", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("batch", ctypes.c_int64),
        ("d", ctypes.c_int64),
        ("h", ctypes.c_int64),
        ("w", ctypes.c_int64),
        ("batch_stride", ctypes.c_int64),
        ("plane_stride", ctypes.c_int64),
        ("row_stride", ctypes.c_int64),
    ]


class HaarRaggedItem(ctypes.Structure):
    _fields_ = [
        ("in_offset", ctypes.c_int64),
        ("out_offset", ctypes.c_int64),
        ("h", ctypes.c_int64),
        ("w", ctypes.c_int64),
        ("in_row_stride", ctypes.c_int64),
        ("out_row_stride", ctypes.c_int64),
        ("levels", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class HaarError(RuntimeError):
    """A non-zero status returned by the library."""

    def __init__(self, status: int, what: str):
        self.status = status
        msg = _LIB.haar_status_string(status).decode() if _LIB is not None else str(status)
        if status == HAAR_ECUDA and _LIB is not None:
            msg += f" (cudaError {_LIB.haar_last_cuda_error()})"
        super().__init__(f"{what}: {msg} [{status}]")


_LIB = None

# name -> (restype, argtypes)
_P = ctypes.c_void_p
_DP = ctypes.POINTER(HaarDesc)
_D3 = ctypes.POINTER(HaarDesc3)
SIGNATURES = {
    "haar_version": (ctypes.c_int, []),
    "haar_last_cuda_error": (ctypes.c_int, []),
    "haar_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "haar_workspace_size": (ctypes.c_int, [ctypes.c_int, _DP, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_size_t)]),
    "haar_dwt_1d": (ctypes.c_int, [_DP, _DP, ctypes.c_int, _P, ctypes.c_size_t, _P]),
    "haar_idwt_1d": (ctypes.c_int, [_DP, _DP, ctypes.c_int, _P, ctypes.c_size_t, _P]),
    "haar_dwt_2d": (ctypes.c_int, [_DP, _DP, ctypes.c_int, _P, ctypes.c_size_t, _P]),
    "haar_idwt_2d": (ctypes.c_int, [_DP, _DP, ctypes.c_int, _P, ctypes.c_size_t, _P]),
    "haar_workspace_size_3d": (ctypes.c_int, [_D3, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    "haar_dwt_3d": (ctypes.c_int, [_D3, _D3, ctypes.c_int, _P, ctypes.c_size_t, _P]),
    "haar_idwt_3d": (ctypes.c_int, [_D3, _D3, ctypes.c_int, _P, ctypes.c_size_t, _P]),
    "haar_dwt_2d_noalloc": (ctypes.c_int, [_DP, _DP, ctypes.c_int, _P]),
    "haar_ragged_plan_create": (ctypes.c_int, [ctypes.POINTER(HaarRaggedItem), ctypes.c_int64,
                                               ctypes.c_int, ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_void_p)]),
    "haar_ragged_workspace_size": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "haar_ragged_plan_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64),
                                             ctypes.POINTER(ctypes.c_int64),
                                             ctypes.POINTER(ctypes.c_int64)]),
    "haar_ragged_upload": (ctypes.c_int, [_P, _P, ctypes.c_size_t, _P]),
    "haar_dwt_2d_ragged": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, ctypes.c_int, _P,
                                          ctypes.c_size_t, _P]),
    "haar_idwt_2d_ragged": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, ctypes.c_int, _P,
                                           ctypes.c_size_t, _P]),
    "haar_ragged_status": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int), _P]),
    "haar_ragged_plan_destroy": (ctypes.c_int, [_P]),
    "haar_norms_f64": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int64, _P, _P]),
    "haar_soft_threshold": (ctypes.c_int, [_DP, _DP, ctypes.c_int, ctypes.c_double, _P, _P]),
    "haar_soft_threshold_backward": (ctypes.c_int, [_DP, _DP, _DP, ctypes.c_int,
                                                    ctypes.c_double, _P, _P]),
    "haar_sq_diff_backward": (ctypes.c_int, [_DP, _DP, _DP, _DP, ctypes.c_double, _P, _P]),
    "haar_filter_dwt_1d": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                          ctypes.c_int, _P]),
    "haar_filter_idwt_1d": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int64,
                                           ctypes.c_int64, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_double), ctypes.c_int, _P]),
    "haar_swt_1d": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                   ctypes.c_int, _P]),
    "haar_iswt_1d": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                    ctypes.c_int, _P]),
    "haar_denoise_1d": (ctypes.c_int, [_DP, _DP, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                       _P]),
    "haar_denoise_2d": (ctypes.c_int, [_DP, _DP, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                       _P]),
    "haar_denoise_forward": (ctypes.c_int, [_DP, ctypes.c_int, ctypes.c_double,
                                            ctypes.c_double, _P, _P, _P]),
    "haar_denoise_backward": (ctypes.c_int, [_DP, _DP, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_double, _P, _P]),
}


def load() -> ctypes.CDLL:
    """Load the built library (raises if it is missing)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"libfasthaar.so not found at {LIB_PATH}; build it with "
                "`python -m paper_1002_2184_gb300.build` (nvcc, sm_103a)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _LIB = lib
    return _LIB


def check(status: int, what: str) -> None:
    if status != HAAR_OK:
        raise HaarError(status, what)


def desc(ptr: int, dtype: int, batch: int, h: int, w: int, batch_stride: int,
         row_stride: int) -> HaarDesc:
    return HaarDesc(ptr, dtype, 0, batch, h, w, batch_stride, row_stride)
