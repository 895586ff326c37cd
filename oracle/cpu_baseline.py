"""The benchmark's FP32 CPU baseline -- TEST INFRASTRUCTURE ONLY, not the oracle.

``cpu_baseline.c`` is the Fast Haar method itself (one 2 x 2 butterfly per
block and level, Section III Fig. 4 and Section IV Eq. 19 along both axes)
as a plain single-threaded FP32 loop compiled with -O3: a fairer CPU
reference for the throughput comparison than the FP64 oracle, which forms
the bank by its definition.  Only the benchmark's CPU-baseline leg and the
tests use it.  ctypes releases the GIL during each call, so Python threads
running it over separate images use separate cores.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import build as _build

_LIB = None
_FP = ctypes.POINTER(ctypes.c_float)


def lib() -> ctypes.CDLL:
    global _LIB
    if _LIB is None:
        L = ctypes.CDLL(_build.build_baseline())
        for name in ("cpu_fast_haar_dwt2d_f32", "cpu_fast_haar_idwt2d_f32"):
            f = getattr(L, name)
            f.argtypes = [_FP, ctypes.c_long, ctypes.c_long, ctypes.c_int, _FP, _FP]
            f.restype = ctypes.c_int
        _LIB = L
    return _LIB


def _run(name: str, a: np.ndarray, levels: int) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float32)
    h, w = a.shape
    out = np.empty_like(a)
    work = np.empty(max(1, h * w // 2), dtype=np.float32)
    rc = getattr(lib(), name)(a.ctypes.data_as(_FP), h, w, levels, out.ctypes.data_as(_FP),
                              work.ctypes.data_as(_FP))
    if rc:
        raise ValueError(f"{name}: bad arguments (h={h}, w={w}, levels={levels})")
    return out


def dwt2d_f32(x: np.ndarray, levels: int) -> np.ndarray:
    """Multi-level 2D Fast Haar analysis of one h x w float32 image."""
    return _run("cpu_fast_haar_dwt2d_f32", x, levels)


def idwt2d_f32(c: np.ndarray, levels: int) -> np.ndarray:
    """Inverse of :func:`dwt2d_f32`."""
    return _run("cpu_fast_haar_idwt2d_f32", c, levels)
