"""FP64 CPU oracle of the Haar filter bank -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library under
``paper_1002_2184_gb300`` never imports it and shares no code with it.

The transforms are the plain definition of the two-channel bank of
arXiv:1002.2184 Section II (Fig. 1): convolve, then decimate; upsample, then
convolve and sum.  They live in ``haar_oracle.c`` (see its header for the
readings of the paper).  This module marshals numpy arrays into it and adds
the pieces of the denoising loss (soft threshold, MSE + L1) used by the
differentiation workload, written out in numpy.

Every function works on float64 and returns new arrays.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import build as _build

_LIB = None
_DP = ctypes.POINTER(ctypes.c_double)


def lib() -> ctypes.CDLL:
    """Load (building first if needed) the compiled oracle."""
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        for name in ("oracle_analysis_1d", "oracle_polyphase_analysis_1d"):
            f = getattr(L, name)
            f.argtypes = [_DP, ctypes.c_long, _DP, _DP, ctypes.c_int]
            f.restype = ctypes.c_int
        for name in ("oracle_synthesis_1d", "oracle_polyphase_synthesis_1d"):
            f = getattr(L, name)
            f.argtypes = [_DP, _DP, ctypes.c_long, _DP, ctypes.c_int]
            f.restype = ctypes.c_int
        for name in ("oracle_dwt_1d", "oracle_idwt_1d"):
            f = getattr(L, name)
            f.argtypes = [_DP, ctypes.c_long, ctypes.c_int, _DP, ctypes.c_int]
            f.restype = ctypes.c_int
        for name in ("oracle_dwt_2d", "oracle_idwt_2d"):
            f = getattr(L, name)
            f.argtypes = [_DP, ctypes.c_long, ctypes.c_long, ctypes.c_int, _DP,
                          ctypes.c_int]
            f.restype = ctypes.c_int
        for name in ("oracle_dwt_3d", "oracle_idwt_3d"):
            f = getattr(L, name)
            f.argtypes = [_DP, ctypes.c_long, ctypes.c_long, ctypes.c_long, ctypes.c_int, _DP,
                          ctypes.c_int]
            f.restype = ctypes.c_int
        _LIB = L
    return _LIB


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"oracle: {what} rejected its arguments")


# --------------------------------------------------------------------------
# One stage of the bank (Section II, Fig. 1) and its polyphase form (Fig. 4,
# Fig. 7), on a single 1D signal.
# --------------------------------------------------------------------------

def analysis_1d(x, detail_sign: int = 1):
    """Convolve with b0/b1 and decimate: returns (d0, d1)."""
    x = _f64(x)
    n = x.shape[-1]
    lo = np.empty(n // 2)
    hi = np.empty(n // 2)
    _check(lib().oracle_analysis_1d(_p(x), n, _p(lo), _p(hi), detail_sign),
           "analysis_1d")
    return lo, hi


def synthesis_1d(lo, hi, detail_sign: int = 1):
    """Upsample d0/d1, convolve with a0/a1 and add (Eq. 13)."""
    lo, hi = _f64(lo), _f64(hi)
    m = lo.shape[-1]
    x = np.empty(2 * m)
    _check(lib().oracle_synthesis_1d(_p(lo), _p(hi), m, _p(x), detail_sign),
           "synthesis_1d")
    return x


def polyphase_analysis_1d(x, detail_sign: int = 1):
    """The Fast Haar analysis bank (Fig. 4); for the existing-vs-fast check."""
    x = _f64(x)
    n = x.shape[-1]
    lo = np.empty(n // 2)
    hi = np.empty(n // 2)
    _check(lib().oracle_polyphase_analysis_1d(_p(x), n, _p(lo), _p(hi),
                                              detail_sign),
           "polyphase_analysis_1d")
    return lo, hi


def polyphase_synthesis_1d(lo, hi, detail_sign: int = 1):
    """The Fast Haar synthesis bank (Eq. 19, Fig. 7)."""
    lo, hi = _f64(lo), _f64(hi)
    m = lo.shape[-1]
    x = np.empty(2 * m)
    _check(lib().oracle_polyphase_synthesis_1d(_p(lo), _p(hi), m, _p(x),
                                               detail_sign),
           "polyphase_synthesis_1d")
    return x


# --------------------------------------------------------------------------
# Multi-level transforms (Mallat layout), any number of leading batch dims.
# --------------------------------------------------------------------------

def dwt1d(x, levels: int, detail_sign: int = 1) -> np.ndarray:
    """Multi-level 1D analysis over the last axis: [a_L | d_L | ... | d_1]."""
    x = _f64(x)
    n = x.shape[-1]
    flat = x.reshape(-1, n)
    out = np.empty_like(flat)
    for i in range(flat.shape[0]):
        src = np.ascontiguousarray(flat[i])
        dst = np.empty(n)
        _check(lib().oracle_dwt_1d(_p(src), n, levels, _p(dst), detail_sign),
               "dwt_1d")
        out[i] = dst
    return out.reshape(x.shape)


def idwt1d(c, levels: int, detail_sign: int = 1) -> np.ndarray:
    """Inverse of :func:`dwt1d`."""
    c = _f64(c)
    n = c.shape[-1]
    flat = c.reshape(-1, n)
    out = np.empty_like(flat)
    for i in range(flat.shape[0]):
        src = np.ascontiguousarray(flat[i])
        dst = np.empty(n)
        _check(lib().oracle_idwt_1d(_p(src), n, levels, _p(dst), detail_sign),
               "idwt_1d")
        out[i] = dst
    return out.reshape(c.shape)


def dwt2d(x, levels: int, detail_sign: int = 1) -> np.ndarray:
    """Multi-level separable 2D analysis over the last two axes (Mallat)."""
    x = _f64(x)
    h, w = x.shape[-2:]
    flat = x.reshape(-1, h, w)
    out = np.empty_like(flat)
    for i in range(flat.shape[0]):
        src = np.ascontiguousarray(flat[i])
        dst = np.empty((h, w))
        _check(lib().oracle_dwt_2d(_p(src), h, w, levels, _p(dst),
                                   detail_sign), "dwt_2d")
        out[i] = dst
    return out.reshape(x.shape)


def idwt2d(c, levels: int, detail_sign: int = 1) -> np.ndarray:
    """Inverse of :func:`dwt2d`."""
    c = _f64(c)
    h, w = c.shape[-2:]
    flat = c.reshape(-1, h, w)
    out = np.empty_like(flat)
    for i in range(flat.shape[0]):
        src = np.ascontiguousarray(flat[i])
        dst = np.empty((h, w))
        _check(lib().oracle_idwt_2d(_p(src), h, w, levels, _p(dst),
                                    detail_sign), "idwt_2d")
        out[i] = dst
    return out.reshape(c.shape)


def dwt3d(x, levels: int, detail_sign: int = 1) -> np.ndarray:
    """Multi-level separable 3D analysis over the last three axes (octant
    Mallat layout; not in the paper)."""
    x = _f64(x)
    d, h, w = x.shape[-3:]
    flat = x.reshape(-1, d, h, w)
    out = np.empty_like(flat)
    for i in range(flat.shape[0]):
        src = np.ascontiguousarray(flat[i])
        dst = np.empty((d, h, w))
        _check(lib().oracle_dwt_3d(_p(src), d, h, w, levels, _p(dst), detail_sign), "dwt_3d")
        out[i] = dst
    return out.reshape(x.shape)


def idwt3d(c, levels: int, detail_sign: int = 1) -> np.ndarray:
    """Inverse of :func:`dwt3d`."""
    c = _f64(c)
    d, h, w = c.shape[-3:]
    flat = c.reshape(-1, d, h, w)
    out = np.empty_like(flat)
    for i in range(flat.shape[0]):
        src = np.ascontiguousarray(flat[i])
        dst = np.empty((d, h, w))
        _check(lib().oracle_idwt_3d(_p(src), d, h, w, levels, _p(dst), detail_sign), "idwt_3d")
        out[i] = dst
    return out.reshape(c.shape)


# --------------------------------------------------------------------------
# Layout helpers: which coefficients are details (everything but a_L / LL_L).
# --------------------------------------------------------------------------

def detail_mask_1d(n: int, levels: int) -> np.ndarray:
    m = np.ones(n, dtype=bool)
    m[: n >> levels] = False
    return m


def detail_mask_2d(h: int, w: int, levels: int) -> np.ndarray:
    m = np.ones((h, w), dtype=bool)
    m[: h >> levels, : w >> levels] = False
    return m


# --------------------------------------------------------------------------
# Denoising loss of the differentiation workload (not in the paper):
#   c = DWT(x);  s = soft(c, t);  xr = IDWT(s)
#   loss = mean((xr - x)^2) + lam * mean(|s| over detail coefficients)
# soft() acts on every coefficient; its subgradient is 0 at |c| <= t.
# --------------------------------------------------------------------------

def soft_threshold(c, t: float) -> np.ndarray:
    c = _f64(c)
    return np.sign(c) * np.maximum(np.abs(c) - t, 0.0)


def denoise_loss(x, levels: int, t: float, lam: float):
    """Returns (loss, mse, l1) for a batch (..., h, w), each image separately
    transformed and the means taken over the whole batch."""
    x = _f64(x)
    h, w = x.shape[-2:]
    c = dwt2d(x, levels)
    s = soft_threshold(c, t)
    xr = idwt2d(s, levels)
    mask = np.broadcast_to(detail_mask_2d(h, w, levels), x.shape)
    mse = float(np.mean((xr - x) ** 2))
    l1 = float(np.mean(np.abs(s[mask])))
    return mse + lam * l1, mse, l1


def denoise_loss_grad(x, levels: int, t: float, lam: float, keep=None) -> np.ndarray:
    """Closed-form gradient of :func:`denoise_loss` with respect to x.

    With W the orthonormal DWT (so IDWT = W^T and its adjoint is W):
      g_xr = 2 (xr - x) / n
      g_s  = W g_xr + lam * sign(s) * mask / n_d
      g_c  = g_s * [|c| > t]
      g_x  = W^T g_c - 2 (xr - x) / n

    keep: optionally the decision [|c| > t] as the implementation under test
    took it, in its own precision.  The gradient jumps where |c| crosses t,
    so a coefficient within rounding of t may be decided differently in FP32
    and FP64; a comparison element by element needs both sides to decide the
    same way, and the mask replaces the FP64 comparison here (the values are
    still FP64)."""
    x = _f64(x)
    h, w = x.shape[-2:]
    n = x.size
    c = dwt2d(x, levels)
    s = soft_threshold(c, t)
    xr = idwt2d(s, levels)
    mask = np.broadcast_to(detail_mask_2d(h, w, levels), x.shape)
    n_d = int(mask.sum())
    g_xr = 2.0 * (xr - x) / n
    g_s = dwt2d(g_xr, levels) + lam * np.sign(s) * mask / n_d
    g_c = g_s * ((np.abs(c) > t) if keep is None else np.asarray(keep, dtype=bool))
    return idwt2d(g_c, levels) - g_xr


# --------------------------------------------------------------------------
# General orthonormal two-channel bank (K taps), periodic boundary: the
# definition -- circular correlation with h and g, keep every other output
# -- and its adjoint.  g[k] = (-1)^(k+1) h[K-1-k].
# --------------------------------------------------------------------------

def qmf_highpass(h) -> np.ndarray:
    h = np.asarray(h, dtype=np.float64)
    K = h.size
    return np.array([(-1.0) ** (k + 1) * h[K - 1 - k] for k in range(K)])


def filter_analysis_1d(x, h):
    x = _f64(x)
    h = np.asarray(h, dtype=np.float64)
    g = qmf_highpass(h)
    n = x.shape[-1]
    lo = np.zeros(x.shape[:-1] + (n // 2,))
    hi = np.zeros_like(lo)
    for k in range(h.size):
        idx = (2 * np.arange(n // 2) + k) % n
        lo += h[k] * x[..., idx]
        hi += g[k] * x[..., idx]
    return lo, hi


def filter_synthesis_1d(lo, hi, h):
    lo, hi = _f64(lo), _f64(hi)
    h = np.asarray(h, dtype=np.float64)
    g = qmf_highpass(h)
    m = lo.shape[-1]
    n = 2 * m
    x = np.zeros(lo.shape[:-1] + (n,))
    for k in range(h.size):
        idx = (2 * np.arange(m) + k) % n
        # adjoint of the analysis: scatter-add each coefficient to the
        # samples it was formed from
        np.add.at(x, (..., idx), h[k] * lo + g[k] * hi)
    return x


def filter_dwt1d(x, levels: int, h) -> np.ndarray:
    x = _f64(x)
    n = x.shape[-1]
    out = np.empty_like(x)
    a = x.copy()
    length = n
    for _ in range(levels):
        lo, hi = filter_analysis_1d(a, h)
        out[..., length // 2: length] = hi
        length //= 2
        a = lo
    out[..., :length] = a
    return out


def filter_idwt1d(c, levels: int, h) -> np.ndarray:
    c = _f64(c)
    n = c.shape[-1]
    length = n >> levels
    a = c[..., :length].copy()
    for _ in range(levels):
        a = filter_synthesis_1d(a, c[..., length: 2 * length], h)
        length *= 2
    return a


# --------------------------------------------------------------------------
# Undecimated (stationary) transform: the bank of Fig. 1 without the
# down-sampler, filters dilated by 2^(l-1) at level l, periodic boundary.
# Output (..., L + 1, n): row 0 = a_L, row l = d_l.
# --------------------------------------------------------------------------

def swt1d(x, levels: int) -> np.ndarray:
    x = _f64(x)
    s2 = 1.0 / np.sqrt(2.0)
    a = x.copy()
    out = np.empty(x.shape[:-1] + (levels + 1, x.shape[-1]))
    for l in range(1, levels + 1):
        s = 1 << (l - 1)
        nxt = np.roll(a, -s, axis=-1)  # a[k + s], wrapping around
        out[..., l, :] = (nxt - a) * s2
        a = (a + nxt) * s2
    out[..., 0, :] = a
    return out


def iswt1d(c, levels: int) -> np.ndarray:
    c = _f64(c)
    s2 = 1.0 / np.sqrt(2.0)
    a = c[..., 0, :].copy()
    for l in range(levels, 0, -1):
        s = 1 << (l - 1)
        d = c[..., l, :]
        # two estimates of a_{l-1}[k]: from position k and from position k - s
        e1 = (a - d) * s2
        e2 = np.roll((a + d) * s2, s, axis=-1)
        a = 0.5 * (e1 + e2)
    return a


# --------------------------------------------------------------------------
# Wavelet shrinkage (denoising): threshold every detail coefficient, keep the
# low band, transform back.
# --------------------------------------------------------------------------

def shrink(d, t: float, hard: bool = False, keep=None) -> np.ndarray:
    """Soft: sign(d) max(|d| - t, 0).  Hard: d [|d| > t]; keep optionally
    gives that decision as the implementation under test took it in its own
    precision (hard shrinkage jumps at |d| = t, so both sides of an
    element-by-element comparison must decide alike)."""
    d = _f64(d)
    if hard:
        k = (np.abs(d) > t) if keep is None else np.asarray(keep, dtype=bool)
        return np.where(k, d, 0.0)
    return np.sign(d) * np.maximum(np.abs(d) - t, 0.0)


def denoise1d(x, levels: int, t: float, hard: bool = False, keep=None) -> np.ndarray:
    x = _f64(x)
    c = dwt1d(x, levels)
    mask = np.broadcast_to(detail_mask_1d(x.shape[-1], levels), c.shape)
    c = np.where(mask, shrink(c, t, hard, keep), c)
    return idwt1d(c, levels)


def denoise2d(x, levels: int, t: float, hard: bool = False, keep=None) -> np.ndarray:
    x = _f64(x)
    h, w = x.shape[-2:]
    c = dwt2d(x, levels)
    mask = np.broadcast_to(detail_mask_2d(h, w, levels), c.shape)
    c = np.where(mask, shrink(c, t, hard, keep), c)
    return idwt2d(c, levels)


# --------------------------------------------------------------------------
# Error measures reported next to every result.
# --------------------------------------------------------------------------

def rel_l2(a, ref) -> float:
    a, ref = _f64(a), _f64(ref)
    den = np.linalg.norm(ref.ravel())
    num = np.linalg.norm((a - ref).ravel())
    return float(num / den) if den > 0 else float(num)


def max_abs(a, ref) -> float:
    a, ref = _f64(a), _f64(ref)
    return float(np.max(np.abs(a - ref))) if a.size else 0.0


__all__ = [
    "lib", "analysis_1d", "synthesis_1d", "polyphase_analysis_1d",
    "polyphase_synthesis_1d", "dwt1d", "idwt1d", "dwt2d", "idwt2d", "dwt3d", "idwt3d",
    "detail_mask_1d", "detail_mask_2d", "soft_threshold", "denoise_loss",
    "denoise_loss_grad", "qmf_highpass", "filter_analysis_1d", "filter_synthesis_1d",
    "filter_dwt1d", "filter_idwt1d", "swt1d", "iswt1d", "shrink", "denoise1d", "denoise2d", "rel_l2", "max_abs",
]
