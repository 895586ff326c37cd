"""PyTorch-facing calls into libfasthaar: tensors in, tensors out.

These functions only describe tensors to the C ABI (pointer, dtype, extents,
strides) and pass torch's current CUDA stream; the transforms run in the
library's kernels.  Inputs must be CUDA tensors whose rows are contiguous and
whose leading dimensions flatten to one batch stride.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Tuple

import torch

from . import _lib

_DTYPES = {
    torch.float32: _lib.HAAR_F32,
    torch.bfloat16: _lib.HAAR_BF16,
    torch.float16: _lib.HAAR_F16,
    torch.uint8: _lib.HAAR_U8,
    torch.float64: _lib.HAAR_F64,
}


def haar_dtype(dt: torch.dtype) -> int:
    try:
        return _DTYPES[dt]
    except KeyError:
        raise TypeError(f"unsupported dtype {dt}") from None


def _lead_stride(t: torch.Tensor, nlead: int, inner: int) -> Tuple[int, int]:
    """(count, stride) of the first ``nlead`` dims flattened into one; raises
    if they are not evenly strided."""
    count, stride = 1, None
    for d in range(nlead - 1, -1, -1):
        n, s = t.shape[d], t.stride(d)
        if n == 1:
            continue
        if stride is None:
            stride = s
            expect = s * n
        else:
            if s != expect:
                raise ValueError("leading dimensions do not flatten to one batch stride; "
                                 "pass a contiguous tensor")
            expect = s * n
        count *= n
    return count, (stride if stride is not None else inner)


def describe(t: torch.Tensor, one_d: bool = False) -> _lib.HaarDesc:
    """The haar_desc of a tensor: (..., h, w) for 2D; (..., w) for 1D, where
    every row is one signal."""
    if not t.is_cuda:
        raise ValueError("libfasthaar works on CUDA tensors only")
    if t.dim() < 1 or (not one_d and t.dim() < 2):
        raise ValueError("tensor has too few dimensions")
    if t.numel() and t.shape[-1] > 1 and t.stride(-1) != 1:
        raise ValueError("rows must be contiguous (last stride 1)")
    w = t.shape[-1]
    if t.dim() == 1:
        h, rs, batch, bs = 1, w, 1, w
    else:
        h, rs = t.shape[-2], t.stride(-2)
        if h == 1:
            rs = w
        batch, bs = _lead_stride(t, t.dim() - 2, h * rs)
    return _lib.desc(t.data_ptr(), haar_dtype(t.dtype), batch, h, w, bs, rs)


def _stream(t: torch.Tensor) -> int:
    return torch.cuda.current_stream(t.device).cuda_stream


def workspace_size(op: int, d: _lib.HaarDesc, levels: int) -> int:
    lib = _lib.load()
    n = ctypes.c_size_t(0)
    _lib.check(lib.haar_workspace_size(op, ctypes.byref(d), levels, ctypes.byref(n)),
               "haar_workspace_size")
    return n.value


def _run(fn_name: str, op: int, src: torch.Tensor, dst: torch.Tensor, levels: int,
         one_d: bool) -> torch.Tensor:
    lib = _lib.load()
    ds, dd = describe(src, one_d), describe(dst, one_d)
    nbytes = workspace_size(op, ds, levels)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=src.device) if nbytes else None
    with torch.cuda.device(src.device):
        rc = getattr(lib, fn_name)(ctypes.byref(ds), ctypes.byref(dd), levels,
                                   ws.data_ptr() if ws is not None else None, nbytes,
                                   _stream(src))
    _lib.check(rc, fn_name)
    return dst


def _out_like(x: torch.Tensor, dtype: torch.dtype, out: Optional[torch.Tensor]) -> torch.Tensor:
    if out is None:
        return torch.empty(x.shape, dtype=dtype, device=x.device)
    if out.shape != x.shape:
        raise ValueError(f"out has shape {tuple(out.shape)}, expected {tuple(x.shape)}")
    if out.device != x.device:
        raise ValueError(f"out is on {out.device}, the input on {x.device}")
    return out


def _check_same_type(what: str, src: torch.Tensor, out: torch.Tensor, shape) -> None:
    """For the entry points that take one element type and plain pointers for
    both buffers: out must have the given shape, src's dtype and device, and
    both must be contiguous CUDA tensors (checked before the library is
    called, so a mismatch never reaches a kernel)."""
    if tuple(out.shape) != tuple(shape):
        raise ValueError(f"{what}: out has shape {tuple(out.shape)}, expected {tuple(shape)}")
    if out.dtype != src.dtype:
        raise ValueError(f"{what}: out has dtype {out.dtype}, the input {src.dtype}")
    if not (src.is_contiguous() and out.is_contiguous()):
        raise ValueError(f"{what} needs contiguous tensors")
    if out.device != src.device:
        raise ValueError(f"{what}: out is on {out.device}, the input on {src.device}")
    if not src.is_cuda:
        raise ValueError("libfasthaar works on CUDA tensors only")


def _coef_dtype(x: torch.Tensor, dtype: Optional[torch.dtype]) -> torch.dtype:
    if dtype is not None:
        return dtype
    return torch.float32 if x.dtype == torch.uint8 else x.dtype


def dwt2d(x: torch.Tensor, levels: int, out: Optional[torch.Tensor] = None,
          dtype: Optional[torch.dtype] = None) -> torch.Tensor:
    """Multi-level 2D Fast Haar analysis of (..., h, w) into the Mallat layout."""
    out = _out_like(x, _coef_dtype(x, dtype) if out is None else out.dtype, out)
    return _run("haar_dwt_2d", _lib.HAAR_OP_DWT_2D, x, out, levels, False)


def idwt2d(c: torch.Tensor, levels: int, out: Optional[torch.Tensor] = None,
           dtype: Optional[torch.dtype] = None) -> torch.Tensor:
    """Inverse of :func:`dwt2d`."""
    out = _out_like(c, (dtype or c.dtype) if out is None else out.dtype, out)
    return _run("haar_idwt_2d", _lib.HAAR_OP_IDWT_2D, c, out, levels, False)


def dwt1d(x: torch.Tensor, levels: int, out: Optional[torch.Tensor] = None,
          dtype: Optional[torch.dtype] = None) -> torch.Tensor:
    """Multi-level 1D Fast Haar analysis of every row of (..., n)."""
    out = _out_like(x, _coef_dtype(x, dtype) if out is None else out.dtype, out)
    return _run("haar_dwt_1d", _lib.HAAR_OP_DWT_1D, x, out, levels, True)


def idwt1d(c: torch.Tensor, levels: int, out: Optional[torch.Tensor] = None,
           dtype: Optional[torch.dtype] = None) -> torch.Tensor:
    """Inverse of :func:`dwt1d`."""
    out = _out_like(c, (dtype or c.dtype) if out is None else out.dtype, out)
    return _run("haar_idwt_1d", _lib.HAAR_OP_IDWT_1D, c, out, levels, True)


class Plan:
    """A transform bound to fixed tensors: descriptors, level count and
    workspace are prepared once, so each call is a single C-ABI call with no
    allocation (safe to capture into a CUDA graph).

    ``Plan(x, coef, levels, y=None, one_d=False)`` plans x -> coef (analysis)
    and, when ``y`` is given, coef -> y (synthesis).
    """

    def __init__(self, x: torch.Tensor, coef: torch.Tensor, levels: int,
                 y: Optional[torch.Tensor] = None, one_d: bool = False):
        for t in (coef, y):
            if t is not None and t.device != x.device:
                raise ValueError(f"Plan: a buffer is on {t.device}, the input on {x.device}")
        self.lib = _lib.load()
        self.levels = int(levels)
        self.device = x.device
        self._dev_index = x.device.index
        self._keep = (x, coef, y)
        self._dx = describe(x, one_d)
        self._dc = describe(coef, one_d)
        self._dy = describe(y, one_d) if y is not None else None
        if one_d:
            ops = (_lib.HAAR_OP_DWT_1D, _lib.HAAR_OP_IDWT_1D)
            self._fwd, self._inv = self.lib.haar_dwt_1d, self.lib.haar_idwt_1d
        else:
            ops = (_lib.HAAR_OP_DWT_2D, _lib.HAAR_OP_IDWT_2D)
            self._fwd, self._inv = self.lib.haar_dwt_2d, self.lib.haar_idwt_2d
        n = max(workspace_size(ops[0], self._dx, self.levels),
                workspace_size(ops[1], self._dc, self.levels))
        self._ws = torch.empty(n, dtype=torch.uint8, device=x.device) if n else None
        self._ws_ptr = self._ws.data_ptr() if n else None
        self._ws_n = n
        self._px, self._pc = ctypes.byref(self._dx), ctypes.byref(self._dc)
        self._py = ctypes.byref(self._dy) if y is not None else None

    def _stream(self, stream) -> int:
        if stream is None:
            return torch.cuda.current_stream(self.device).cuda_stream
        return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)

    # The library launches on the calling thread's current device: the call
    # is made with the plan's device current (switched only when another
    # device is current, so the common case costs one device query).
    def _call(self, fn, a, b, stream, what):
        if torch.cuda.current_device() == self._dev_index:
            rc = fn(a, b, self.levels, self._ws_ptr, self._ws_n, self._stream(stream))
        else:
            with torch.cuda.device(self.device):
                rc = fn(a, b, self.levels, self._ws_ptr, self._ws_n, self._stream(stream))
        if rc:
            _lib.check(rc, what)

    def dwt(self, stream=None) -> None:
        self._call(self._fwd, self._px, self._pc, stream, "dwt")

    def idwt(self, stream=None) -> None:
        if self._py is None:
            raise ValueError("plan has no synthesis output")
        self._call(self._inv, self._pc, self._py, stream, "idwt")


class RaggedPlan:
    """A ragged batch of 2D images (different sizes and level counts) packed
    one after another in flat buffers, transformed by one persistent launch.

    ``items`` is a list of (h, w, levels); image i occupies elements
    ``offsets[i] : offsets[i] + h*w`` (row-major, contiguous) of every flat
    buffer used with this plan.  ``unit`` and ``blocks_per_sm`` select the
    work-unit shape and the persistent grid (see autotune.tune_ragged).
    The workspace is allocated and uploaded once; dwt()/idwt() are then
    single launches, safe to capture into a CUDA graph.
    """

    def __init__(self, items, device, unit: int = _lib.HAAR_UNIT_64x128,
                 blocks_per_sm: int = 4):
        self.lib = _lib.load()
        self.items = [(int(h), int(w), int(L)) for h, w, L in items]
        self.device = torch.device(device)
        if self.device.type == "cuda" and self.device.index is None:  # "cuda": the current GPU
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.unit, self.blocks_per_sm = int(unit), int(blocks_per_sm)
        offs, o = [], 0
        for h, w, _ in self.items:
            offs.append(o)
            o += h * w
        self.offsets, self.numel = offs, o
        arr = (_lib.HaarRaggedItem * max(1, len(self.items)))()
        for i, ((h, w, L), off) in enumerate(zip(self.items, offs)):
            arr[i] = _lib.HaarRaggedItem(off, off, h, w, w, w, L, 0)
        handle = ctypes.c_void_p()
        _lib.check(self.lib.haar_ragged_plan_create(arr, len(self.items), self.unit,
                                                    self.blocks_per_sm, ctypes.byref(handle)),
                   "haar_ragged_plan_create")
        self._h = handle
        n = ctypes.c_size_t()
        _lib.check(self.lib.haar_ragged_workspace_size(handle, ctypes.byref(n)),
                   "haar_ragged_workspace_size")
        self._ws_n = n.value
        self._ws = torch.empty(self._ws_n, dtype=torch.uint8, device=self.device)
        with torch.cuda.device(self.device):
            _lib.check(self.lib.haar_ragged_upload(handle, self._ws.data_ptr(), self._ws_n,
                                                   torch.cuda.current_stream(self.device)
                                                   .cuda_stream), "haar_ragged_upload")

    def info(self):
        u, p, g = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        with torch.cuda.device(self.device):
            _lib.check(self.lib.haar_ragged_plan_info(self._h, ctypes.byref(u), ctypes.byref(p),
                                                      ctypes.byref(g)), "haar_ragged_plan_info")
        return {"units": u.value, "pixels": p.value, "grid": g.value}

    def empty(self, dtype=torch.float32) -> torch.Tensor:
        return torch.empty(self.numel, dtype=dtype, device=self.device)

    def views(self, flat: torch.Tensor):
        """The (h, w) image views of a flat buffer laid out by this plan."""
        return [flat[o:o + h * w].view(h, w) for (h, w, _), o in zip(self.items, self.offsets)]

    def _run(self, fn, src: torch.Tensor, dst: torch.Tensor, stream=None):
        if src.numel() < self.numel or dst.numel() < self.numel:
            raise ValueError("buffer smaller than the plan's layout")
        if src.device != self.device or dst.device != self.device:
            raise ValueError(f"ragged buffers must be on the plan's device {self.device}")
        if not (src.is_contiguous() and dst.is_contiguous()):
            raise ValueError("ragged buffers must be contiguous")
        st = (torch.cuda.current_stream(self.device).cuda_stream if stream is None
              else getattr(stream, "cuda_stream", stream))
        # the persistent grid is sized from the current device's SM count
        if torch.cuda.current_device() == self.device.index:
            rc = fn(self._h, src.data_ptr(), haar_dtype(src.dtype), dst.data_ptr(),
                    haar_dtype(dst.dtype), self._ws.data_ptr(), self._ws_n, st)
        else:
            with torch.cuda.device(self.device):
                rc = fn(self._h, src.data_ptr(), haar_dtype(src.dtype), dst.data_ptr(),
                        haar_dtype(dst.dtype), self._ws.data_ptr(), self._ws_n, st)
        if rc:
            _lib.check(rc, "ragged transform")
        return dst

    def dwt(self, x: torch.Tensor, out: torch.Tensor, stream=None) -> torch.Tensor:
        return self._run(self.lib.haar_dwt_2d_ragged, x, out, stream)

    def idwt(self, c: torch.Tensor, out: torch.Tensor, stream=None) -> torch.Tensor:
        return self._run(self.lib.haar_idwt_2d_ragged, c, out, stream)

    def status(self) -> int:
        """HAAR_OK, or HAAR_EQUEUE if a launch saw an inconsistent queue
        (synchronises the current stream)."""
        st = ctypes.c_int(0)
        with torch.cuda.device(self.device):
            _lib.check(self.lib.haar_ragged_status(self._h, self._ws.data_ptr(), ctypes.byref(st),
                                                   torch.cuda.current_stream(self.device)
                                                   .cuda_stream), "haar_ragged_status")
        return st.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib._LIB is not None:
            _lib._LIB.haar_ragged_plan_destroy(h)
            self._h = None


def denoise1d(x: torch.Tensor, levels: int, threshold: float, hard: bool = False,
              out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """One-pass wavelet shrinkage of every row of (..., n): analysis, soft
    (or hard) thresholding of the detail coefficients, synthesis."""
    out = _out_like(x, x.dtype, out)
    lib = _lib.load()
    with torch.cuda.device(x.device):
        rc = lib.haar_denoise_1d(ctypes.byref(describe(x, True)), ctypes.byref(describe(out, True)),
                                 levels, float(threshold),
                                 _lib.HAAR_THRESH_HARD if hard else _lib.HAAR_THRESH_SOFT,
                                 _stream(x))
    _lib.check(rc, "haar_denoise_1d")
    return out


def denoise2d(x: torch.Tensor, levels: int, threshold: float, hard: bool = False,
              out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """One-pass wavelet shrinkage of every image of (..., h, w)."""
    out = _out_like(x, x.dtype, out)
    lib = _lib.load()
    with torch.cuda.device(x.device):
        rc = lib.haar_denoise_2d(ctypes.byref(describe(x)), ctypes.byref(describe(out)), levels,
                                 float(threshold),
                                 _lib.HAAR_THRESH_HARD if hard else _lib.HAAR_THRESH_SOFT,
                                 _stream(x))
    _lib.check(rc, "haar_denoise_2d")
    return out


def swt1d(x: torch.Tensor, levels: int, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Undecimated Haar transform of every row of (..., n) (contiguous):
    returns (..., levels + 1, n) with [a_L, d_1, ..., d_L]."""
    n = x.shape[-1]
    rows = x.numel() // max(n, 1)
    shape = tuple(x.shape[:-1]) + (levels + 1, n)
    out = torch.empty(shape, dtype=x.dtype, device=x.device) if out is None else out
    _check_same_type("swt1d", x, out, shape)
    lib = _lib.load()
    with torch.cuda.device(x.device):
        rc = lib.haar_swt_1d(x.data_ptr(), out.data_ptr(), haar_dtype(x.dtype), rows, n, levels,
                             _stream(x))
    _lib.check(rc, "haar_swt_1d")
    return out


def iswt1d(c: torch.Tensor, levels: int, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Inverse of :func:`swt1d`."""
    n = c.shape[-1]
    if c.dim() < 2 or c.shape[-2] != levels + 1:
        raise ValueError(f"iswt1d: coefficients of shape (..., {levels + 1}, n) expected, "
                         f"got {tuple(c.shape)}")
    shape = tuple(c.shape[:-2]) + (n,)
    rows = c.numel() // max((levels + 1) * n, 1)
    out = torch.empty(shape, dtype=c.dtype, device=c.device) if out is None else out
    _check_same_type("iswt1d", c, out, shape)
    lib = _lib.load()
    with torch.cuda.device(c.device):
        rc = lib.haar_iswt_1d(c.data_ptr(), out.data_ptr(), haar_dtype(c.dtype), rows, n, levels,
                              _stream(c))
    _lib.check(rc, "haar_iswt_1d")
    return out


def describe3(t: torch.Tensor) -> _lib.HaarDesc3:
    """The haar_desc3 of a (..., d, h, w) CUDA tensor with contiguous rows."""
    if not t.is_cuda:
        raise ValueError("libfasthaar works on CUDA tensors only")
    if t.dim() < 3:
        raise ValueError("a volume needs three dimensions")
    if t.numel() and t.shape[-1] > 1 and t.stride(-1) != 1:
        raise ValueError("rows must be contiguous (last stride 1)")
    d, h, w = t.shape[-3:]
    rs = t.stride(-2) if h > 1 else w
    zs = t.stride(-3) if d > 1 else h * rs
    batch, bs = _lead_stride(t, t.dim() - 3, d * zs)
    return _lib.HaarDesc3(t.data_ptr(), haar_dtype(t.dtype), 0, batch, d, h, w, bs, zs, rs)


def _run3(fn_name: str, src: torch.Tensor, dst: torch.Tensor, levels: int) -> torch.Tensor:
    lib = _lib.load()
    ds, dd = describe3(src), describe3(dst)
    # the workspace depends on which kernels take the transform, which both
    # arrays' layouts decide: the larger of the two answers covers it
    need = 0
    for d in (ds, dd):
        n = ctypes.c_size_t(0)
        _lib.check(lib.haar_workspace_size_3d(ctypes.byref(d), levels, ctypes.byref(n)),
                   "haar_workspace_size_3d")
        need = max(need, n.value)
    n = ctypes.c_size_t(need)
    ws = torch.empty(need, dtype=torch.uint8, device=src.device) if need else None
    with torch.cuda.device(src.device):
        rc = getattr(lib, fn_name)(ctypes.byref(ds), ctypes.byref(dd), levels,
                                   ws.data_ptr() if ws is not None else None, n.value,
                                   _stream(src))
    _lib.check(rc, fn_name)
    return dst


def dwt3d(x: torch.Tensor, levels: int, out: Optional[torch.Tensor] = None,
          dtype: Optional[torch.dtype] = None) -> torch.Tensor:
    """Multi-level separable 3D analysis of (..., d, h, w) (octant layout)."""
    out = _out_like(x, (dtype or x.dtype) if out is None else out.dtype, out)
    return _run3("haar_dwt_3d", x, out, levels)


def idwt3d(c: torch.Tensor, levels: int, out: Optional[torch.Tensor] = None,
           dtype: Optional[torch.dtype] = None) -> torch.Tensor:
    """Inverse of :func:`dwt3d`."""
    out = _out_like(c, (dtype or c.dtype) if out is None else out.dtype, out)
    return _run3("haar_idwt_3d", c, out, levels)


# Orthonormal Daubechies low-pass filters (closed forms).
_R3 = 3.0 ** 0.5
DAUBECHIES4 = tuple(v / (4.0 * 2.0 ** 0.5) for v in (1 + _R3, 3 + _R3, 3 - _R3, 1 - _R3))
HAAR2 = (2.0 ** -0.5, 2.0 ** -0.5)


def daubechies(ntaps: int) -> Tuple[float, ...]:
    """Daubechies' orthonormal low-pass with ntaps / 2 vanishing moments
    (ntaps in {2, 4, 6, 8}: the lengths the K-tap kernels take), by the
    spectral factorisation of Daubechies' construction: with N = ntaps / 2,
    |m0(w)|^2 = cos^(2N)(w/2) Q(sin^2(w/2)), Q(y) = sum_{k<N} C(N-1+k, k) y^k;
    substituting y = -(z - 1)^2 / (4z) makes z^(N-1) Q a polynomial in z
    whose roots come in pairs r, 1/r, and the filter is (1 + z)^N times the
    factor with the roots inside the unit circle (minimum phase), scaled to
    sum(h) = sqrt(2).  ntaps = 2 gives HAAR2 and 4 gives DAUBECHIES4."""
    import numpy as np
    from math import comb
    if ntaps not in (2, 4, 6, 8):
        raise ValueError("ntaps must be 2, 4, 6 or 8")
    n = ntaps // 2
    poly = np.zeros(1)
    for k in range(n):
        term = np.array([comb(n - 1 + k, k) * (-0.25) ** k])
        for _ in range(k):
            term = np.polymul(term, [1.0, -2.0, 1.0])  # (z - 1)^2
        term = np.polymul(term, np.r_[1.0, np.zeros(n - 1 - k)])  # z^(n-1-k)
        poly = np.polyadd(poly, term)
    h = np.array([1.0])
    if n > 1:
        roots = np.roots(poly)
        h = np.real(np.poly(roots[np.abs(roots) < 1.0]))
    for _ in range(n):
        h = np.polymul(h, [1.0, 1.0])
    h = h * (2.0 ** 0.5) / h.sum()
    return tuple(float(v) for v in h)


def _filter_call(fn_name, src, dst, levels, taps):
    _check_same_type(fn_name, src, dst, src.shape)
    n = src.shape[-1]
    rows = src.numel() // max(n, 1)
    arr = (ctypes.c_double * len(taps))(*taps)
    lib = _lib.load()
    with torch.cuda.device(src.device):
        rc = getattr(lib, fn_name)(src.data_ptr(), dst.data_ptr(), haar_dtype(src.dtype), rows, n,
                                   levels, arr, len(taps), _stream(src))
    _lib.check(rc, fn_name)
    return dst


def filter_dwt1d(x: torch.Tensor, levels: int, taps=DAUBECHIES4,
                 out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Multi-level 1D analysis with an orthonormal K-tap low-pass (periodic)."""
    return _filter_call("haar_filter_dwt_1d", x, _out_like(x, x.dtype, out), levels, taps)


def filter_idwt1d(c: torch.Tensor, levels: int, taps=DAUBECHIES4,
                  out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Inverse of :func:`filter_dwt1d`."""
    return _filter_call("haar_filter_idwt_1d", c, _out_like(c, c.dtype, out), levels, taps)
