"""Differentiable Fast Haar transforms and the wavelet-denoising loss.

The analysis W of the Haar bank is orthonormal (its synthesis taps are the
time-reversed analysis taps, arXiv:1002.2184 Section II), so W^-1 = W^T:
the adjoint (backward) of the analysis is the synthesis and vice versa.
Every forward and backward below runs in libfasthaar's kernels.

Two forms of the loss
    c = W x,  s = soft(c, t),  xr = W^T s,
    loss = mean((xr - x)^2) + lam * mean(|s| over detail coefficients):
  * ``denoise_loss``: fused -- because W W^T = I the residual is
    xr - x = -W^T clamp(c, -t, t) and the gradient is W^T q with q a
    per-coefficient map of c, so the forward and the backward are one launch
    each that read x only (4 and 8 bytes per pixel);
  * ``denoise_loss_unfused``: composed from DWT2d, SoftThresholdL1, IDWT2d
    and MSE, each a separate launch (autograd adds the two gradient
    contributions to x and the loss terms with torch's own elementwise ops).
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib, api


def _contig(t: torch.Tensor) -> torch.Tensor:
    return t if t.is_contiguous() else t.contiguous()


def _stream(t: torch.Tensor) -> int:
    return torch.cuda.current_stream(t.device).cuda_stream


def _n_detail(shape, levels) -> int:
    h, w = shape[-2], shape[-1]
    b = 1
    for d in shape[:-2]:
        b *= d
    return b * (h * w - (h >> levels) * (w >> levels))


class DWT2d(torch.autograd.Function):
    """Multi-level 2D analysis; backward = synthesis of the gradient."""

    @staticmethod
    def forward(ctx, x, levels: int):
        ctx.levels = levels
        return api.dwt2d(x, levels)

    @staticmethod
    def backward(ctx, g):
        return api.idwt2d(_contig(g), ctx.levels), None


class IDWT2d(torch.autograd.Function):
    """Multi-level 2D synthesis; backward = analysis of the gradient."""

    @staticmethod
    def forward(ctx, c, levels: int):
        ctx.levels = levels
        return api.idwt2d(c, levels)

    @staticmethod
    def backward(ctx, g):
        return api.dwt2d(_contig(g), ctx.levels), None


class DWT1d(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, levels: int):
        ctx.levels = levels
        return api.dwt1d(x, levels)

    @staticmethod
    def backward(ctx, g):
        return api.idwt1d(_contig(g), ctx.levels), None


class IDWT1d(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c, levels: int):
        ctx.levels = levels
        return api.idwt1d(c, levels)

    @staticmethod
    def backward(ctx, g):
        return api.dwt1d(_contig(g), ctx.levels), None


class SoftThresholdL1(torch.autograd.Function):
    """(s, l1) = (soft(c, t), mean |s| over detail coefficients)."""

    @staticmethod
    def forward(ctx, c, levels: int, t: float):
        lib = _lib.load()
        c = _contig(c)
        s = torch.empty_like(c)
        acc = torch.zeros(1, dtype=torch.float64, device=c.device)
        _lib.check(lib.haar_soft_threshold(ctypes.byref(api.describe(c)),
                                           ctypes.byref(api.describe(s)), levels, float(t),
                                           acc.data_ptr(), _stream(c)), "haar_soft_threshold")
        nd = _n_detail(c.shape, levels)
        ctx.levels, ctx.nd = levels, nd
        ctx.save_for_backward(s)
        return s, (acc / max(nd, 1)).to(c.dtype).reshape(())

    @staticmethod
    def backward(ctx, g_s, g_l1):
        lib = _lib.load()
        (s,) = ctx.saved_tensors
        g_s = torch.zeros_like(s) if g_s is None else _contig(g_s)
        g_c = torch.empty_like(s)
        gl = None if g_l1 is None else _contig(g_l1.to(s.dtype).reshape(1))
        _lib.check(lib.haar_soft_threshold_backward(
            ctypes.byref(api.describe(g_s)), ctypes.byref(api.describe(s)),
            ctypes.byref(api.describe(g_c)), ctx.levels, 1.0 / max(ctx.nd, 1),
            gl.data_ptr() if gl is not None else None, _stream(s)),
            "haar_soft_threshold_backward")
        return g_c, None, None


class MSE(torch.autograd.Function):
    """mean((a - b)^2) with an FP64 reduction."""

    @staticmethod
    def forward(ctx, a, b):
        lib = _lib.load()
        a, b = _contig(a), _contig(b)
        acc = torch.zeros(3, dtype=torch.float64, device=a.device)
        _lib.check(lib.haar_norms_f64(a.data_ptr(), b.data_ptr(), api.haar_dtype(a.dtype),
                                      a.numel(), acc.data_ptr(), _stream(a)), "haar_norms_f64")
        ctx.save_for_backward(a, b)
        return (acc[1] / max(a.numel(), 1)).to(a.dtype)

    @staticmethod
    def backward(ctx, g):
        lib = _lib.load()
        a, b = ctx.saved_tensors
        need_a, need_b = ctx.needs_input_grad
        ga = torch.empty_like(a) if need_a else None
        gb = torch.empty_like(b) if need_b else None
        gg = _contig(g.to(a.dtype).reshape(1))
        _lib.check(lib.haar_sq_diff_backward(
            ctypes.byref(api.describe(a)), ctypes.byref(api.describe(b)),
            ctypes.byref(api.describe(ga)) if ga is not None else None,
            ctypes.byref(api.describe(gb)) if gb is not None else None,
            2.0 / max(a.numel(), 1), gg.data_ptr(), _stream(a)), "haar_sq_diff_backward")
        return ga, gb


class DenoiseLoss(torch.autograd.Function):
    """The fused loss (haar_denoise_forward / haar_denoise_backward): both
    directions read x only and recompute the transform, so nothing but x is
    kept for the backward pass."""

    @staticmethod
    def forward(ctx, x, levels: int, t: float, lam: float):
        lib = _lib.load()
        x = _contig(x)
        acc = torch.zeros(2, dtype=torch.float64, device=x.device)
        loss = torch.empty((), dtype=x.dtype, device=x.device)
        _lib.check(lib.haar_denoise_forward(ctypes.byref(api.describe(x)), levels, float(t),
                                            float(lam), acc.data_ptr(), loss.data_ptr(),
                                            _stream(x)), "haar_denoise_forward")
        ctx.levels, ctx.t, ctx.lam = levels, float(t), float(lam)
        ctx.save_for_backward(x)
        return loss

    @staticmethod
    def backward(ctx, g):
        lib = _lib.load()
        (x,) = ctx.saved_tensors
        g_x = torch.empty_like(x)
        gg = _contig(g.to(x.dtype).reshape(1))
        _lib.check(lib.haar_denoise_backward(ctypes.byref(api.describe(x)),
                                             ctypes.byref(api.describe(g_x)), ctx.levels,
                                             ctx.t, ctx.lam, gg.data_ptr(), _stream(x)),
                   "haar_denoise_backward")
        return g_x, None, None, None


def dwt2d(x: torch.Tensor, levels: int) -> torch.Tensor:
    return DWT2d.apply(x, levels)


def idwt2d(c: torch.Tensor, levels: int) -> torch.Tensor:
    return IDWT2d.apply(c, levels)


def dwt1d(x: torch.Tensor, levels: int) -> torch.Tensor:
    return DWT1d.apply(x, levels)


def idwt1d(c: torch.Tensor, levels: int) -> torch.Tensor:
    return IDWT1d.apply(c, levels)


def denoise_loss(x: torch.Tensor, levels: int, t: float = 0.05, lam: float = 1e-3):
    """Fused wavelet-denoising loss (sides multiples of 32, levels <= 6)."""
    return DenoiseLoss.apply(x, levels, t, lam)


def denoise_loss_unfused(x: torch.Tensor, levels: int, t: float = 0.05, lam: float = 1e-3):
    """The same loss composed from separate differentiable ops."""
    c = DWT2d.apply(x, levels)
    s, l1 = SoftThresholdL1.apply(c, levels, t)
    xr = IDWT2d.apply(s, levels)
    return MSE.apply(xr, x) + lam * l1


class DenoisePlan:
    """The fused loss with its buffers bound once, for loops and CUDA
    graphs: forward() and backward() are fixed launch sequences with no
    allocation.  After forward(), ``loss`` holds the value; after
    backward(), ``grad`` holds d loss / d x (times ``g`` if given)."""

    def __init__(self, x: torch.Tensor, levels: int, t: float = 0.05, lam: float = 1e-3):
        self.lib = _lib.load()
        if not x.is_contiguous():
            raise ValueError("x must be contiguous")
        self.x, self.levels, self.t, self.lam = x, int(levels), float(t), float(lam)
        self.grad = torch.empty_like(x)
        self.acc = torch.zeros(2, dtype=torch.float64, device=x.device)
        self.loss = torch.empty((), dtype=x.dtype, device=x.device)
        self._dx, self._dg = api.describe(x), api.describe(self.grad)
        self._px, self._pg = ctypes.byref(self._dx), ctypes.byref(self._dg)

    def forward(self, stream=None) -> torch.Tensor:
        st = _stream(self.x) if stream is None else getattr(stream, "cuda_stream", stream)
        rc = self.lib.haar_denoise_forward(self._px, self.levels, self.t, self.lam,
                                           self.acc.data_ptr(), self.loss.data_ptr(), st)
        if rc:
            _lib.check(rc, "haar_denoise_forward")
        return self.loss

    def backward(self, g: torch.Tensor = None, stream=None) -> torch.Tensor:
        st = _stream(self.x) if stream is None else getattr(stream, "cuda_stream", stream)
        rc = self.lib.haar_denoise_backward(self._px, self._pg, self.levels, self.t, self.lam,
                                            g.data_ptr() if g is not None else None, st)
        if rc:
            _lib.check(rc, "haar_denoise_backward")
        return self.grad
