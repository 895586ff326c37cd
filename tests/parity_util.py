"""Shared comparison rules for the GPU parity tests (no GPU needed to import).

Every comparison of a CUDA result with the FP64 oracle checks two things:
the relative L2 error over the compared array (the bar of the method's
accuracy statement: 1e-6 for fp32 storage, 1e-2 for bf16) and an
element-wise bound, so that a few wrong elements in a large array (a
wrapped window edge, a partial tile, a seam between chunks) cannot hide
under the norm.

Tolerances per storage type (rel-L2, max-abs relative to max|ref|):
  fp32: 1e-6, 4e-6    -- a handful of fp32 roundings (u = 2^-24 = 6e-8) per
                         output, each bounded by u times the largest input
  bf16: 1e-2, 2^-7    -- one bf16 rounding of the output (2^-8 relative)
  fp16: 2e-3, 2^-9    -- one fp16 rounding (2^-11 relative) plus input scale
  fp64: 1e-13, 1e-13
"""
import numpy as np
import torch

import oracle

TOL = {
    torch.float32: (1e-6, 4e-6),
    torch.bfloat16: (1e-2, 2.0 ** -7),
    torch.float16: (2e-3, 2.0 ** -9),
    torch.float64: (1e-13, 1e-13),
}


def _host(a) -> np.ndarray:
    if isinstance(a, torch.Tensor):
        return a.detach().double().cpu().numpy()
    return np.asarray(a, dtype=np.float64)


def assert_close(gpu, ref, dtype, what="", scale=None):
    """rel-L2 <= TOL[dtype][0] and max|gpu - ref| <= TOL[dtype][1] * scale,
    scale defaulting to max|ref| (the largest magnitude that fed the
    result).  Returns (rel_l2, max_abs)."""
    got = _host(gpu)
    ref = _host(ref)
    assert got.shape == ref.shape, f"{what}: shape {got.shape} != {ref.shape}"
    rel_tol, abs_tol = TOL[dtype]
    err = oracle.rel_l2(got, ref)
    if scale is None:
        scale = float(np.max(np.abs(ref))) if ref.size else 0.0
    mx = oracle.max_abs(got, ref)
    assert err <= rel_tol, f"{what}: rel-L2 {err:.3e} > {rel_tol:.1e}"
    assert mx <= abs_tol * max(scale, 1e-30), f"{what}: max-abs {mx:.3e} (scale {scale:.3e})"
    return err, mx


def mallat_bands_1d(n: int, levels: int):
    """(name, start, stop, level) of every band of a 1D Mallat row
    [a_L | d_L | ... | d_1]; level is the level whose input produced it."""
    bands = [("a%d" % levels, 0, n >> levels, levels)]
    for l in range(levels, 0, -1):
        bands.append(("d%d" % l, n >> l, n >> (l - 1), l))
    return bands


def assert_bands_close_1d(got, ref, approx, levels, dtype, what="", abs_factor=1.0):
    """Band-by-band comparison of 1D Mallat coefficient rows.

    ``approx[l]`` is the oracle's level-l approximation a_l (approx[0] = the
    input), the signal a level-l band is computed from.  Each band of level l
    must satisfy ||band - ref|| <= rel_tol * ||a_{l-1}|| (rows taken
    separately) and max|band - ref| <= abs_tol * abs_factor * max|a_{l-1}|.
    Scaling by the band's own input, not by the whole row, keeps the bound
    as strict for the few coefficients of the deepest level as for d_1: an
    error confined to a coarse band or a chunk seam cannot hide under the
    norm of the finer bands."""
    got = _host(got)
    ref = _host(ref)
    n = got.shape[-1]
    assert got.shape == ref.shape, f"{what}: shape {got.shape} != {ref.shape}"
    rel_tol, abs_tol = TOL[dtype]
    g2 = got.reshape(-1, n)
    r2 = ref.reshape(-1, n)
    for name, lo, hi, l in mallat_bands_1d(n, levels):
        src = _host(approx[l - 1]).reshape(g2.shape[0], -1)
        diff = g2[:, lo:hi] - r2[:, lo:hi]
        num = np.linalg.norm(diff, axis=1)
        den = np.linalg.norm(src, axis=1)
        worst = float(np.max(num / np.maximum(den, 1e-300)))
        assert worst <= rel_tol, f"{what} band {name}: rel {worst:.3e} > {rel_tol:.1e}"
        mx = float(np.max(np.abs(diff))) if diff.size else 0.0
        scale = float(np.max(np.abs(src)))
        assert mx <= abs_tol * abs_factor * max(scale, 1e-30), \
            f"{what} band {name}: max-abs {mx:.3e} (input scale {scale:.3e})"
