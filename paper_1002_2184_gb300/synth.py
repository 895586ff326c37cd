"""Seeded synthetic inputs shaped like the paper's workloads.

The paper's own data (a laser-Doppler recording of one subject and the Lena
image, Section V) are not available, so these generators stand in for them.
This module holds no transform arithmetic: it only draws inputs, and both the
CUDA path and the test oracle are fed from it.

All draws use numpy's PCG64 seeded from ``SEED_BASE + workload index`` and a
per-item index, so any single image of a batch can be regenerated alone.
Values are drawn in float64; callers cast them to the storage dtype.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED_BASE = 10022184


def rng(seed: int, index: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, index])))


# --------------------------------------------------------------------------
# Workload shapes (one per benchmark configuration).
# --------------------------------------------------------------------------

@dataclass(frozen=True)
class Signal1D:
    """1D fp32 signal, 2^16 samples, one level."""
    n: int = 1 << 16
    levels: int = 1
    seed: int = SEED_BASE + 0


@dataclass(frozen=True)
class Image2D:
    """4096 x 4096 fp32 piecewise-smooth image, 5 levels."""
    h: int = 4096
    w: int = 4096
    levels: int = 5
    seed: int = SEED_BASE + 1


@dataclass(frozen=True)
class PrecisionBatch:
    """64 single-channel 2048 x 2048 images, bf16/fp16/u8 storage, 4 levels."""
    batch: int = 64
    h: int = 2048
    w: int = 2048
    levels: int = 4
    seed: int = SEED_BASE + 2


@dataclass(frozen=True)
class RaggedBatch:
    """512 images, h and w each uniform on {64, 128, ..., 2048}, levels 3..6."""
    count: int = 512
    side_step: int = 64
    side_max: int = 2048
    level_min: int = 3
    level_max: int = 6
    seed: int = SEED_BASE + 3


@dataclass(frozen=True)
class GradBatch:
    """32 x 3 x 512 x 512 fp32, 3 levels, soft threshold 0.05, L1 weight 1e-3."""
    shape: tuple = (32, 3, 512, 512)
    levels: int = 3
    threshold: float = 0.05
    l1_weight: float = 1e-3
    seed: int = SEED_BASE + 4


# --------------------------------------------------------------------------
# Generators.
# --------------------------------------------------------------------------

def signal_1d(n: int, seed: int = Signal1D.seed, index: int = 0) -> np.ndarray:
    """i.i.d. N(0,1) noise plus three sinusoids with frequencies U(0, 0.5)
    cycles/sample, amplitudes U[0.5, 2] and phases U[0, 2 pi)."""
    g = rng(seed, index)
    t = np.arange(n, dtype=np.float64)
    x = g.standard_normal(n)
    for _ in range(3):
        f = g.uniform(0.0, 0.5)
        a = g.uniform(0.5, 2.0)
        ph = g.uniform(0.0, 2.0 * math.pi)
        x += a * np.sin(2.0 * math.pi * f * t + ph)
    return x


def piecewise_smooth_image(h: int, w: int, seed: int = Image2D.seed,
                           index: int = 0, rectangles: int = 200,
                           noise_sigma: float = 0.01) -> np.ndarray:
    """Linear-gradient background 0.5 (x/w + y/h), then ``rectangles``
    axis-aligned rectangles painted in order (later ones overwrite), each
    with width ~ U[w/64, w/4], height ~ U[h/64, h/4], a uniform position and
    intensity U[0, 1]; then Gaussian noise of standard deviation 0.01."""
    g = rng(seed, index)
    yy = np.arange(h, dtype=np.float64)[:, None] / h
    xx = np.arange(w, dtype=np.float64)[None, :] / w
    img = 0.5 * (xx + yy)
    for _ in range(rectangles):
        rw = max(1, int(g.uniform(w / 64, w / 4)))
        rh = max(1, int(g.uniform(h / 64, h / 4)))
        x0 = int(g.integers(0, w - rw + 1))
        y0 = int(g.integers(0, h - rh + 1))
        img[y0:y0 + rh, x0:x0 + rw] = g.uniform(0.0, 1.0)
    img += noise_sigma * g.standard_normal((h, w))
    return img


def image_batch(count: int, h: int, w: int, seed: int,
                dtype=np.float32) -> np.ndarray:
    """``count`` independent piecewise-smooth images, cast to ``dtype``."""
    out = np.empty((count, h, w), dtype=dtype)
    for i in range(count):
        out[i] = piecewise_smooth_image(h, w, seed, i)
    return out


def quantize_u8(x: np.ndarray) -> np.ndarray:
    """The uint8 copy of an image: round(clip(x, 0, 1) * 255)."""
    return np.rint(np.clip(x, 0.0, 1.0) * 255.0).astype(np.uint8)


def ragged_shapes(cfg: RaggedBatch = RaggedBatch()):
    """List of (h, w, levels): h and w drawn independently and uniformly from
    {step, 2 step, ..., side_max}; levels uniform on level_min..level_max,
    capped at log2(min(h, w)) and at the largest power of two dividing both
    sides."""
    g = rng(cfg.seed, 1 << 20)
    sides = np.arange(cfg.side_step, cfg.side_max + 1, cfg.side_step)
    shapes = []
    for _ in range(cfg.count):
        h = int(g.choice(sides))
        w = int(g.choice(sides))
        lv = int(g.integers(cfg.level_min, cfg.level_max + 1))
        cap = int(math.floor(math.log2(min(h, w))))
        while lv > 0 and (h % (1 << lv) or w % (1 << lv)):
            lv -= 1
        shapes.append((h, w, min(lv, cap)))
    return shapes


def ragged_images(shapes, cfg: RaggedBatch = RaggedBatch(),
                  dtype=np.float32, indices=None):
    """The images of a ragged batch (all of them, or only ``indices``)."""
    idx = range(len(shapes)) if indices is None else indices
    return {i: piecewise_smooth_image(shapes[i][0], shapes[i][1], cfg.seed, i)
            .astype(dtype) for i in idx}
