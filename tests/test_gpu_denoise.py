"""One-pass wavelet shrinkage (haar_denoise_1d / haar_denoise_2d) and the
warp-block 1D transforms, against the FP64 oracle."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1002_2184_gb300 import _lib, api, synth
from parity_util import assert_close

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


def gpu_decision(c: torch.Tensor, t: float) -> np.ndarray:
    """|c| > t taken as the kernels take it: on the FP32 coefficients (the
    separate analysis performs the same operations as the one inside the
    fused kernels) against the threshold rounded to FP32.  Hard shrinkage
    jumps at |c| = t, so the oracle is handed this decision: a coefficient
    within rounding of t would otherwise be kept on one side only."""
    return (c.abs() > torch.tensor(t, dtype=torch.float32)).cpu().numpy()


def signals(rows, n, seed, dtype=torch.float32):
    return torch.from_numpy(np.stack([synth.signal_1d(n, seed=seed, index=i)
                                      for i in range(rows)])).to(DEV).to(dtype)


def images(b, h, w, seed, dtype=torch.float32):
    return torch.from_numpy(np.stack([synth.piecewise_smooth_image(h, w, seed=seed, index=i)
                                      for i in range(b)])).to(DEV).to(dtype)


@pytest.mark.parametrize("levels", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("hard", [False, True])
def test_denoise1d_matches_oracle(levels, hard):
    x = signals(6, 4096, seed=levels).reshape(2, 3, 4096)
    t = 0.8
    y = api.denoise1d(x, levels, t, hard)
    ref = oracle.denoise1d(x.double().cpu().numpy(), levels, t, hard,
                           keep=gpu_decision(api.dwt1d(x, levels), t) if hard else None)
    assert_close(y, ref, torch.float32, f"denoise1d L{levels} hard={hard}")
    y64 = api.denoise1d(x.double(), levels, t, hard)
    assert_close(y64, ref, torch.float64, f"denoise1d fp64 L{levels} hard={hard}")


@pytest.mark.parametrize("levels", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("hard", [False, True])
def test_denoise2d_matches_oracle(levels, hard):
    x = images(3, 96, 160, seed=levels)
    t = 0.05
    y = api.denoise2d(x, levels, t, hard)
    ref = oracle.denoise2d(x.double().cpu().numpy(), levels, t, hard,
                           keep=gpu_decision(api.dwt2d(x, levels), t) if hard else None)
    assert_close(y, ref, torch.float32, f"denoise2d L{levels} hard={hard}")
    y64 = api.denoise2d(x.double(), levels, t, hard)
    assert_close(y64, ref, torch.float64, f"denoise2d fp64 L{levels} hard={hard}")


def test_denoise_limits_on_gpu():
    """Infinite threshold: block means; zero threshold: the input."""
    x = signals(2, 2048, seed=3)
    y = api.denoise1d(x, 5, 1e30)
    blocks = x.reshape(2, -1, 32).double().mean(-1)
    assert torch.allclose(y.double(), blocks.repeat_interleave(32, -1), atol=1e-5)
    assert torch.allclose(api.denoise1d(x, 5, 0.0, hard=True), x, atol=1e-5)
    im = images(1, 64, 64, seed=4)
    y2 = api.denoise2d(im, 5, 1e30)
    m = im.double().reshape(1, 2, 32, 2, 32).mean(dim=(2, 4))
    assert torch.allclose(y2.double(), m.repeat_interleave(32, 1).repeat_interleave(32, 2),
                          atol=1e-5)


def test_denoise_strided_views():
    base = images(2, 96, 320, seed=5)
    x = base[:, :64, 32:288]          # row stride 320, aligned offset
    y = api.denoise2d(x, 4, 0.05)
    ref = oracle.denoise2d(x.double().cpu().numpy(), 4, 0.05)
    assert_close(y, ref, torch.float32, "denoise2d strided view")


def test_denoise_rejections():
    lib = _lib.load()
    x = torch.zeros(2, 1000, device=DEV)
    y = torch.zeros_like(x)
    st = torch.cuda.current_stream().cuda_stream
    d = lambda t, one: ctypes.byref(api.describe(t, one))
    assert lib.haar_denoise_1d(d(x, True), d(y, True), 3, 0.1, 0, st) == _lib.HAAR_ESHAPE
    x2 = torch.zeros(2, 256, device=DEV)
    assert lib.haar_denoise_1d(d(x2, True), d(x2, True), 3, 0.1, 0, st) == _lib.HAAR_EALIAS
    assert lib.haar_denoise_1d(d(x2, True), d(torch.zeros_like(x2), True), 9, 0.1, 0, st) \
        == _lib.HAAR_EINVAL
    assert lib.haar_denoise_1d(d(x2, True), d(torch.zeros_like(x2), True), 3, 0.1, 7, st) \
        == _lib.HAAR_EINVAL
    im = torch.zeros(1, 48, 64, device=DEV)
    assert lib.haar_denoise_2d(d(im, False), d(torch.zeros_like(im), False), 3, 0.1, 0, st) \
        == _lib.HAAR_ESHAPE
    bf = torch.zeros(1, 64, 64, device=DEV, dtype=torch.bfloat16)
    assert lib.haar_denoise_2d(d(bf, False), d(torch.zeros_like(bf), False), 3, 0.1, 0, st) \
        == _lib.HAAR_EDTYPE


# The warp-block 1D transform: every level count 1..8, partial blocks of 8
# warps, batches of rows, fp32 / bf16 and a deep transform that chains a
# chunk pass and a warp-block pass.
@pytest.mark.parametrize("rows,n,levels", [(3, 256, 8), (2, 768, 4), (4, 2048, 1),
                                           (1, 4096, 5), (2, 6144, 7), (1, 512, 2),
                                           (2, 1280, 3), (1, 1 << 18, 14)])
@pytest.mark.parametrize("dt", [torch.float32, torch.bfloat16])
def test_warp_block_1d(rows, n, levels, dt):
    x = signals(rows, n, seed=n + levels, dtype=dt)
    c = api.dwt1d(x, levels)
    ref = oracle.dwt1d(x.double().cpu().numpy(), levels)
    assert_close(c, ref, dt, f"warp-block dwt1d {rows}x{n} L{levels}")
    y = api.idwt1d(c, levels)
    yref = oracle.idwt1d(c.double().cpu().numpy(), levels)
    assert_close(y, yref, dt, f"warp-block idwt1d {rows}x{n} L{levels}")
