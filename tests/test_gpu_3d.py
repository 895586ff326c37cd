"""3D separable Haar transform on the GPU against the FP64 oracle."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1002_2184_gb300 import _lib, api, synth
from parity_util import assert_close

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


def volume(shape, seed, dtype=torch.float32):
    b = int(np.prod(shape[:-3]))
    d, h, w = shape[-3:]
    arr = np.stack([np.stack([synth.piecewise_smooth_image(h, w, seed=seed, index=i * d + z)
                              for z in range(d)]) for i in range(b)])
    return torch.from_numpy(arr.reshape(shape)).to(DEV).to(dtype)


CASES = [((1, 8, 8, 64), 1), ((1, 8, 8, 64), 2), ((2, 16, 32, 64), 3), ((1, 24, 40, 72), 3),
         ((1, 32, 32, 128), 5), ((3, 8, 16, 128), 3), ((1, 64, 64, 64), 6),
         ((1, 16, 24, 96), 3), ((2, 8, 8, 64), 3)]  # full and partial tiles mixed; batch


@pytest.mark.parametrize("shape,levels", CASES)
@pytest.mark.parametrize("dt", [torch.float32, torch.bfloat16])
def test_3d_matches_oracle(shape, levels, dt):
    x = volume(shape, seed=levels, dtype=dt)
    c = api.dwt3d(x, levels)
    ref = oracle.dwt3d(x.double().cpu().numpy(), levels)
    assert_close(c, ref, dt, f"dwt3d {shape} L{levels}")
    y = api.idwt3d(c, levels)
    yref = oracle.idwt3d(c.double().cpu().numpy(), levels)
    assert_close(y, yref, dt, f"idwt3d {shape} L{levels}")
    if dt == torch.float32:
        assert_close(y, x.double().cpu().numpy(), dt, f"3d round trip {shape} L{levels}")


def test_3d_fp64_and_strided():
    x = volume((2, 8, 16, 64), seed=3, dtype=torch.float64)
    c = api.dwt3d(x, 3)
    assert_close(c, oracle.dwt3d(x.cpu().numpy(), 3), torch.float64, "dwt3d fp64")
    big = volume((1, 12, 20, 160), seed=4)
    v = big[:, 2:10, 2:18, 32:96]   # plane stride 20*160, row stride 160
    cv = api.dwt3d(v, 3)
    assert_close(cv, oracle.dwt3d(v.double().cpu().numpy(), 3), torch.float32, "dwt3d strided")


# Volumes the tiled kernels cannot take run the generic per-level kernel:
# widths that are not multiples of 8, a second pass narrower than 8, rows
# that start off a 16-byte boundary; mixed storage types and fp64 too.
GENERIC = [((1, 8, 8, 12), 2), ((2, 16, 12, 20), 2), ((1, 16, 16, 48), 4), ((1, 4, 6, 2), 1),
           ((2, 32, 32, 36), 2)]


@pytest.mark.parametrize("shape,levels", GENERIC)
@pytest.mark.parametrize("dt,cdt", [(torch.float32, torch.float32), (torch.bfloat16, torch.bfloat16),
                                    (torch.float32, torch.bfloat16), (torch.float16, torch.float32)])
def test_3d_generic_path(shape, levels, dt, cdt):
    x = volume(shape, seed=levels + shape[-1], dtype=dt)
    c = api.dwt3d(x, levels, dtype=cdt)
    xh = x.double().cpu().numpy()
    assert_close(c, oracle.dwt3d(xh, levels), cdt if cdt != torch.float32 else dt,
                 f"generic dwt3d {shape} L{levels}")
    y = api.idwt3d(c, levels, dtype=dt)
    assert_close(y, oracle.idwt3d(c.double().cpu().numpy(), levels), cdt if cdt != torch.float32 else dt,
                 f"generic idwt3d {shape} L{levels}")


def test_3d_generic_unaligned_and_fp64():
    big = volume((1, 10, 18, 70), seed=6)
    v = big[:, 1:9, 1:17, 3:67]  # 8 x 16 x 64, rows starting 12 bytes past the allocation
    c = api.dwt3d(v, 3)
    assert_close(c, oracle.dwt3d(v.double().cpu().numpy(), 3), torch.float32, "unaligned dwt3d")
    y = api.idwt3d(c, 3)
    assert_close(y, v.double().cpu().numpy(), torch.float32, "unaligned round trip")
    x = volume((2, 8, 8, 12), seed=7, dtype=torch.float64)
    c = api.dwt3d(x, 2)
    assert_close(c, oracle.dwt3d(x.cpu().numpy(), 2), torch.float64, "generic fp64")


def test_3d_constant_exact_zero_detail():
    x = torch.full((1, 16, 16, 64), 0.25, device=DEV)
    c = api.dwt3d(x, 3).cpu().numpy()[0]
    low = c[:2, :2, :8]
    assert np.count_nonzero(c) == low.size


def test_3d_rejections():
    lib = _lib.load()
    st = torch.cuda.current_stream().cuda_stream
    x = torch.zeros(1, 8, 8, 12, device=DEV)
    assert lib.haar_dwt_3d(ctypes.byref(api.describe3(x)),
                           ctypes.byref(api.describe3(torch.zeros_like(x))), 3, None, 0, st) \
        == _lib.HAAR_ESHAPE  # 12 not divisible by 2^3
    y = torch.zeros(1, 8, 8, 64, device=DEV)
    assert lib.haar_dwt_3d(ctypes.byref(api.describe3(y)), ctypes.byref(api.describe3(y)), 1,
                           None, 0, st) == _lib.HAAR_EALIAS
    z = torch.zeros(1, 32, 32, 64, device=DEV)
    assert lib.haar_dwt_3d(ctypes.byref(api.describe3(z)),
                           ctypes.byref(api.describe3(torch.zeros_like(z))), 5, None, 0, st) \
        == _lib.HAAR_EWORKSPACE
    u = torch.zeros(1, 8, 8, 64, device=DEV, dtype=torch.uint8)
    assert lib.haar_dwt_3d(ctypes.byref(api.describe3(u)),
                           ctypes.byref(api.describe3(torch.zeros_like(y))), 1, None, 0, st) \
        == _lib.HAAR_EDTYPE
