"""Undecimated Haar transform on the GPU against the FP64 oracle."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1002_2184_gb300 import _lib, api, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


@pytest.mark.parametrize("rows,n,levels", [(1, 16, 1), (3, 2048, 4), (2, 6244, 3),
                                           (1, 1024, 10), (2, 5000, 7), (1, 65536, 6)])
@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
def test_swt_matches_oracle(rows, n, levels, dt):
    x = torch.from_numpy(np.stack([synth.signal_1d(n, seed=n, index=i) for i in range(rows)]))
    x = x.to(DEV).to(dt)
    u = api.swt1d(x, levels)
    ref = oracle.swt1d(x.double().cpu().numpy(), levels)
    tol = 1e-6 if dt == torch.float32 else 1e-13
    assert oracle.rel_l2(u.double().cpu().numpy(), ref) <= tol
    y = api.iswt1d(u, levels)
    yref = oracle.iswt1d(u.double().cpu().numpy(), levels)
    assert oracle.rel_l2(y.double().cpu().numpy(), yref) <= tol
    assert oracle.rel_l2(y.double().cpu().numpy(), x.double().cpu().numpy()) <= tol


def test_swt_decimated_equals_fast_dwt_on_gpu():
    """The direct (undecimated) form, decimated, is bit-identical to the
    Fast Haar analysis at level 1 (same two operations per output)."""
    x = torch.from_numpy(synth.signal_1d(1 << 16).astype(np.float32)).to(DEV)
    u = api.swt1d(x, 1)
    c = api.dwt1d(x, 1)
    n = x.numel()
    assert torch.equal(u[1, ::2], c[n // 2:])
    assert torch.equal(u[0, ::2], c[: n // 2])


def test_swt_rejections():
    lib = _lib.load()
    x = torch.zeros(2, 100, device=DEV)
    u = torch.zeros(2, 8, 100, device=DEV)
    st = torch.cuda.current_stream().cuda_stream
    assert lib.haar_swt_1d(x.data_ptr(), u.data_ptr(), 0, 2, 100, 7, st) == _lib.HAAR_ESHAPE
    assert lib.haar_swt_1d(x.data_ptr(), u.data_ptr(), 0, 2, 100, 11, st) == _lib.HAAR_EINVAL
    assert lib.haar_swt_1d(x.data_ptr(), x.data_ptr(), 0, 2, 100, 1, st) == _lib.HAAR_EALIAS
    assert lib.haar_swt_1d(x.data_ptr(), u.data_ptr(), 1, 2, 100, 1, st) == _lib.HAAR_EDTYPE
