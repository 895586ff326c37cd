"""Undecimated Haar transform on the GPU against the FP64 oracle."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1002_2184_gb300 import _lib, api, synth
from parity_util import assert_close

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


@pytest.mark.parametrize("rows,n,levels", [(1, 16, 1), (3, 2048, 4), (2, 6244, 3),
                                           (1, 1024, 10), (2, 5000, 7), (1, 65536, 6)])
@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
def test_swt_matches_oracle(rows, n, levels, dt):
    x = torch.from_numpy(np.stack([synth.signal_1d(n, seed=n, index=i) for i in range(rows)]))
    x = x.to(DEV).to(dt)
    u = api.swt1d(x, levels)
    xh = x.double().cpu().numpy()
    ref = oracle.swt1d(xh, levels)
    # level by level: d_l (row l) is scaled by its own input a_{l-1}, a_L by
    # a_{L-1}, so an error confined to one level cannot hide in the others
    for l in range(levels + 1):
        lev = levels if l == 0 else l
        src = xh if lev == 1 else oracle.swt1d(xh, lev - 1)[..., 0, :]
        assert_close(u[..., l, :], ref[..., l, :], dt, f"swt row {l} {rows}x{n} L{levels}",
                     scale=float(np.max(np.abs(src))))
    y = api.iswt1d(u, levels)
    yref = oracle.iswt1d(u.double().cpu().numpy(), levels)
    assert_close(y, yref, dt, f"iswt {rows}x{n} L{levels}")
    assert_close(y, xh, dt, f"swt round trip {rows}x{n} L{levels}")


@pytest.mark.parametrize("rows,n,levels", [(2, 64, 1), (3, 2048, 4), (1, 5000, 7),
                                           (2, 1024, 10)])
@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
def test_iswt_inconsistent_coefficients(rows, n, levels, dt):
    """The inverse on coefficients that are not the transform of any signal
    (independent random rows, as after shrinkage or noise): each level must
    average the two estimates of a_{l-1}, as the oracle does.  Keeping only
    one estimate agrees with the oracle on consistent input but not here."""
    rng = np.random.default_rng(1000 + n + levels)
    u = rng.standard_normal((rows, levels + 1, n))
    ud = torch.from_numpy(u).to(DEV).to(dt)
    y = api.iswt1d(ud, levels)
    yref = oracle.iswt1d(ud.double().cpu().numpy(), levels)
    assert_close(y, yref, dt, f"iswt inconsistent {rows}x{n} L{levels}")


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
