"""The polyphase bank with longer orthonormal filters on the GPU against the
FP64 oracle (K = 2, 4, 6, 8 taps, several level counts, chunk seams)."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1002_2184_gb300 import _lib, api, synth
from parity_util import assert_bands_close_1d, assert_close
from test_oracle_pins import _d4, lattice_lowpass

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)

def approximations(x: np.ndarray, levels: int, h) -> list:
    """The oracle's a_0 = x, a_1, ..., a_levels (the input of each level)."""
    n = x.shape[-1]
    return [x] + [oracle.filter_dwt1d(x, l, np.array(h))[..., : n >> l]
                  for l in range(1, levels + 1)]


TAPS = {"haar": tuple(np.full(2, 1 / np.sqrt(2.0))), "d4": tuple(_d4()),
        "lattice6": tuple(lattice_lowpass([0.3, -0.7, 1.1])),
        "lattice8": tuple(lattice_lowpass([0.2, 0.5, -0.4, 0.9])),
        "db6": api.daubechies(6), "db8": api.daubechies(8)}


@pytest.mark.parametrize("name", list(TAPS))
@pytest.mark.parametrize("rows,n,levels", [(1, 64, 3), (3, 4096, 6), (2, 6144, 10),
                                           (1, 1 << 16, 4), (2, 1024, 10), (1, 16, 4),
                                           # one or two levels (a single pass), odd and even
                                           # level counts, full chunks followed by a ragged one
                                           # (4096- and 8192-sample chunks)
                                           (3, 4096, 1), (2, 8192, 2), (1, 2048, 5),
                                           (2, 4096 + 256, 7), (2, 10240, 9), (1, 12288, 8)])
@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
def test_filter_bank_matches_oracle(name, rows, n, levels, dt):
    h = TAPS[name]
    x = torch.from_numpy(np.stack([synth.signal_1d(n, seed=n, index=i) for i in range(rows)]))
    x = x.to(DEV).to(dt)
    c = api.filter_dwt1d(x, levels, h)
    xh = x.double().cpu().numpy()
    ref = oracle.filter_dwt1d(xh, levels, np.array(h))
    what = f"{name} dwt {rows}x{n} L{levels}"
    assert_close(c, ref, dt, what)
    # every band on its own, against the scale of the signal it came from
    assert_bands_close_1d(c, ref, approximations(xh, levels, h), levels, dt, what)
    y = api.filter_idwt1d(c, levels, h)
    yref = oracle.filter_idwt1d(c.double().cpu().numpy(), levels, np.array(h))
    assert_close(y, yref, dt, f"{name} idwt {rows}x{n} L{levels}")
    assert_close(y, xh, dt, f"{name} round trip {rows}x{n} L{levels}")


def test_filter_rejections():
    lib = _lib.load()
    x = torch.zeros(2, 96, device=DEV)
    y = torch.zeros_like(x)
    st = torch.cuda.current_stream().cuda_stream
    h4 = (ctypes.c_double * 4)(*TAPS["d4"])
    assert lib.haar_filter_dwt_1d(x.data_ptr(), y.data_ptr(), 0, 2, 96, 6, h4, 4, st) \
        == _lib.HAAR_ESHAPE
    assert lib.haar_filter_dwt_1d(x.data_ptr(), y.data_ptr(), 0, 2, 96, 1, h4, 3, st) \
        == _lib.HAAR_EINVAL
    assert lib.haar_filter_dwt_1d(x.data_ptr(), x.data_ptr(), 0, 2, 96, 1, h4, 4, st) \
        == _lib.HAAR_EALIAS
    assert lib.haar_filter_dwt_1d(x.data_ptr(), y.data_ptr(), 0, 2, 96, 11, h4, 4, st) \
        == _lib.HAAR_EINVAL


@pytest.mark.parametrize("name", ["d4", "lattice8"])
def test_filter_bank_full_size_rows(name):
    """The benchmark's shape (64 signals of 2^20 fp32 samples, 8 levels: 256
    or 128 chunks per row, every chunk seam and the deepest halo): two whole
    rows against the oracle, coefficient by coefficient and through the
    inverse, and the round trip of every row."""
    h = TAPS[name]
    rows, n, levels = 64, 1 << 20, 8
    base = torch.from_numpy(np.stack([synth.signal_1d(n, seed=7, index=i) for i in range(4)]))
    x = base.to(DEV).float().repeat(rows // 4, 1)
    x[5] *= -0.5  # rows 5 and 62 differ from the repeated ones
    x[62] = torch.flip(x[62], [0])
    c = api.filter_dwt1d(x, levels, h)
    y = api.filter_idwt1d(c, levels, h)
    for r in (5, 62):
        xr = x[r].double().cpu().numpy()
        ref = oracle.filter_dwt1d(xr[None], levels, np.array(h))[0]
        assert_close(c[r], ref, torch.float32, f"{name} full-size row {r}")
        assert_bands_close_1d(c[r], ref, approximations(xr, levels, h), levels, torch.float32,
                              f"{name} full-size row {r}")
        yref = oracle.filter_idwt1d(c[r].double().cpu().numpy()[None], levels, np.array(h))[0]
        assert_close(y[r], yref, torch.float32, f"{name} full-size inverse row {r}")
    err = torch.linalg.vector_norm((y - x).double(), dim=1) / torch.linalg.vector_norm(x.double(), dim=1)
    assert float(err.max()) <= 1e-6
