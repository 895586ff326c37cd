"""Out-of-bounds write checks without a sanitizer: every output is a view
into a larger buffer whose other elements hold a sentinel bit pattern, and
after the call every sentinel must be intact (guard zones before and after
the view, and the gaps between rows of strided views)."""
import numpy as np
import pytest
import torch

from paper_1002_2184_gb300 import api, synth
from test_oracle_pins import lattice_lowpass

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
PAD = 4096  # guard elements on each side (keeps 16-byte alignment for every dtype)

_BITS = {torch.float32: torch.int32, torch.float64: torch.int64,
         torch.bfloat16: torch.int16, torch.float16: torch.int16}
_SENT = {torch.float32: 0x7FC0DEAD, torch.float64: 0x7FF8DEADBEEF0001,
         torch.bfloat16: 0x7FDE, torch.float16: 0x7DEA}


def guarded(shape, dtype, row_gap=0):
    """(buffer, view): the view has the given shape (rows padded by row_gap
    elements) and sits PAD elements into a buffer full of the sentinel."""
    shape = tuple(shape)
    rows = int(np.prod(shape[:-1])) if len(shape) > 1 else 1
    w = shape[-1]
    rs = w + row_gap
    n = rows * rs
    buf = torch.empty(n + 2 * PAD, dtype=dtype, device=DEV)
    buf.view(_BITS[dtype]).fill_(_SENT[dtype])
    view = buf[PAD:PAD + n].view(*shape[:-1], rs)[..., :w]
    return buf, view


def intact(buf, view, dtype):
    """True if every element of buf outside the view still holds the sentinel."""
    mask = torch.ones(buf.numel(), dtype=torch.bool, device=DEV)
    idx = torch.arange(view.numel(), device=DEV).view(view.shape)
    # element offsets of the view inside buf
    offs = view.storage_offset() - buf.storage_offset()
    strides = torch.tensor(view.stride(), device=DEV)
    coords = torch.stack(torch.unravel_index(idx.flatten(), view.shape), dim=1)
    mask[offs + (coords * strides).sum(1)] = False
    bits = buf.view(_BITS[dtype])[mask]
    return bool((bits == _SENT[dtype]).all())


def images(b, h, w, seed=0):
    return torch.from_numpy(np.stack([synth.piecewise_smooth_image(h, w, seed=seed, index=i)
                                      for i in range(b)])).to(DEV)


@pytest.mark.parametrize("b,h,w,levels,gap", [(2, 64, 128, 3, 0),   # warp kernels
                                              (1, 48, 40, 3, 0),    # tile kernels
                                              (1, 48, 36, 2, 0),    # scalar tile kernels
                                              (2, 64, 256, 5, 32),  # strided rows
                                              (1, 256, 512, 8, 0)])  # chained passes
@pytest.mark.parametrize("dt", [torch.float32, torch.bfloat16])
def test_2d_writes_stay_inside(b, h, w, levels, gap, dt):
    x = images(b, h, w, seed=h + w).to(dt)
    cb, c = guarded((b, h, w), dt, gap)
    api.dwt2d(x, levels, out=c)
    yb, y = guarded((b, h, w), dt, gap)
    api.idwt2d(c, levels, out=y)
    torch.cuda.synchronize()
    assert intact(cb, c, dt) and intact(yb, y, dt)


@pytest.mark.parametrize("rows,n,levels", [(3, 4096, 8), (2, 96, 5), (4, 2560, 9)])
def test_1d_writes_stay_inside(rows, n, levels):
    x = torch.from_numpy(np.stack([synth.signal_1d(n, seed=n, index=i)
                                   for i in range(rows)]).astype(np.float32)).to(DEV)
    cb, c = guarded((rows, n), torch.float32)
    api.dwt1d(x, levels, out=c)
    yb, y = guarded((rows, n), torch.float32)
    api.idwt1d(c, levels, out=y)
    db, dn = guarded((rows, n), torch.float32)
    if n % 256 == 0 and levels <= 8:
        api.denoise1d(x, levels, 0.5, out=dn)
    else:
        dn.copy_(x)
    torch.cuda.synchronize()
    assert intact(cb, c, torch.float32) and intact(yb, y, torch.float32)
    assert intact(db, dn, torch.float32)


@pytest.mark.parametrize("shape,levels", [((1, 16, 16, 64), 2), ((1, 24, 40, 72), 3),
                                          ((2, 8, 8, 64), 3),
                                          # the generic per-level path
                                          ((1, 8, 8, 12), 2), ((2, 16, 12, 20), 2)])
def test_3d_writes_stay_inside(shape, levels):
    x = torch.rand(shape, device=DEV)
    cb, c = guarded(shape, torch.float32)
    api.dwt3d(x, levels, out=c)
    yb, y = guarded(shape, torch.float32)
    api.idwt3d(c, levels, out=y)
    torch.cuda.synchronize()
    assert intact(cb, c, torch.float32) and intact(yb, y, torch.float32)


@pytest.mark.parametrize("K", [2, 4, 8])
def test_filter_and_undecimated_writes_stay_inside(K):
    taps = {2: api.HAAR2, 4: api.DAUBECHIES4,
            8: tuple(lattice_lowpass([0.2, 0.5, -0.4, 0.9]))}[K]
    x = torch.rand(3, 6144, device=DEV)
    cb, c = guarded((3, 6144), torch.float32)
    api.filter_dwt1d(x, 4, taps, out=c)
    yb, y = guarded((3, 6144), torch.float32)
    api.filter_idwt1d(c, 4, taps, out=y)
    ub, u = guarded((3, 4, 6144), torch.float32)
    api.swt1d(x, 3, out=u)
    vb, v = guarded((3, 6144), torch.float32)
    api.iswt1d(u, 3, out=v)
    torch.cuda.synchronize()
    for buf, view in ((cb, c), (yb, y), (ub, u), (vb, v)):
        assert intact(buf, view, torch.float32)


def test_shrinkage_2d_writes_stay_inside():
    x = images(2, 64, 256, seed=3).float()
    yb, y = guarded((2, 64, 256), torch.float32, 16)
    api.denoise2d(x, 5, 0.05, out=y)
    torch.cuda.synchronize()
    assert intact(yb, y, torch.float32)


def test_ragged_writes_stay_inside():
    items = [(64, 128, 3), (192, 64, 6), (128, 320, 4), (64, 64, 6)]
    plan = api.RaggedPlan(items, DEV)
    x = plan.empty()
    x.uniform_()
    cb = torch.empty(plan.numel + 2 * PAD, device=DEV)
    cb.view(torch.int32).fill_(_SENT[torch.float32])
    c = cb[PAD:PAD + plan.numel]
    plan.dwt(x, c)
    yb = torch.empty_like(cb)
    yb.view(torch.int32).fill_(_SENT[torch.float32])
    y = yb[PAD:PAD + plan.numel]
    plan.idwt(c, y)
    torch.cuda.synchronize()
    assert plan.status() == 0
    for buf in (cb, yb):
        bits = buf.view(torch.int32)
        assert bool((bits[:PAD] == _SENT[torch.float32]).all())
        assert bool((bits[PAD + plan.numel:] == _SENT[torch.float32]).all())
    assert float((y - x).abs().max()) <= 1e-5
