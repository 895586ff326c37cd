"""A seeded sweep of shapes, level counts, storage types and memory layouts
for the 1D and 2D transforms and the K-tap bank, each case against the FP64
oracle element by element (analysis, and synthesis of the GPU's own
coefficients).

The fixed case lists elsewhere pin the kernel families one by one; this sweep
draws the combinations they do not name: batches of 1-3, sides from 2^L to
a few hundred, views whose rows are padded and whose first element is moved
by a vector-keeping or a vector-breaking offset, and coefficient arrays that
are themselves views.  Sizes stay small enough for the oracle to finish in
seconds."""
import numpy as np
import pytest
import torch

import oracle
from paper_1002_2184_gb300 import api
from parity_util import assert_close

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
DTYPES = (torch.float32, torch.bfloat16, torch.float16)


def host64(t: torch.Tensor) -> np.ndarray:
    return t.detach().double().cpu().numpy()


def padded_view(vals: torch.Tensor, off: int, pad: int) -> torch.Tensor:
    """The same values in a buffer whose rows are off + pad elements longer,
    starting `off` elements in: a strided view of the buffer."""
    *lead, w = vals.shape
    buf = torch.zeros(*lead, w + pad + off, dtype=vals.dtype, device=vals.device)
    view = buf[..., off:off + w]
    view.copy_(vals)
    return view


def cases_2d(count=96, seed=20261204):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        L = int(rng.integers(1, 7))
        h = (1 << L) * int(rng.integers(1, 1 + max(1, 256 >> L)))
        w = (1 << L) * int(rng.integers(1, 1 + max(1, 256 >> L)))
        b = int(rng.integers(1, 4))
        dt = DTYPES[int(rng.integers(0, 3))]
        off = int(rng.choice([0, 8, 1]))
        pad = int(rng.choice([0, 8, 24, 3]))
        out.append((i, b, h, w, L, dt, off, pad))
    return out


def cases_1d(count=64, seed=4122026):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        L = int(rng.integers(1, 11))
        n = (1 << L) * int(rng.integers(1, 1 + max(1, 8192 >> L)))
        rows = int(rng.integers(1, 5))
        dt = DTYPES[int(rng.integers(0, 3))]
        off = int(rng.choice([0, 8, 1]))
        pad = int(rng.choice([0, 16, 5]))
        out.append((i, rows, n, L, dt, off, pad))
    return out


@pytest.mark.parametrize("i,b,h,w,L,dt,off,pad", cases_2d())
def test_sweep_2d(i, b, h, w, L, dt, off, pad):
    g = torch.Generator(device="cpu").manual_seed(1000 + i)
    vals = (torch.rand(b, h, w, generator=g, dtype=torch.float64) * 4 - 2).to(dt).to(DEV)
    x = padded_view(vals, off, pad)
    assert x.shape == (b, h, w)
    c = padded_view(torch.zeros(b, h, w, dtype=dt, device=DEV), 8 if off else 0, pad)
    api.dwt2d(x, L, out=c)
    assert_close(c, oracle.dwt2d(host64(x), L), dt, f"sweep 2D analysis {i}")
    y = api.idwt2d(c, L)
    assert_close(y, oracle.idwt2d(host64(c), L), dt, f"sweep 2D synthesis {i}")


@pytest.mark.parametrize("i,rows,n,L,dt,off,pad", cases_1d())
def test_sweep_1d(i, rows, n, L, dt, off, pad):
    g = torch.Generator(device="cpu").manual_seed(2000 + i)
    vals = (torch.rand(rows, n, generator=g, dtype=torch.float64) * 4 - 2).to(dt).to(DEV)
    x = padded_view(vals, off, pad)
    assert x.shape == (rows, n)
    c = api.dwt1d(x, L)
    assert_close(c, oracle.dwt1d(host64(x), L), dt, f"sweep 1D analysis {i}")
    y = padded_view(torch.zeros(rows, n, dtype=dt, device=DEV), off, pad)
    api.idwt1d(c, L, out=y)
    assert_close(y, oracle.idwt1d(host64(c), L), dt, f"sweep 1D synthesis {i}")


def cases_filter(count=48, seed=777):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        K = int(rng.choice([2, 4, 6, 8]))
        L = int(rng.integers(1, 11))
        n = (1 << L) * int(rng.integers(1, 1 + max(1, 20000 >> L)))
        rows = int(rng.integers(1, 4))
        dt = (torch.float32, torch.float64)[int(rng.integers(0, 2))]
        off = int(rng.choice([0, 0, 1, 4]))  # elements; 1 breaks 16-byte alignment
        out.append((i, K, rows, n, L, dt, off))
    return out


@pytest.mark.parametrize("i,K,rows,n,L,dt,off", cases_filter())
def test_sweep_filter_bank(i, K, rows, n, L, dt, off):
    h = api.daubechies(K)
    g = torch.Generator(device="cpu").manual_seed(3000 + i)
    vals = (torch.rand(rows * n, generator=g, dtype=torch.float64) * 4 - 2).to(dt).to(DEV)
    buf = torch.zeros(rows * n + off, dtype=dt, device=DEV)
    x = buf[off:].view(rows, n)
    x.copy_(vals.view(rows, n))
    cbuf = torch.zeros(rows * n + off, dtype=dt, device=DEV)
    c = cbuf[off:].view(rows, n)
    api.filter_dwt1d(x, L, h, out=c)
    ref = oracle.filter_dwt1d(host64(x), L, np.array(h))
    assert_close(c, ref, dt, f"sweep K-tap analysis {i} (K={K})")
    y = api.filter_idwt1d(c, L, h)
    yref = oracle.filter_idwt1d(host64(c), L, np.array(h))
    assert_close(y, yref, dt, f"sweep K-tap synthesis {i} (K={K})")


def cases_3d(count=40, seed=31337):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        L = int(rng.integers(1, 5))
        d, h, w = ((1 << L) * int(rng.integers(1, 1 + max(1, 48 >> L))) for _ in range(3))
        b = int(rng.integers(1, 3))
        dt = DTYPES[int(rng.integers(0, 3))]
        pad = int(rng.choice([0, 8, 3]))  # row padding; 3 breaks the tiled kernels' alignment
        out.append((i, b, d, h, w, L, dt, pad))
    return out


@pytest.mark.parametrize("i,b,d,h,w,L,dt,pad", cases_3d())
def test_sweep_3d(i, b, d, h, w, L, dt, pad):
    """Volumes of every side mix, padded rows (some breaking the tiles'
    alignment, which moves them to the per-level kernels)."""
    g = torch.Generator(device="cpu").manual_seed(4000 + i)
    vals = (torch.rand(b, d, h, w, generator=g, dtype=torch.float64) * 4 - 2).to(dt).to(DEV)
    x = padded_view(vals, 0, pad)
    c = api.dwt3d(x, L)
    assert_close(c, oracle.dwt3d(host64(x), L), dt, f"sweep 3D analysis {i}")
    y = padded_view(torch.zeros(b, d, h, w, dtype=dt, device=DEV), 0, pad)
    api.idwt3d(c, L, out=y)
    assert_close(y, oracle.idwt3d(host64(c), L), dt, f"sweep 3D synthesis {i}")


def cases_shrink(count=40, seed=99):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        two_d = bool(rng.integers(0, 2))
        L = int(rng.integers(1, 6 if two_d else 9))
        if two_d:
            shape = (int(rng.integers(1, 3)), 32 * int(rng.integers(1, 9)),
                     32 * int(rng.integers(1, 9)))
        else:
            shape = (int(rng.integers(1, 5)), 256 * int(rng.integers(1, 17)))
        dt = (torch.float32, torch.float64)[int(rng.integers(0, 2))]
        t = float(rng.choice([0.0, 0.05, 0.3, 1.0]))
        pad = int(rng.choice([0, 8]))  # 16-byte aligned rows, padded or not
        out.append((i, two_d, shape, L, dt, t, pad))
    return out


@pytest.mark.parametrize("i,two_d,shape,L,dt,t,pad", cases_shrink())
def test_sweep_soft_shrinkage(i, two_d, shape, L, dt, t, pad):
    """One-pass soft shrinkage (continuous in the coefficients, so no
    threshold decision to match) against the oracle's analysis, shrink and
    synthesis."""
    g = torch.Generator(device="cpu").manual_seed(5000 + i)
    vals = (torch.rand(*shape, generator=g, dtype=torch.float64) * 4 - 2).to(dt).to(DEV)
    x = padded_view(vals, 0, pad)
    y = padded_view(torch.zeros(*shape, dtype=dt, device=DEV), 0, pad)
    if two_d:
        api.denoise2d(x, L, t, out=y)
        ref = oracle.denoise2d(host64(x), L, t)
    else:
        api.denoise1d(x, L, t, out=y)
        ref = oracle.denoise1d(host64(x), L, t)
    assert_close(y, ref, dt, f"sweep shrinkage {i} ({'2D' if two_d else '1D'}, t={t})")
