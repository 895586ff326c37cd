"""Arrays beyond 2^31 elements (int64 offsets everywhere).  The oracle cannot
take these sizes, so sampled outputs are checked against values computed on
the host from their definition: in 2D the level-l coefficients of a block
are the 2x2 butterfly of four level-(l-1) low-pass values, each the sum of
its 2^(l-1) x 2^(l-1) input block divided by 2^(l-1); in 1D the pair
formulas applied level by level.  The round trip is checked on sampled rows
near the end of the array."""
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


def _free_gb():
    free, _ = torch.cuda.mem_get_info(DEV)
    return free / 2**30


def _seeded(shape, seed):
    g = torch.Generator(device=DEV)
    g.manual_seed(seed)
    return torch.rand(shape, generator=g, device=DEV, dtype=torch.float32)


def _ll(block: np.ndarray, l: int) -> float:
    """Level-l low-pass of a 2^l x 2^l block: its sum / 2^l."""
    return float(block.sum()) / 2.0 ** l


@pytest.mark.parametrize("h,w,L", [(32768, 65552, 2),   # w % 32 != 0: the tile kernels
                                   (32800, 65536, 2)])  # both % 32 == 0: the warp kernels
def test_image_beyond_2_31_pixels(h, w, L):
    from paper_1002_2184_gb300 import api
    assert h * w > 2 ** 31
    if _free_gb() < 3 * h * w * 4 / 2**30 + 2:
        pytest.skip("needs ~26 GB of free device memory")
    x = _seeded((h, w), 11)
    c = api.dwt2d(x, L)
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    h1, w1, h2, w2 = h // 2, w // 2, h // 4, w // 4
    # level 2 (and LL2) at sampled block positions, biased to the end of the array
    for _ in range(24):
        i = int(rng.integers(h2 - 64, h2)) if rng.random() < 0.7 else int(rng.integers(0, h2))
        j = int(rng.integers(0, w2))
        blk = x[4 * i:4 * i + 4, 4 * j:4 * j + 4].double().cpu().numpy()
        a, b = _ll(blk[:2, :2], 1), _ll(blk[:2, 2:], 1)
        cc, d = _ll(blk[2:, :2], 1), _ll(blk[2:, 2:], 1)
        want = {"ll": (a + b + cc + d) / 2, "hx": (b - a + d - cc) / 2,
                "hy": (cc + d - a - b) / 2, "hh": (a - b - cc + d) / 2}
        got = {"ll": c[i, j], "hx": c[i, w2 + j], "hy": c[h2 + i, j], "hh": c[h2 + i, w2 + j]}
        for k in want:
            assert abs(float(got[k]) - want[k]) <= 1e-5 * max(1.0, abs(want[k])), (k, i, j)
    # level 1 details at sampled positions
    for _ in range(24):
        i = int(rng.integers(h1 - 32, h1))
        j = int(rng.integers(0, w1))
        a, b = float(x[2 * i, 2 * j]), float(x[2 * i, 2 * j + 1])
        cc, d = float(x[2 * i + 1, 2 * j]), float(x[2 * i + 1, 2 * j + 1])
        assert abs(float(c[i, w1 + j]) - (b - a + d - cc) / 2) <= 1e-6
        assert abs(float(c[h1 + i, j]) - (cc + d - a - b) / 2) <= 1e-6
        assert abs(float(c[h1 + i, w1 + j]) - (a - b - cc + d) / 2) <= 1e-6
    y = api.idwt2d(c, L)
    del c
    torch.cuda.synchronize()
    rows = [0, h // 2, h - 4, h - 1]
    err = max(float((y[r] - x[r]).abs().max()) for r in rows)
    assert err <= 1e-5


def test_signals_beyond_2_31_samples():
    from paper_1002_2184_gb300 import api
    rows, n, L = 2048, 1048640, 3  # 2,147,614,720 samples > 2^31; n % 64 == 0, not % 256
    if _free_gb() < 3 * rows * n * 4 / 2**30 + 2:
        pytest.skip("needs ~26 GB of free device memory")
    x = _seeded((rows, n), 12)
    c = api.dwt1d(x, L)
    torch.cuda.synchronize()
    s = 1.0 / math.sqrt(2.0)
    rng = np.random.default_rng(6)
    for _ in range(24):
        r = int(rng.integers(rows - 4, rows))
        k = int(rng.integers(0, n >> L))
        seg = x[r, k << L:(k + 1) << L].double().cpu().numpy()
        a = seg
        details = []
        for l in range(1, L + 1):
            lo = (a[0::2] + a[1::2]) * s
            hi = (a[1::2] - a[0::2]) * s
            details.append(hi)
            a = lo
        assert abs(float(c[r, k]) - a[0]) <= 1e-5
        for l in range(1, L + 1):
            m = 1 << (L - l)  # details of level l inside this segment
            got = c[r, (n >> l) + k * m:(n >> l) + (k + 1) * m].double().cpu().numpy()
            assert np.allclose(got, details[l - 1], atol=1e-5), (r, k, l)
    y = api.idwt1d(c, L)
    del c
    torch.cuda.synchronize()
    err = max(float((y[r] - x[r]).abs().max()) for r in (0, rows // 2, rows - 1))
    assert err <= 1e-5


def test_volume_beyond_2_31_voxels():
    from paper_1002_2184_gb300 import api
    side = 1280  # 2,097,152,000 voxels < 2^31; with a batch of 2: 4.19e9 > 2^31
    if _free_gb() < 3 * 2 * side ** 3 * 4 / 2**30 + 2:
        pytest.skip("needs ~50 GB of free device memory")
    x = _seeded((2, side, side, side), 13)
    c = api.dwt3d(x, 1)
    torch.cuda.synchronize()
    s = 1.0 / math.sqrt(2.0)
    hs = side // 2
    rng = np.random.default_rng(7)
    for _ in range(16):
        z, yv, xv = (int(v) for v in rng.integers(hs - 16, hs, size=3))
        blk = x[1, 2 * z:2 * z + 2, 2 * yv:2 * yv + 2, 2 * xv:2 * xv + 2].double().cpu().numpy()
        # octant (bz, by, bx): x and y stages (x 1/2), then z (x 1/sqrt 2)
        for bz in (0, 1):
            for by in (0, 1):
                for bx in (0, 1):
                    sx = np.array([1.0, 1.0]) if bx == 0 else np.array([-1.0, 1.0])
                    sy = np.array([1.0, 1.0]) if by == 0 else np.array([-1.0, 1.0])
                    sz = np.array([1.0, 1.0]) if bz == 0 else np.array([-1.0, 1.0])
                    want = float(np.einsum("zyx,z,y,x->", blk, sz, sy, sx)) * 0.5 * s
                    got = float(c[1, bz * hs + z, by * hs + yv, bx * hs + xv])
                    assert abs(got - want) <= 1e-5, (bz, by, bx, z, yv, xv)
    y = api.idwt3d(c, 1)
    del c
    torch.cuda.synchronize()
    err = float((y[1, -2:] - x[1, -2:]).abs().max())
    assert err <= 1e-5


def test_filter_bank_beyond_2_31_samples():
    """The K-tap bank on 2049 rows of 2^20 samples (2,148,532,224 > 2^31;
    Daubechies-4, 8 levels): the last rows, whose offsets need 64 bits, are
    whole rows the oracle can take, checked coefficient by coefficient and
    through the round trip."""
    import oracle
    from paper_1002_2184_gb300 import api
    rows, n, L = 2049, 1 << 20, 8
    assert rows * n > 2 ** 31
    if _free_gb() < 3 * rows * n * 4 / 2**30 + 2:
        pytest.skip("needs ~26 GB of free device memory")
    h = api.DAUBECHIES4
    x = _seeded((rows, n), 13)
    c = api.filter_dwt1d(x, L, h)
    y = api.filter_idwt1d(c, L, h)
    torch.cuda.synchronize()
    for r in (2047, 2048):
        xr = x[r].double().cpu().numpy()
        ref = oracle.filter_dwt1d(xr[None], L, np.array(h))[0]
        assert oracle.rel_l2(c[r].double().cpu().numpy(), ref) <= 1e-6, r
        assert float((y[r] - x[r]).abs().max()) <= 1e-5, r
