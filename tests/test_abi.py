"""The C ABI library loads and exports every entry point its header declares,
and rejects bad arguments on the host before any device work (no GPU needed:
these calls fail validation, so nothing is launched)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "fasthaar.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(haar_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1002_2184_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("haar_dwt_1d", "haar_idwt_1d", "haar_dwt_2d", "haar_idwt_2d",
              "haar_workspace_size", "haar_status_string"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_1002_2184_gb300 import _lib
    assert set(declared_functions()) <= set(_lib.SIGNATURES)


def test_version_and_strings(lib):
    assert lib.haar_version() == 1
    for s in range(0, -8, -1):
        assert lib.haar_status_string(s) not in (None, b"", b"unknown status")
    assert lib.haar_status_string(-99) == b"unknown status"


# ---------------------------------------------------------------------------
# Host-side validation (T11).  Fake, never-dereferenced device addresses.
# ---------------------------------------------------------------------------
A = 1 << 40          # fake device address, 256-byte aligned
B = A + (1 << 30)    # far away from A


def d(ptr, dt=0, b=1, h=8, w=8, bs=None, rs=None):
    from paper_1002_2184_gb300 import _lib
    rs = w if rs is None else rs
    bs = h * rs if bs is None else bs
    return _lib.desc(ptr, dt, b, h, w, bs, rs)


def call(lib, name, src, dst, levels, ws=None, wsb=0):
    return getattr(lib, name)(ctypes.byref(src), ctypes.byref(dst), levels, ws, wsb, None)


@pytest.mark.parametrize("name", ["haar_dwt_2d", "haar_idwt_2d", "haar_dwt_1d", "haar_idwt_1d"])
def test_rejections(lib, name):
    from paper_1002_2184_gb300 import _lib as L
    two_d = name.endswith("2d")
    # level count
    assert call(lib, name, d(A), d(B), 0) == L.HAAR_EINVAL
    assert call(lib, name, d(A), d(B), 63) == L.HAAR_EINVAL
    # not divisible by 2^levels
    assert call(lib, name, d(A, w=12), d(B, w=12), 3) == L.HAAR_ESHAPE
    if two_d:
        assert call(lib, name, d(A, h=12), d(B, h=12), 3) == L.HAAR_ESHAPE
    # null pointer with data
    assert call(lib, name, d(0), d(B), 1) == L.HAAR_EINVAL
    # shape mismatch
    assert call(lib, name, d(A), d(B, w=16), 1) == L.HAAR_EINVAL
    # overlapping input and output
    assert call(lib, name, d(A), d(A + 16), 1) == L.HAAR_EALIAS
    # negative or too-small strides
    assert call(lib, name, d(A, rs=4), d(B), 1) == L.HAAR_EINVAL
    assert call(lib, name, d(A, b=2, bs=8), d(B, b=2), 1) == L.HAAR_EINVAL
    # reserved field
    bad = d(A)
    bad.reserved = 1
    assert call(lib, name, bad, d(B), 1) == L.HAAR_EINVAL
    # unknown dtype
    assert call(lib, name, d(A, dt=9), d(B), 1) == L.HAAR_EDTYPE
    # fp64 only pairs with fp64
    assert call(lib, name, d(A, dt=4), d(B, dt=0), 1) == L.HAAR_EDTYPE
    # uint8 is never an output
    assert call(lib, name, d(A), d(B, dt=3), 1) == L.HAAR_EDTYPE
    # empty input: nothing to do, success without touching the device
    assert call(lib, name, d(A, b=0), d(B, b=0), 3) == L.HAAR_OK
    assert call(lib, name, d(0, h=0), d(0, h=0), 3) == L.HAAR_OK


def test_uint8_only_as_analysis_input(lib):
    from paper_1002_2184_gb300 import _lib as L
    assert call(lib, "haar_idwt_2d", d(A, dt=3), d(B), 1) == L.HAAR_EDTYPE
    assert call(lib, "haar_idwt_1d", d(A, dt=3), d(B), 1) == L.HAAR_EDTYPE


def test_workspace_sizes(lib):
    from paper_1002_2184_gb300 import _lib as L
    n = ctypes.c_size_t()
    src = d(A, h=4096, w=4096)
    for op in (L.HAAR_OP_DWT_2D, L.HAAR_OP_IDWT_2D):
        assert lib.haar_workspace_size(op, ctypes.byref(src), 6, ctypes.byref(n)) == 0
        assert n.value == 0  # six levels fuse into one launch
        assert lib.haar_workspace_size(op, ctypes.byref(src), 7, ctypes.byref(n)) == 0
        assert n.value == 64 * 64 * 4  # LL after 6 levels, fp32
    src1 = d(A, h=3, w=1 << 20)
    assert lib.haar_workspace_size(L.HAAR_OP_DWT_1D, ctypes.byref(src1), 12,
                                   ctypes.byref(n)) == 0 and n.value == 0
    assert lib.haar_workspace_size(L.HAAR_OP_DWT_1D, ctypes.byref(src1), 20,
                                   ctypes.byref(n)) == 0 and n.value == 3 * 256 * 4
    # a deep transform refuses a missing or short workspace
    assert call(lib, "haar_dwt_2d", src, d(B, h=4096, w=4096), 7) == L.HAAR_EWORKSPACE
    assert call(lib, "haar_dwt_2d", src, d(B, h=4096, w=4096), 7,
                ws=1 << 41, wsb=100) == L.HAAR_EWORKSPACE
    assert lib.haar_workspace_size(9, ctypes.byref(src), 1, ctypes.byref(n)) == L.HAAR_EINVAL


# ---------------------------------------------------------------------------
# Ragged plans: host-only validation (no device call is made by these).
# ---------------------------------------------------------------------------
def _items(spec):
    from paper_1002_2184_gb300 import _lib as L
    arr = (L.HaarRaggedItem * max(1, len(spec)))()
    off = 0
    for i, (h, w, lv) in enumerate(spec):
        arr[i] = L.HaarRaggedItem(off, off, h, w, w, w, lv, 0)
        off += h * w
    return arr


def _create(lib, spec, unit=0, bps=4):
    h = ctypes.c_void_p()
    rc = lib.haar_ragged_plan_create(_items(spec), len(spec), unit, bps, ctypes.byref(h))
    return rc, h


def test_ragged_plan_validation(lib):
    from paper_1002_2184_gb300 import _lib as L
    assert _create(lib, [(48, 64, 3)])[0] == L.HAAR_ESHAPE        # 48 % 32 != 0
    assert _create(lib, [(64, 64, 7)])[0] == L.HAAR_EINVAL        # more than 6 levels
    assert _create(lib, [(64, 64, 0)])[0] == L.HAAR_EINVAL
    assert _create(lib, [(96, 64, 6)])[0] == L.HAAR_ESHAPE        # 96 % 64 != 0
    assert _create(lib, [(64, 64, 6)], unit=1)[0] == L.HAAR_ESHAPE  # 6 levels need 64 rows
    for unit in (0, 2, 3):                                            # units of >= 64 rows
        rc, h = _create(lib, [(64, 64, 6)], unit=unit)
        assert rc == L.HAAR_OK
        lib.haar_ragged_plan_destroy(h)
    assert _create(lib, [(64, 64, 3)], unit=7)[0] == L.HAAR_EINVAL
    assert _create(lib, [(64, 64, 3)], unit=4)[0] == L.HAAR_EINVAL
    assert _create(lib, [(64, 64, 3)], bps=0)[0] == L.HAAR_EINVAL
    bad = _items([(64, 64, 3)])
    bad[0].in_row_stride = 32
    assert lib.haar_ragged_plan_create(bad, 1, 0, 4, ctypes.byref(ctypes.c_void_p())) \
        == L.HAAR_EINVAL


def test_ragged_plan_geometry(lib):
    from paper_1002_2184_gb300 import _lib as L
    spec = [(64, 128, 6), (64, 64, 3), (128, 256, 5), (32, 32, 1)]
    rc, h = _create(lib, spec)
    assert rc == L.HAAR_OK
    units, px = ctypes.c_int64(), ctypes.c_int64()
    assert lib.haar_ragged_plan_info(h, ctypes.byref(units), ctypes.byref(px), None) == 0
    # 64 x 128 units: 1 + 1 + 2*2 + 1
    assert units.value == 7
    assert px.value == sum(a * b for a, b, _ in spec)
    n = ctypes.c_size_t()
    assert lib.haar_ragged_workspace_size(h, ctypes.byref(n)) == 0
    assert n.value >= 256 + 64 * len(spec) and n.value % 256 == 0
    # argument checks that run before any device work
    A, B = 1 << 40, 1 << 41
    assert lib.haar_dwt_2d_ragged(h, A, 0, B, 3, 1 << 42, n.value, None) == L.HAAR_EDTYPE
    assert lib.haar_idwt_2d_ragged(h, A, 3, B, 0, 1 << 42, n.value, None) == L.HAAR_EDTYPE
    assert lib.haar_dwt_2d_ragged(h, A, 0, B, 0, None, n.value, None) == L.HAAR_EWORKSPACE
    assert lib.haar_dwt_2d_ragged(h, A, 0, B, 0, 1 << 42, 8, None) == L.HAAR_EWORKSPACE
    assert lib.haar_dwt_2d_ragged(h, A + 4, 0, B, 0, 1 << 42, n.value, None) == L.HAAR_EINVAL
    assert lib.haar_dwt_2d_ragged(h, A, 0, A + 1024, 0, 1 << 42, n.value, None) == L.HAAR_EALIAS
    assert lib.haar_dwt_2d_ragged(h, None, 0, B, 0, 1 << 42, n.value, None) == L.HAAR_EINVAL
    assert lib.haar_ragged_plan_destroy(h) == 0
    rc, h0 = _create(lib, [])
    assert rc == 0
    assert lib.haar_dwt_2d_ragged(h0, None, 0, None, 0, None, 0, None) == 0  # nothing to do
    lib.haar_ragged_plan_destroy(h0)


@pytest.mark.parametrize("unit,expect", [(1, 2 + 2 + 4 * 1 + 1),   # 32 x 256 (5 levels max)
                                         (2, 2 + 1 + 2 * 4 + 1),   # 64 x 64
                                         (3, 1 + 1 + 1 * 2 + 1)])  # 128 x 128
def test_ragged_unit_counts(lib, unit, expect):
    """Each image is cut into ceil(h / UH) x ceil(w / UW) units."""
    spec = [(64, 128, 5), (64, 64, 3), (128, 256, 5), (32, 32, 1)]
    rc, h = _create(lib, spec, unit=unit)
    assert rc == 0
    units = ctypes.c_int64()
    assert lib.haar_ragged_plan_info(h, ctypes.byref(units), None, None) == 0
    assert units.value == expect
    lib.haar_ragged_plan_destroy(h)


# ---------------------------------------------------------------------------
# The other entry points: every case below is refused by the host-side
# checks before anything is launched (fake device addresses, never touched).
# ---------------------------------------------------------------------------
def test_filter_bank_rejections(lib):
    from paper_1002_2184_gb300 import _lib as L
    h4 = (ctypes.c_double * 4)(0.48, 0.84, 0.22, -0.13)
    for fn in (lib.haar_filter_dwt_1d, lib.haar_filter_idwt_1d):
        assert fn(A, B, 2, 1, 64, 1, h4, 4, None) == L.HAAR_EDTYPE      # bf16: fp32/fp64 only
        assert fn(A, B, 0, 1, 64, 0, h4, 4, None) == L.HAAR_EINVAL      # levels < 1
        assert fn(A, B, 0, 1, 64, 11, h4, 4, None) == L.HAAR_EINVAL     # levels > 10
        assert fn(A, B, 0, 1, 64, 1, h4, 3, None) == L.HAAR_EINVAL      # odd tap count
        assert fn(A, B, 0, 1, 64, 1, None, 4, None) == L.HAAR_EINVAL    # no filter
        assert fn(0, B, 0, 1, 64, 1, h4, 4, None) == L.HAAR_EINVAL      # null with data
        assert fn(A, B, 0, 1, 96, 6, h4, 4, None) == L.HAAR_ESHAPE      # 96 % 64 != 0
        assert fn(A, A + 64, 0, 2, 64, 1, h4, 4, None) == L.HAAR_EALIAS
        assert fn(A, B, 0, 0, 64, 1, h4, 4, None) == L.HAAR_OK          # nothing to do


def test_undecimated_rejections(lib):
    from paper_1002_2184_gb300 import _lib as L
    for fn in (lib.haar_swt_1d, lib.haar_iswt_1d):
        assert fn(A, B, 3, 1, 64, 1, None) == L.HAAR_EDTYPE             # u8
        assert fn(A, B, 0, 1, 64, 0, None) == L.HAAR_EINVAL
        assert fn(A, B, 0, 1, 64, 11, None) == L.HAAR_EINVAL
        assert fn(A, B, 0, 1, 8, 4, None) == L.HAAR_ESHAPE              # n < 2^levels
        assert fn(0, B, 0, 1, 64, 1, None) == L.HAAR_EINVAL
        assert fn(A, A + 64, 0, 1, 64, 1, None) == L.HAAR_EALIAS        # (L+1) rows overlap
        assert fn(A, B, 0, 0, 64, 1, None) == L.HAAR_OK


@pytest.mark.parametrize("name,two_d", [("haar_denoise_1d", False), ("haar_denoise_2d", True)])
def test_shrinkage_rejections(lib, name, two_d):
    from paper_1002_2184_gb300 import _lib as L
    fn = getattr(lib, name)
    h = 64 if two_d else 1
    x, y = d(A, h=h, w=256), d(B, h=h, w=256)

    def run(xd, yd, levels=2, t=0.1, mode=L.HAAR_THRESH_SOFT):
        return fn(ctypes.byref(xd), ctypes.byref(yd), levels, ctypes.c_double(t), mode, None)

    assert run(x, y, mode=7) == L.HAAR_EINVAL
    assert run(x, y, t=-1.0) == L.HAAR_EINVAL
    assert run(x, y, t=float("nan")) == L.HAAR_EINVAL
    assert run(x, y, levels=0) == L.HAAR_EINVAL
    assert run(x, y, levels=6 if two_d else 9) == L.HAAR_EINVAL       # beyond the fused depth
    assert run(d(A, dt=2, h=h, w=256), d(B, dt=2, h=h, w=256)) == L.HAAR_EDTYPE
    assert run(x, d(B, dt=4, h=h, w=256)) == L.HAAR_EDTYPE            # mixed dtypes
    bad_w = 80 if two_d else 96  # 2D rows in multiples of 32, 1D in multiples of 256
    assert run(d(A, h=h, w=bad_w), d(B, h=h, w=bad_w)) == L.HAAR_ESHAPE
    assert run(x, d(A + 64, h=h, w=256)) == L.HAAR_EALIAS
    assert run(d(A, b=0, h=h, w=256), d(B, b=0, h=h, w=256)) == L.HAAR_OK


def test_volume_rejections(lib):
    from paper_1002_2184_gb300 import _lib as L

    def v(ptr, dt=0, b=1, dd=16, h=16, w=64, bs=None, zs=None, rs=None):
        rs = w if rs is None else rs
        zs = h * rs if zs is None else zs
        bs = dd * zs if bs is None else bs
        return L.HaarDesc3(ptr, dt, 0, b, dd, h, w, bs, zs, rs)

    def run(fn, s, t, levels):
        return fn(ctypes.byref(s), ctypes.byref(t), levels, None, 0, None)

    for fn in (lib.haar_dwt_3d, lib.haar_idwt_3d):
        assert run(fn, v(A), v(B), 0) == L.HAAR_EINVAL
        assert run(fn, v(A), v(B), 31) == L.HAAR_EINVAL
        assert run(fn, v(A, dd=12), v(B, dd=12), 3) == L.HAAR_ESHAPE     # depth % 8
        assert run(fn, v(A), v(B, w=32), 1) == L.HAAR_EINVAL             # shapes differ
        assert run(fn, v(A, dt=4), v(B, dt=0), 1) == L.HAAR_EDTYPE       # fp64 only with fp64
        assert run(fn, v(A), v(A + 256), 1) == L.HAAR_EALIAS
        assert run(fn, v(0), v(B), 1) == L.HAAR_EINVAL
        assert run(fn, v(A, rs=32), v(B), 1) == L.HAAR_EINVAL            # row stride < w
        assert run(fn, v(A), v(B), 4) == L.HAAR_EWORKSPACE               # deep: needs scratch
        assert run(fn, v(A, b=0), v(B, b=0), 2) == L.HAAR_OK
        assert run(fn, v(A, w=12), v(B, w=12), 2) == L.HAAR_EWORKSPACE   # generic: low bands
    # the workspace of the generic path: the low band of every level but the last
    n = ctypes.c_size_t()
    assert lib.haar_workspace_size_3d(ctypes.byref(v(A, w=12)), 2, ctypes.byref(n)) == 0
    assert n.value == ((1 * 8 * 8 * 6 * 4 + 255) // 256) * 256
    assert lib.haar_workspace_size_3d(ctypes.byref(v(A)), 3, ctypes.byref(n)) == 0
    assert n.value == 0  # three levels fuse in one tiled pass


def test_noalloc_validates_both_descriptors_before_the_scratch_size(lib):
    """The allocation-free 2D analysis reports a bad output descriptor as
    such even when the input is too large for its built-in scratch; only a
    valid call gets HAAR_EWORKSPACE.  No device work: every call fails
    validation."""
    from paper_1002_2184_gb300 import _lib as L

    def noalloc(src, dst, levels):
        return lib.haar_dwt_2d_noalloc(ctypes.byref(src), ctypes.byref(dst), levels, None)

    n = 1 << 17  # 2^34 pixels: 7 levels need far more than the built-in 4 MiB
    big = d(A, h=n, w=n)
    far = 1 << 44
    assert noalloc(big, d(far, h=n, w=n // 2), 7) == L.HAAR_EINVAL      # shape mismatch
    assert noalloc(big, d(far, dt=3, h=n, w=n), 7) == L.HAAR_EDTYPE     # uint8 output
    assert noalloc(big, d(A + 64, h=n, w=n), 7) == L.HAAR_EALIAS        # overlapping output
    assert noalloc(big, d(far, h=n, w=n), 0) == L.HAAR_EINVAL           # level count
    assert noalloc(big, d(far, h=n, w=n), 7) == L.HAAR_EWORKSPACE       # valid, too large
    assert noalloc(d(A, b=0), d(B, b=0), 3) == L.HAAR_OK                # empty: nothing to do
