"""haar_dwt_2d_noalloc: the 2D analysis for callers that cannot allocate
device memory (its scratch lives in a fixed array inside the library).

Checked through the C ABI against haar_dwt_2d with a caller-provided
workspace, on two calls in a row (the second sees the first call's leftover
scratch contents).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1002_2184_gb300 import _lib, api, synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)
SCRATCH_BYTES = 4 << 20


def _images(batch, h, w, seed):
    return torch.from_numpy(np.stack([
        synth.piecewise_smooth_image(h, w, seed=seed, index=i) for i in range(batch)
    ]).astype(np.float32)).to(DEV)


def _reference(x, levels):
    """haar_dwt_2d with a workspace the test allocates."""
    lib = _lib.load()
    c = torch.empty_like(x)
    dx, dc = api.describe(x), api.describe(c)
    n = api.workspace_size(_lib.HAAR_OP_DWT_2D, dx, levels)
    ws = torch.empty(max(n, 1), dtype=torch.uint8, device=DEV)
    rc = lib.haar_dwt_2d(ctypes.byref(dx), ctypes.byref(dc), levels, ws.data_ptr(), n,
                         torch.cuda.current_stream(DEV).cuda_stream)
    assert rc == 0
    return c, n


def _noalloc(x, levels):
    lib = _lib.load()
    c = torch.full_like(x, float("nan"))
    dx, dc = api.describe(x), api.describe(c)
    rc = lib.haar_dwt_2d_noalloc(ctypes.byref(dx), ctypes.byref(dc), levels,
                                 torch.cuda.current_stream(DEV).cuda_stream)
    return rc, c


def test_noalloc_matches_workspace_entry_point_twice():
    # 10 levels on 2 x 2048 x 2048: six fused, then four more through scratch
    levels = 10
    for call, seed in enumerate((11, 12)):
        x = _images(2, 2048, 2048, seed)
        ref, need = _reference(x, levels)
        assert 0 < need <= SCRATCH_BYTES
        rc, c = _noalloc(x, levels)
        assert rc == _lib.HAAR_OK, f"call {call}: status {rc}"
        torch.cuda.synchronize()
        err = float(torch.linalg.vector_norm((c - ref).double()) /
                    torch.linalg.vector_norm(ref.double()))
        assert err <= 1e-6, f"call {call}: rel-L2 {err:.3e}"
        assert torch.isfinite(c).all()


def test_noalloc_shallow_and_oversized():
    # six levels need no scratch at all
    x = _images(1, 256, 512, 3)
    ref, need = _reference(x, 6)
    assert need == 0
    rc, c = _noalloc(x, 6)
    assert rc == _lib.HAAR_OK
    torch.cuda.synchronize()
    assert torch.equal(c, ref)
    # a transform whose scratch exceeds the built-in array is refused before
    # any device work (descriptors only; the pointers are never touched)
    big = _lib.desc(1 << 40, _lib.HAAR_F32, 1, 1 << 17, 1 << 17, 1 << 34, 1 << 17)
    out = _lib.desc(1 << 41, _lib.HAAR_F32, 1, 1 << 17, 1 << 17, 1 << 34, 1 << 17)
    n = api.workspace_size(_lib.HAAR_OP_DWT_2D, big, 7)
    assert n > SCRATCH_BYTES
    rc = _lib.load().haar_dwt_2d_noalloc(ctypes.byref(big), ctypes.byref(out), 7, None)
    assert rc == _lib.HAAR_EWORKSPACE
