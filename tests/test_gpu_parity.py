"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (relative L2 over the whole output, plus an element-wise bound
relative to the largest reference magnitude):
  fp32 storage: rel-L2 <= 1e-6, max-abs <= 4e-6 * max|ref|
  bf16 storage: rel-L2 <= 1e-2, max-abs <= 2^-7 * max|ref|
  fp16 storage: rel-L2 <= 2e-3, max-abs <= 2^-9 * max|ref|
  fp64 storage: rel-L2 <= 1e-13
The oracle always receives exactly the values the GPU read (inputs are cast
to the storage type first, then widened back to float64).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1002_2184_gb300 import api, synth
from parity_util import TOL, assert_close  # noqa: F401  (shared comparison rules)

pytestmark = pytest.mark.gpu

DEV = "cuda"


def dev(a: np.ndarray, dtype) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV).to(dtype)


def host64(t: torch.Tensor) -> np.ndarray:
    return t.detach().double().cpu().numpy()


def images(batch, h, w, seed=0):
    return np.stack([synth.piecewise_smooth_image(h, w, seed=seed, index=i)
                     for i in range(batch)])


# ---------------------------------------------------------------------------
# 2D
# ---------------------------------------------------------------------------
# Sides that are multiples of 32 run the register/shuffle kernels (one per
# level count 1..6); other sides divisible by 8 run the shared-memory tile
# kernels; the rest (or misaligned rows) run the scalar tile kernels.
CASES_2D = [
    (1, 2, 2, 1),        # smallest image (scalar)
    (1, 8, 8, 3),        # full depth of a tiny image (tile kernel)
    (2, 64, 64, 6),      # fast, six levels, CTA half outside the image
    (1, 96, 160, 5),     # fast, partial CTA in both directions
    (3, 32, 256, 5),     # fast, batch of 3
    (1, 128, 64, 6),     # fast, tall image
    (1, 256, 512, 8),    # two chained passes (6 fast + 2 on a 4 x 8 image)
    (1, 1024, 1024, 10),
    (2, 192, 320, 1),    # fast, one level
    (1, 64, 96, 2),      # fast, two levels
    (2, 128, 96, 3),     # fast, three levels
    (1, 96, 64, 4),      # fast, four levels
    (1, 48, 40, 3),      # sides not multiples of 32 -> tile kernel
    (1, 80, 120, 3),     # tile kernel, ragged tiles
    (1, 48, 36, 2),      # w % 8 != 0 -> scalar kernel
]


@pytest.mark.parametrize("b,h,w,levels", CASES_2D)
@pytest.mark.parametrize("dt", [torch.float32, torch.bfloat16, torch.float16])
def test_dwt2d_matches_oracle(b, h, w, levels, dt):
    x = dev(images(b, h, w, seed=h * 7 + w), dt)
    c = api.dwt2d(x, levels)
    assert c.dtype == dt
    ref = oracle.dwt2d(host64(x), levels)
    assert_close(c, ref, dt, f"dwt2d {b}x{h}x{w} L{levels} {dt}")


@pytest.mark.parametrize("b,h,w,levels", CASES_2D)
@pytest.mark.parametrize("dt", [torch.float32, torch.bfloat16, torch.float16])
def test_idwt2d_matches_oracle(b, h, w, levels, dt):
    x = images(b, h, w, seed=h * 5 + w)
    c = dev(oracle.dwt2d(x, levels), dt)
    y = api.idwt2d(c, levels)
    ref = oracle.idwt2d(host64(c), levels)
    assert_close(y, ref, dt, f"idwt2d {b}x{h}x{w} L{levels} {dt}")


@pytest.mark.parametrize("b,h,w,levels", CASES_2D)
def test_round_trip_2d_fp32(b, h, w, levels):
    x = dev(images(b, h, w, seed=3), torch.float32)
    y = api.idwt2d(api.dwt2d(x, levels), levels)
    assert oracle.rel_l2(host64(y), host64(x)) <= 1e-6


def test_image_workload_full_size():
    """4096 x 4096 fp32, 5 levels: every coefficient and every reconstructed
    pixel against the oracle."""
    cfg = synth.Image2D()
    xn = synth.piecewise_smooth_image(cfg.h, cfg.w, cfg.seed).astype(np.float32)
    x = dev(xn, torch.float32)
    c = api.dwt2d(x, cfg.levels)
    ref = oracle.dwt2d(xn.astype(np.float64), cfg.levels)
    assert_close(c, ref, torch.float32, "dwt2d 4096^2 L5")
    y = api.idwt2d(c, cfg.levels)
    assert_close(y, oracle.idwt2d(host64(c), cfg.levels), torch.float32, "idwt2d 4096^2 L5")
    assert oracle.rel_l2(host64(y), xn) <= 1e-6


def test_precision_workload_full_size():
    """64 x 2048 x 2048, 4 levels, through Plan (the benchmark's launch
    configuration): bf16 storage, and uint8 input with bf16 coefficients and
    fp32 output.  Three images spread over the batch are checked coefficient
    by coefficient against the oracle (on exactly the values the GPU read);
    the whole batch through its round-trip error."""
    cfg = synth.PrecisionBatch()
    distinct = 8  # the batch repeats 8 generated images, as the benchmark does
    base = np.stack([synth.piecewise_smooth_image(cfg.h, cfg.w, cfg.seed, i)
                     for i in range(distinct)])
    xb = dev(base, torch.bfloat16).repeat(cfg.batch // distinct, 1, 1)
    checked = (0, 37, cfg.batch - 1)
    for x, cdt, ydt, tol in ((xb, torch.bfloat16, torch.bfloat16, 1e-2),
                             ((xb.float().clamp(0, 1) * 255).round().to(torch.uint8),
                              torch.bfloat16, torch.float32, 1e-2)):
        c = torch.empty(x.shape, dtype=cdt, device=DEV)
        y = torch.empty(x.shape, dtype=ydt, device=DEV)
        plan = api.Plan(x, c, cfg.levels, y)
        plan.dwt()
        plan.idwt()
        torch.cuda.synchronize()
        for i in checked:
            ref = oracle.dwt2d(host64(x[i]), cfg.levels)
            assert_close(c[i], ref, cdt, f"precision dwt image {i} {x.dtype}")
        xs = x.double()
        err = float(torch.linalg.vector_norm(y.double() - xs) / torch.linalg.vector_norm(xs))
        assert err <= tol, f"precision round trip {x.dtype}: {err:.3e}"
        del c, y, plan


@pytest.mark.parametrize("levels", [7, 12])
def test_deep_2d_chained_passes(levels):
    x = dev(images(1, 4096, 4096, seed=levels), torch.float32)
    c = api.dwt2d(x, levels)
    ref = oracle.dwt2d(host64(x), levels)
    assert_close(c, ref, torch.float32, f"dwt2d 4096^2 L{levels}")
    y = api.idwt2d(c, levels)
    assert_close(y, oracle.idwt2d(host64(c), levels), torch.float32, f"idwt2d L{levels}")


def test_strided_and_offset_views():
    """Views with row_stride > w and batch_stride > h*row_stride; an offset
    of 8 elements keeps the vector path, an offset of 1 forces the scalar
    path."""
    base = dev(images(2, 80, 200, seed=9), torch.float32)
    for off in (8, 1):
        x = base[:, 8:72, off:off + 128]
        assert x.stride(-2) == 200
        c = torch.empty((2, 64, 160), device=DEV)[:, :, 16:144]
        api.dwt2d(x, 4, out=c)
        assert_close(c, oracle.dwt2d(host64(x), 4), torch.float32, f"strided off={off}")
        y = api.idwt2d(c, 4)
        assert oracle.rel_l2(host64(y), host64(x)) <= 1e-6


@pytest.mark.parametrize("cdt", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("b,h,w,levels", [(3, 64, 256, 3), (4, 32, 64, 1), (2, 96, 160, 5)])
def test_idwt2d_half_coefficients_to_fp32_batched(cdt, b, h, w, levels):
    """Synthesis from 16-bit coefficients into fp32 output, several batch
    items: every item's low band is read at its own offset."""
    x = images(b, h, w, seed=b + h)
    c = dev(oracle.dwt2d(x, levels), cdt)
    y = api.idwt2d(c, levels, dtype=torch.float32)
    assert y.dtype == torch.float32
    ref = oracle.idwt2d(host64(c), levels)
    assert_close(y, ref, torch.float32, f"idwt2d {cdt} -> fp32 {b}x{h}x{w} L{levels}")


def test_uint8_input():
    xn = synth.quantize_u8(images(2, 128, 256, seed=4))
    x = torch.from_numpy(xn).to(DEV)
    for dt in (torch.float32, torch.bfloat16):
        c = api.dwt2d(x, 4, dtype=dt)
        assert_close(c, oracle.dwt2d(xn.astype(np.float64), 4), dt, f"u8 -> {dt}")


# 1-byte images: sides that are multiples of 64 with 16-byte aligned rows take
# the wide-lane analysis (4 x 16 pixels per lane), others the 4 x 8 one.  The
# bytes are exact in FP32 and every kernel performs the same butterflies, so
# the coefficients must equal those of the same image given as fp32.
@pytest.mark.parametrize("b,h,w,levels", [(2, 32, 64, 1), (1, 64, 128, 2), (3, 96, 192, 3),
                                          (2, 128, 256, 4), (1, 64, 320, 5), (1, 2048, 2048, 4),
                                          (2, 64, 96, 4)])
@pytest.mark.parametrize("dt", [torch.float32, torch.bfloat16, torch.float16])
def test_uint8_analysis_equals_fp32_input_path(b, h, w, levels, dt):
    xn = synth.quantize_u8(images(b, h, w, seed=h + w + levels))
    x = torch.from_numpy(xn).to(DEV)
    c = api.dwt2d(x, levels, dtype=dt)
    assert torch.equal(c, api.dwt2d(x.float(), levels, dtype=dt))
    assert_close(c, oracle.dwt2d(xn.astype(np.float64), levels), dt, f"u8 {b}x{h}x{w} L{levels}")


@pytest.mark.parametrize("b,h,w,levels", [(2, 32, 64, 1), (1, 64, 128, 2), (3, 96, 192, 3),
                                          (2, 128, 256, 4), (1, 64, 320, 5), (2, 64, 96, 4)])
@pytest.mark.parametrize("tin", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("dt", [torch.float32, torch.bfloat16])
def test_half_analysis_equals_fp32_input_path(b, h, w, levels, tin, dt):
    """16-bit images (wide-lane analysis for sides multiple of 64): exact in
    FP32, so the coefficients equal those of the same values given as fp32."""
    x = dev(images(b, h, w, seed=h * 3 + w + levels), tin)
    c = api.dwt2d(x, levels, dtype=dt)
    assert torch.equal(c, api.dwt2d(x.float(), levels, dtype=dt))


def test_uint8_analysis_unaligned_rows():
    """Rows starting 8 bytes past a 16-byte boundary take the 4 x 8 lane
    layout (8-byte loads); the result is the same."""
    base = torch.from_numpy(synth.quantize_u8(images(2, 64, 272, seed=12))).to(DEV)
    x = base[:, :, 8:264]
    c = api.dwt2d(x, 5, dtype=torch.bfloat16)
    assert torch.equal(c, api.dwt2d(x.float(), 5, dtype=torch.bfloat16))
    assert_close(c, oracle.dwt2d(host64(x), 5), torch.bfloat16, "u8 offset 8")


def test_fp64_path():
    x = dev(images(2, 64, 128, seed=5), torch.float64)
    c = api.dwt2d(x, 6)
    assert_close(c, oracle.dwt2d(host64(x), 6), torch.float64, "fp64 dwt2d")
    y = api.idwt2d(c, 6)
    assert np.max(np.abs(host64(y) - host64(x))) < 1e-14


def test_constant_image_has_exact_zero_detail():
    """A constant image gives exactly zero detail in fp32 (x1 - x0 = 0) and
    LL_L = 2^L c exactly for c a power of two."""
    x = torch.full((1, 256, 512), 0.25, device=DEV)
    c = host64(api.dwt2d(x, 6))[0]
    mask = oracle.detail_mask_2d(256, 512, 6)
    assert np.all(c[mask] == 0.0)
    assert np.all(c[~mask] == 0.25 * 64)


def test_impulse_responses_match_oracle_columns():
    """W e_i for every pixel i of a 16 x 32 image (L = 3): the GPU's linear
    map equals the oracle's, column by column."""
    h, w, L = 16, 32, 3
    eye = torch.eye(h * w, device=DEV).reshape(h * w, h, w)
    cols = host64(api.dwt2d(eye, L)).reshape(h * w, h * w).T
    ref = np.stack([oracle.dwt2d(np.eye(h * w)[i].reshape(h, w), L).ravel()
                    for i in range(h * w)], axis=1)
    assert np.max(np.abs(cols - ref)) < 1e-7


# ---------------------------------------------------------------------------
# 1D
# ---------------------------------------------------------------------------
CASES_1D = [
    (1, 1, 2, 1),
    (1, 1, 8, 3),
    (1, 1, 65536, 1),        # the signal workload
    (2, 3, 3112, 3),         # ragged chunk tail, batch x rows
    (1, 4, 1024, 10),
    (1, 1, 4096 + 8, 3),
    (1, 2, 1 << 20, 16),     # two chained passes (12 + 4)
    (1, 1, 1000, 3),         # ragged chunk tail
    (1, 3, 1004, 2),         # n % 8 != 0 -> scalar path
]


@pytest.mark.parametrize("b,r,n,levels", CASES_1D)
@pytest.mark.parametrize("dt", [torch.float32, torch.bfloat16, torch.float16])
def test_dwt1d_matches_oracle(b, r, n, levels, dt):
    xs = np.stack([synth.signal_1d(n, seed=n, index=i) for i in range(b * r)]).reshape(b, r, n)
    x = dev(xs, dt)
    c = api.dwt1d(x, levels)
    assert_close(c, oracle.dwt1d(host64(x), levels), dt, f"dwt1d {b}x{r}x{n} L{levels}")
    y = api.idwt1d(c, levels)
    assert_close(y, oracle.idwt1d(host64(c), levels), dt, f"idwt1d {b}x{r}x{n} L{levels}")
    if dt == torch.float32:
        assert oracle.rel_l2(host64(y), host64(x)) <= 1e-6


def test_signal_workload_round_trip():
    cfg = synth.Signal1D()
    xn = synth.signal_1d(cfg.n, cfg.seed).astype(np.float32)
    x = dev(xn, torch.float32)
    c = api.dwt1d(x, cfg.levels)
    assert_close(c, oracle.dwt1d(xn.astype(np.float64), cfg.levels), torch.float32, "signal")
    y = api.idwt1d(c, cfg.levels)
    assert oracle.rel_l2(host64(y), xn) <= 1e-6
    lo, hi = oracle.polyphase_analysis_1d(xn.astype(np.float64))
    got = host64(c)
    assert oracle.rel_l2(got[:cfg.n // 2], lo) <= 1e-6
    assert oracle.rel_l2(got[cfg.n // 2:], hi) <= 1e-6


def test_1d_fp64_and_u8():
    x = dev(synth.signal_1d(4096, seed=1), torch.float64)
    c = api.dwt1d(x, 12)
    assert_close(c, oracle.dwt1d(host64(x), 12), torch.float64, "fp64 dwt1d")
    u = torch.from_numpy(synth.quantize_u8(synth.signal_1d(2048, seed=2) * 0.2 + 0.5)).to(DEV)
    cu = api.dwt1d(u, 5)
    assert_close(cu, oracle.dwt1d(host64(u), 5), torch.float32, "u8 dwt1d")


def test_empty_tensors():
    x = torch.empty((0, 64, 64), device=DEV)
    assert api.dwt2d(x, 3).shape == (0, 64, 64)
    assert api.idwt1d(torch.empty((3, 0), device=DEV), 2).shape == (3, 0)


def test_plan_and_graph_capture_match_eager():
    """A Plan replayed from a CUDA graph gives the same coefficients and
    reconstruction as the one-shot calls, including a deep (chained,
    workspace-using) transform."""
    for levels in (5, 8):
        x = dev(images(2, 256, 512, seed=levels), torch.float32)
        c = torch.empty_like(x)
        y = torch.empty_like(x)
        plan = api.Plan(x, c, levels, y)
        plan.dwt()
        plan.idwt()
        torch.cuda.synchronize()
        c.zero_()
        y.zero_()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            plan.dwt()
            plan.idwt()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(c, api.dwt2d(x, levels))
        assert torch.equal(y, api.idwt2d(api.dwt2d(x, levels), levels))
