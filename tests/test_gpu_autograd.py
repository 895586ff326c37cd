"""Differentiation form: adjoint backward of the transforms, the soft
threshold + L1 + MSE pieces and the fused loss, checked with gradcheck in
FP64, against the oracle's closed-form gradient, and against each other."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1002_2184_gb300 import _lib, api, autograd as ad, synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


def images(shape, seed, dtype):
    b = int(np.prod(shape[:-2]))
    h, w = shape[-2:]
    arr = np.stack([synth.piecewise_smooth_image(h, w, seed=seed, index=i) for i in range(b)])
    return torch.from_numpy(arr.reshape(shape)).to(DEV).to(dtype)


def off_kinks(shape, levels, t, dtype=torch.float64, seed0=0, margin=1e-4):
    """An input whose coefficients all stay at least `margin` away from the
    soft-threshold kinks |c| = t (finite differences must not cross them)."""
    for seed in range(seed0, seed0 + 200):
        x = images(shape, seed, dtype) * 0.3
        c = oracle.dwt2d(x.double().cpu().numpy(), levels)
        if np.min(np.abs(np.abs(c) - t)) > margin:
            return x
    raise RuntimeError("no input away from the kinks")


def test_gradcheck_transforms_fp64():
    x = torch.randn(2, 1, 16, 16, dtype=torch.float64, device=DEV, requires_grad=True)
    assert torch.autograd.gradcheck(lambda v: ad.dwt2d(v, 3), (x,))
    assert torch.autograd.gradcheck(lambda v: ad.idwt2d(v, 3), (x,))
    y = torch.randn(3, 64, dtype=torch.float64, device=DEV, requires_grad=True)
    assert torch.autograd.gradcheck(lambda v: ad.dwt1d(v, 4), (y,))
    assert torch.autograd.gradcheck(lambda v: ad.idwt1d(v, 4), (y,))


def test_adjoint_dot_product():
    """<W x, y> = <x, W^T y> with W^T the synthesis, on a config-sized batch."""
    x = images((4, 3, 128, 128), 1, torch.float64)
    y = images((4, 3, 128, 128), 2, torch.float64)
    lhs = float((api.dwt2d(x, 3) * y).sum())
    rhs = float((x * api.idwt2d(y, 3)).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_gradcheck_unfused_loss_fp64():
    """gradcheck of the composed loss at 2 x 1 x 16 x 16, 3 levels."""
    x = off_kinks((2, 1, 16, 16), 3, 0.05).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda v: ad.denoise_loss_unfused(v, 3, 0.05, 1e-3), (x,),
                                    eps=1e-6, atol=1e-8)


def test_gradcheck_fused_loss_fp64():
    """The fused kernels need sides that are multiples of 32."""
    x = off_kinks((2, 1, 32, 32), 3, 0.05).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda v: ad.denoise_loss(v, 3, 0.05, 1e-3), (x,),
                                    eps=1e-6, atol=1e-8)


def gpu_decision(x: torch.Tensor, levels: int, t: float) -> np.ndarray:
    """[|c| > t] as the kernels decide it: on the FP32 coefficients (the
    analysis inside the loss kernels performs the same operations as the
    separate one) against the threshold rounded to FP32.  The gradient jumps
    where |c| crosses t, so the oracle is handed this decision for an
    element-by-element comparison."""
    c = api.dwt2d(x, levels)
    return (c.abs() > torch.tensor(t, dtype=torch.float32)).cpu().numpy()


def assert_grad_close(g: torch.Tensor, ref: np.ndarray, what: str):
    """rel-L2 <= 1e-5 and every element within 1e-5 of the largest gradient
    magnitude (the FP32 analysis, map and synthesis each round; the loss
    scale 2/n leaves the gradient near 1e-9, so the bound is relative)."""
    got = g.detach().double().cpu().numpy()
    err = oracle.rel_l2(got, ref)
    mx = oracle.max_abs(got, ref)
    scale = float(np.max(np.abs(ref)))
    assert err <= 1e-5, f"{what}: gradient rel-L2 {err:.3e}"
    assert mx <= 1e-5 * scale, f"{what}: gradient max-abs {mx:.3e} (scale {scale:.3e})"


@pytest.mark.parametrize("fused", [True, False])
def test_loss_and_gradient_match_oracle_fp32(fused):
    """Config-shaped batch (reduced batch) in fp32 against the oracle's loss
    and closed-form gradient in fp64."""
    x = images((4, 3, 256, 256), 7, torch.float32).requires_grad_(True)
    fn = ad.denoise_loss if fused else ad.denoise_loss_unfused
    loss = fn(x, 3, 0.05, 1e-3)
    loss.backward()
    xn = x.detach().double().cpu().numpy()
    ref_loss, _, _ = oracle.denoise_loss(xn, 3, 0.05, 1e-3)
    ref_g = oracle.denoise_loss_grad(xn, 3, 0.05, 1e-3, keep=gpu_decision(x.detach(), 3, 0.05))
    assert abs(float(loss.detach()) - ref_loss) <= 1e-5 * abs(ref_loss)
    assert_grad_close(x.grad, ref_g, "fused" if fused else "unfused")


def test_fused_equals_unfused_fp32():
    x = images((2, 3, 128, 256), 3, torch.float32)
    xa = x.clone().requires_grad_(True)
    xb = x.clone().requires_grad_(True)
    la = ad.denoise_loss(xa, 3, 0.05, 1e-3)
    lb = ad.denoise_loss_unfused(xb, 3, 0.05, 1e-3)
    la.backward()
    lb.backward()
    va, vb = float(la.detach()), float(lb.detach())
    assert abs(va - vb) <= 1e-6 * abs(vb)
    err = float(torch.linalg.vector_norm(xa.grad - xb.grad) / torch.linalg.vector_norm(xb.grad))
    assert err <= 1e-5


def test_gradient_workload_full_size():
    """32 x 3 x 512 x 512, 3 levels: loss and gradient of the fused pipeline
    against the oracle over the whole batch."""
    cfg = synth.GradBatch()
    x = images(cfg.shape, cfg.seed, torch.float32).requires_grad_(True)
    loss = ad.denoise_loss(x, cfg.levels, cfg.threshold, cfg.l1_weight)
    loss.backward()
    xn = x.detach().double().cpu().numpy()
    ref_loss, _, _ = oracle.denoise_loss(xn, cfg.levels, cfg.threshold, cfg.l1_weight)
    assert abs(float(loss.detach()) - ref_loss) <= 1e-5 * abs(ref_loss)
    ref_g = oracle.denoise_loss_grad(xn, cfg.levels, cfg.threshold, cfg.l1_weight,
                                     keep=gpu_decision(x.detach(), cfg.levels, cfg.threshold))
    assert_grad_close(x.grad, ref_g, "full-size batch")


def test_soft_threshold_and_l1_pieces():
    c = images((2, 64, 64), 4, torch.float32) - 0.5
    s, l1 = ad.SoftThresholdL1.apply(c, 2, 0.1)
    ref = oracle.soft_threshold(c.double().cpu().numpy(), 0.1)
    assert np.max(np.abs(s.double().cpu().numpy() - ref)) <= 1e-6
    mask = np.broadcast_to(oracle.detail_mask_2d(64, 64, 2), ref.shape)
    assert abs(float(l1) - np.mean(np.abs(ref[mask]))) <= 1e-6


def test_norms_f64():
    a = images((2, 64, 128), 5, torch.float32)
    b = a + 1e-3 * torch.sin(a)
    out = torch.zeros(3, dtype=torch.float64, device=DEV)
    rc = _lib.load().haar_norms_f64(a.data_ptr(), b.data_ptr(), _lib.HAAR_F32, a.numel(),
                                    out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    an, bn = a.double().cpu().numpy(), b.double().cpu().numpy()
    o = out.cpu().numpy()
    assert abs(o[0] - np.sum(an ** 2)) <= 1e-12 * np.sum(an ** 2)
    assert abs(o[1] - np.sum((an - bn) ** 2)) <= 1e-12 * np.sum((an - bn) ** 2)
    assert o[2] == np.max(np.abs(an - bn))


def test_parseval_at_full_size_fp64_reduction():
    """Energy preservation of the 5-level transform of the 4096 x 4096 image,
    measured with the FP64 reductions on the GPU."""
    cfg = synth.Image2D()
    x = images((1, cfg.h, cfg.w), cfg.seed, torch.float32)
    c = api.dwt2d(x, cfg.levels)
    lib = _lib.load()
    ex = torch.zeros(3, dtype=torch.float64, device=DEV)
    ec = torch.zeros(3, dtype=torch.float64, device=DEV)
    st = torch.cuda.current_stream().cuda_stream
    assert lib.haar_norms_f64(x.data_ptr(), None, 0, x.numel(), ex.data_ptr(), st) == 0
    assert lib.haar_norms_f64(c.data_ptr(), None, 0, c.numel(), ec.data_ptr(), st) == 0
    assert abs(float(ec[0]) / float(ex[0]) - 1.0) <= 1e-6


@pytest.mark.parametrize("levels", [1, 2, 3, 4, 5])
def test_fused_every_level_count_fp64(levels):
    """Every compiled level count of the fused loss, in FP64, against the
    oracle's loss and closed-form gradient (tight tolerance)."""
    x = images((2, 2, 64, 96), 9, torch.float64).requires_grad_(True)
    loss = ad.denoise_loss(x, levels, 0.05, 1e-3)
    loss.backward()
    xn = x.detach().cpu().numpy()
    ref_loss, _, _ = oracle.denoise_loss(xn, levels, 0.05, 1e-3)
    ref_g = oracle.denoise_loss_grad(xn, levels, 0.05, 1e-3)
    assert abs(float(loss.detach()) - ref_loss) <= 1e-12 * abs(ref_loss)
    assert oracle.rel_l2(x.grad.cpu().numpy(), ref_g) <= 1e-11


def test_fused_rejects_unsupported_shapes():
    lib = _lib.load()
    acc = torch.zeros(2, dtype=torch.float64, device=DEV)
    loss = torch.empty((), device=DEV)
    x = torch.zeros(1, 64, 64, device=DEV)
    d = api.describe(x)
    st = torch.cuda.current_stream().cuda_stream
    assert lib.haar_denoise_forward(ctypes.byref(d), 6, 0.05, 1e-3, acc.data_ptr(),
                                    loss.data_ptr(), st) == _lib.HAAR_EINVAL
    y = torch.zeros(1, 48, 64, device=DEV)
    assert lib.haar_denoise_forward(ctypes.byref(api.describe(y)), 3, 0.05, 1e-3, acc.data_ptr(),
                                    loss.data_ptr(), st) == _lib.HAAR_ESHAPE
    g = torch.empty_like(x)
    assert lib.haar_denoise_backward(ctypes.byref(d), ctypes.byref(d), 3, 0.05, 1e-3, None,
                                     st) == _lib.HAAR_EALIAS
    assert lib.haar_denoise_backward(ctypes.byref(d), ctypes.byref(api.describe(g)), 3, 0.05,
                                     1e-3, None, st) == _lib.HAAR_OK


def test_denoise_plan_in_a_graph_matches_autograd():
    x = images((2, 3, 128, 128), 6, torch.float32)
    plan = ad.DenoisePlan(x, 3, 0.05, 1e-3)
    plan.forward()
    plan.backward()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.forward()
        plan.backward()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    xr = x.clone().requires_grad_(True)
    loss = ad.denoise_loss(xr, 3, 0.05, 1e-3)
    loss.backward()
    lv = float(loss.detach())
    assert abs(float(plan.loss) - lv) <= 1e-6 * abs(lv)
    assert torch.allclose(plan.grad, xr.grad, rtol=0, atol=0)
