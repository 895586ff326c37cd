"""Ragged batches: one persistent launch over images of different sizes and
level counts, checked against the FP64 oracle (small and sampled cases) and,
at the full 512-image workload, element by element against the strided
single-image path (the same per-warp arithmetic, so the results must be
identical)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1002_2184_gb300 import _lib, api, autotune, synth
from parity_util import assert_close

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


def fill(plan, dtype, seed):
    flat = plan.empty(torch.float64)
    for i, v in enumerate(plan.views(flat)):
        h, w, _ = plan.items[i]
        v.copy_(torch.from_numpy(synth.piecewise_smooth_image(h, w, seed=seed, index=i)))
    return flat.to(dtype)


SMALL = [(32, 32, 1), (64, 64, 6), (32, 96, 5), (96, 32, 3), (64, 128, 4), (128, 64, 2),
         (192, 256, 6), (32, 224, 5), (256, 192, 4), (64, 320, 6)]


UNITS = [_lib.HAAR_UNIT_64x128, _lib.HAAR_UNIT_32x256, _lib.HAAR_UNIT_64x64,
         _lib.HAAR_UNIT_128x128]


@pytest.mark.parametrize("unit", UNITS)
@pytest.mark.parametrize("dt", [torch.float32, torch.bfloat16])
def test_ragged_small_matches_oracle(unit, dt):
    # the 32 x 256 unit takes at most 5 levels; every image of SMALL has sides
    # that leave partial units for the larger shapes
    items = SMALL if unit != _lib.HAAR_UNIT_32x256 else [
        (h, w, min(L, 5)) for h, w, L in SMALL]
    plan = api.RaggedPlan(items, DEV, unit, blocks_per_sm=2)
    x = fill(plan, dt, seed=31)
    c = plan.empty(dt)
    y = plan.empty(dt)
    plan.dwt(x, c)
    plan.idwt(c, y)
    torch.cuda.synchronize()
    for i, (xv, cv, yv) in enumerate(zip(plan.views(x), plan.views(c), plan.views(y))):
        L = items[i][2]
        xr = xv.double().cpu().numpy()
        ref = oracle.dwt2d(xr, L)
        assert_close(cv, ref, dt, f"ragged dwt image {i} {items[i]}")
        yref = oracle.idwt2d(cv.double().cpu().numpy(), L)
        assert_close(yv, yref, dt, f"ragged idwt image {i} {items[i]}")
    assert plan.status() == _lib.HAAR_OK


@pytest.mark.parametrize("unit", UNITS)
def test_ragged_matches_strided_path_bitwise(unit):
    items = SMALL if unit != _lib.HAAR_UNIT_32x256 else [(h, w, min(L, 5)) for h, w, L in SMALL]
    plan = api.RaggedPlan(items, DEV, unit)
    x = fill(plan, torch.float32, seed=5)
    c = plan.empty()
    y = plan.empty()
    plan.dwt(x, c)
    plan.idwt(c, y)
    for i, (xv, cv, yv) in enumerate(zip(plan.views(x), plan.views(c), plan.views(y))):
        L = items[i][2]
        assert torch.equal(cv, api.dwt2d(xv, L)), i
        assert torch.equal(yv, api.idwt2d(cv, L)), i


def test_ragged_graph_replay_and_queue_reset():
    """The last block resets the work queue, so a captured launch can be
    replayed many times; the integrity word stays clear."""
    plan = api.RaggedPlan(SMALL, DEV, blocks_per_sm=3)
    x = fill(plan, torch.float32, seed=8)
    c = plan.empty()
    y = plan.empty()
    plan.dwt(x, c)
    plan.idwt(c, y)
    torch.cuda.synchronize()
    ref_c, ref_y = c.clone(), y.clone()
    c.zero_()
    y.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.dwt(x, c)
        plan.idwt(c, y)
    for _ in range(5):
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(c, ref_c) and torch.equal(y, ref_y)
    assert plan.status() == _lib.HAAR_OK


def test_ragged_queue_fault_is_reported():
    """A work queue left in a wrong state (planted on the host: the unit
    counter starts at 3 instead of 0) makes the launch skip units; the last
    block notices and sets the error word, which status() reports once."""
    plan = api.RaggedPlan(SMALL, DEV, blocks_per_sm=2)
    x = fill(plan, torch.float32, seed=2)
    c = plan.empty()
    torch.cuda.synchronize()
    plan._ws[:8].view(torch.int64).fill_(3)
    plan.dwt(x, c)
    assert plan.status() == _lib.HAAR_EQUEUE
    assert plan.status() == _lib.HAAR_OK  # the word was cleared
    plan.dwt(x, c)                          # the kernel reset the counters
    assert plan.status() == _lib.HAAR_OK
    for i, (xv, cv) in enumerate(zip(plan.views(x), plan.views(c))):
        assert torch.equal(cv, api.dwt2d(xv, SMALL[i][2])), i


def test_ragged_full_workload():
    """512 images, sides uniform on {64, ..., 2048}, levels 3..6: every
    image equals the strided path exactly; six sampled images match the
    oracle; the round trip is exact to 1e-6."""
    cfg = synth.RaggedBatch()
    items = synth.ragged_shapes(cfg)
    plan = api.RaggedPlan(items, DEV)
    x = plan.empty()
    for i, v in enumerate(plan.views(x)):
        h, w, _ = items[i]
        v.copy_(torch.from_numpy(synth.piecewise_smooth_image(h, w, cfg.seed, i)
                                 .astype(np.float32)))
    c = plan.empty()
    y = plan.empty()
    plan.dwt(x, c)
    plan.idwt(c, y)
    torch.cuda.synchronize()
    assert plan.status() == _lib.HAAR_OK
    xv, cv, yv = plan.views(x), plan.views(c), plan.views(y)
    for i in range(len(items)):
        assert torch.equal(cv[i], api.dwt2d(xv[i], items[i][2])), i
    err = torch.linalg.vector_norm((y - x).double()) / torch.linalg.vector_norm(x.double())
    assert float(err) <= 1e-6
    rng = np.random.default_rng(0)
    for i in rng.choice(len(items), size=6, replace=False):
        L = items[i][2]
        ref = oracle.dwt2d(xv[i].double().cpu().numpy(), L)
        assert_close(cv[i], ref, torch.float32, f"ragged full workload image {i} {items[i]}")
        yref = oracle.idwt2d(cv[i].double().cpu().numpy(), L)
        assert_close(yv[i], yref, torch.float32, f"ragged full workload inverse {i}")


def test_autotuner_picks_a_valid_config(tmp_path):
    items = SMALL
    plan = api.RaggedPlan(items, DEV)
    x = fill(plan, torch.float32, seed=1)
    unit, bps, rep = autotune.tune_ragged(items, DEV, x, reps=2,
                                          cache_path=str(tmp_path / "cache.json"))
    assert unit in UNITS and unit != _lib.HAAR_UNIT_32x256  # SMALL has 6-level images
    assert bps in autotune.BLOCKS_PER_SM
    shapes = {k.split("/")[0] for k in rep["timings"]}
    assert shapes == {"64x128", "64x64", "128x128"}
    assert not rep["cached"] and rep["timings"]
    unit2, bps2, rep2 = autotune.tune_ragged(items, DEV, x, reps=2,
                                             cache_path=str(tmp_path / "cache.json"))
    assert rep2["cached"] and (unit2, bps2) == (unit, bps)
