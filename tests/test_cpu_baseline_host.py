"""The benchmark's FP32 CPU baseline (oracle/cpu_baseline.c, the Fast Haar
method as a plain loop) computes the same transform as the FP64 oracle, so
its throughput is a like-for-like CPU reference (no GPU needed)."""
import numpy as np
import pytest

import oracle
from oracle import cpu_baseline
from paper_1002_2184_gb300 import synth


@pytest.mark.parametrize("h,w,levels", [(2, 2, 1), (8, 16, 3), (96, 160, 5), (256, 128, 7),
                                        (64, 64, 6)])
def test_cpu_baseline_matches_oracle(h, w, levels):
    x = synth.piecewise_smooth_image(h, w, seed=h + w, index=levels).astype(np.float32)
    c = cpu_baseline.dwt2d_f32(x, levels)
    ref = oracle.dwt2d(x.astype(np.float64), levels)
    assert oracle.rel_l2(c, ref) <= 1e-6
    assert oracle.max_abs(c, ref) <= 4e-6 * np.max(np.abs(ref))
    y = cpu_baseline.idwt2d_f32(c, levels)
    assert oracle.rel_l2(y, x) <= 1e-6


def test_cpu_baseline_rejects_bad_shapes():
    with pytest.raises(ValueError):
        cpu_baseline.dwt2d_f32(np.zeros((6, 8), np.float32), 2)
