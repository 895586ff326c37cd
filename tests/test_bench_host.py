"""Host-side helpers of bench.py (no GPU)."""
import numpy as np
import pytest

import bench


@pytest.mark.parametrize("angles", [[0.2, 0.5, -0.4, 0.9], [0.7], [1.1, -0.3, 0.25]])
def test_lattice_taps_are_orthonormal(angles):
    """The K-tap workload's filter must be double-shift orthonormal
    (sum_k h[k] h[k + 2m] = delta_m), the condition for the bank's perfect
    reconstruction that the benchmark checks on its round trip."""
    h = np.array(bench.lattice_taps(angles))
    assert h.size == 2 * len(angles)
    for m in range(len(angles)):
        s = float(np.dot(h[:h.size - 2 * m], h[2 * m:]))
        assert abs(s - (1.0 if m == 0 else 0.0)) <= 1e-14, (m, s)


def test_lattice_taps_with_one_angle_is_a_rotation():
    # one stage: h = (cos a, sin a); a = pi/4 gives the Haar low-pass
    h = bench.lattice_taps([np.pi / 4])
    assert np.allclose(h, [2 ** -0.5, 2 ** -0.5], atol=1e-15)
