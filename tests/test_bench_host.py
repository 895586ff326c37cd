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


def test_kernel_hash_ignores_comments_and_layout():
    """The recorded DRAM traffic is keyed to the kernel code: comment or
    whitespace edits keep the key, a change of code changes it."""
    a = "int f(int x) {\n  return x + 1;  // add one\n}\n/* trailing */"
    b = "/* header */ int f(int x) { return x + 1; }"
    c = "int f(int x) { return x + 2; }"
    assert bench.code_only(a) == bench.code_only(b)
    assert bench.code_only(a) != bench.code_only(c)
    s = 'asm("cp.async.bulk [%0]; // not a comment");'
    assert "// not a comment" in bench.code_only(s)
