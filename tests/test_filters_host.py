"""The Daubechies low-pass generator of the API (no GPU): each filter is
pinned by the properties that determine it -- double-shift orthonormality,
sum sqrt(2), ntaps/2 vanishing moments of the high-pass -- and by the
closed forms of the Haar and Daubechies-4 filters."""
import numpy as np
import pytest

from paper_1002_2184_gb300 import api


@pytest.mark.parametrize("k", [2, 4, 6, 8])
def test_daubechies_is_orthonormal_with_vanishing_moments(k):
    h = np.array(api.daubechies(k))
    assert h.size == k
    assert abs(h.sum() - np.sqrt(2.0)) <= 1e-13
    for m in range(k // 2):
        s = float(np.dot(h[:k - 2 * m], h[2 * m:]))
        assert abs(s - (1.0 if m == 0 else 0.0)) <= 1e-13, (m, s)
    # the high-pass g[j] = (-1)^(j+1) h[k-1-j] annihilates polynomials of degree < k/2
    g = np.array([(-1.0) ** (j + 1) * h[k - 1 - j] for j in range(k)])
    for p in range(k // 2):
        assert abs(float(np.sum(g * np.arange(k) ** p))) <= 1e-11, p


def test_daubechies_closed_forms():
    assert np.allclose(api.daubechies(2), api.HAAR2, rtol=0, atol=1e-15)
    assert np.allclose(api.daubechies(4), api.DAUBECHIES4, rtol=0, atol=1e-14)


def test_daubechies_rejects_other_lengths():
    for k in (1, 3, 10):
        with pytest.raises(ValueError):
            api.daubechies(k)
