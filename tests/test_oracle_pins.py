"""Pins of the FP64 oracle against what arXiv:1002.2184 and mathematics fix.

None of these compare the oracle with itself: each expected value comes from
the taps printed in Section II, the pair formulas of Fig. 4, a textbook
closed form (the Haar basis functions), a polynomial identity, numpy's own
convolution, or brute force on tiny inputs.  The mutation test at the end
shows that a plausible mistake (wrong sign, transposed operand, wrong phase,
dropped level, wrong scale) fails at least one pin.
"""
import math
import types

import numpy as np
import pytest

import oracle
from conftest import golden
from paper_1002_2184_gb300 import synth

S = 1.0 / math.sqrt(2.0)


def _taps_from_paper():
    rows = {r[0]: np.array([float(v) for v in r[1:]]) for r in golden("paper_taps.txt")}
    return rows["b0"], rows["b1"], rows["a0"], rows["a1"]


def _matrix(fn, n):
    """Columns are fn(e_i): the linear map as a dense matrix."""
    cols = []
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        cols.append(np.asarray(fn(e)).ravel())
    return np.stack(cols, axis=1)


# --------------------------------------------------------------------------
# Textbook Haar basis (independent closed form).  phi_l is the normalised box
# of width 2^l; psi_l is -1 on its first half and +1 on its second half (the
# high-pass sign of Eq. 9), both scaled by 2^(-l/2).
# --------------------------------------------------------------------------

def _phi(n, l, m):
    v = np.zeros(n)
    v[m << l:(m + 1) << l] = 2.0 ** (-l / 2)
    return v


def _psi(n, l, m):
    v = np.zeros(n)
    half = 1 << (l - 1)
    v[m << l:(m << l) + half] = -(2.0 ** (-l / 2))
    v[(m << l) + half:(m + 1) << l] = 2.0 ** (-l / 2)
    return v


def textbook_1d(n, levels):
    rows = [None] * n
    na = n >> levels
    for m in range(na):
        rows[m] = _phi(n, levels, m)
    for l in range(levels, 0, -1):
        nd = n >> l
        for m in range(nd):
            rows[nd + m] = _psi(n, l, m)
    return np.stack(rows)


def textbook_2d(h, w, levels):
    B = np.zeros((h * w, h * w))

    def put(r, c, vy, vx):
        B[r * w + c] = np.outer(vy, vx).ravel()

    hL, wL = h >> levels, w >> levels
    for i in range(hL):
        for j in range(wL):
            put(i, j, _phi(h, levels, i), _phi(w, levels, j))
    for l in range(1, levels + 1):
        hl, wl = h >> l, w >> l
        for i in range(hl):
            for j in range(wl):
                put(i, wl + j, _phi(h, l, i), _psi(w, l, j))       # Hx
                put(hl + i, j, _psi(h, l, i), _phi(w, l, j))       # Hy
                put(hl + i, wl + j, _psi(h, l, i), _psi(w, l, j))  # HH
    return B


# --------------------------------------------------------------------------
# Pin checks, written against an implementation object so that mutants can
# be run through them.  Each returns True when the pin holds.
# --------------------------------------------------------------------------

def pin_paper_pair_formulas(impl):
    """Fig. 4 / Section II: one analysis stage on (x0, x1) is
    d0 = (x0 + x1) s, d1 = (x1 - x0) s, with the printed analysis taps in
    printed order weighting (x[2n], x[2n+1])."""
    b0, b1, _, _ = _taps_from_paper()
    rng = synth.rng(1, 0)
    x = rng.standard_normal(64)
    lo, hi = impl.analysis_1d(x)
    pairs = x.reshape(-1, 2)
    return (np.allclose(lo, pairs @ b0, rtol=0, atol=1e-14)
            and np.allclose(hi, pairs @ b1, rtol=0, atol=1e-14))


def pin_two_sample_matrix(impl):
    """H2 = s [[1, 1], [-1, 1]]: det +1 (a rotation), orthogonal."""
    M = _matrix(lambda e: np.concatenate(impl.analysis_1d(e)), 2)
    H2 = S * np.array([[1.0, 1.0], [-1.0, 1.0]])
    return (np.allclose(M, H2, atol=1e-15)
            and abs(np.linalg.det(M) - 1.0) < 1e-14
            and np.allclose(M @ M.T, np.eye(2), atol=1e-15))


def pin_4pt_golden(impl):
    G = np.array([[float(v) for v in r] for r in golden("haar_1d_4pt_2level.txt")])
    M = _matrix(lambda e: impl.dwt1d(e, 2), 4)
    return np.allclose(M, G, rtol=0, atol=1e-15)


def pin_2x2_golden(impl):
    G = np.array([[float(v) for v in r] for r in golden("haar_2d_2x2_butterfly.txt")])
    M = _matrix(lambda e: impl.dwt2d(e.reshape(2, 2), 1).ravel(), 4)
    return np.allclose(M, G, rtol=0, atol=1e-15)


def pin_textbook_1d(impl):
    for n, levels in [(2, 1), (8, 1), (8, 3), (16, 2), (32, 5), (64, 4)]:
        M = _matrix(lambda e: impl.dwt1d(e, levels), n)
        if not np.allclose(M, textbook_1d(n, levels), rtol=0, atol=1e-14):
            return False
    return True


def pin_textbook_2d(impl):
    for h, w, levels in [(2, 2, 1), (4, 4, 2), (8, 8, 3), (4, 8, 2), (8, 4, 1),
                         (16, 8, 3)]:
        M = _matrix(lambda e: impl.dwt2d(e.reshape(h, w), levels).ravel(), h * w)
        if not np.allclose(M, textbook_2d(h, w, levels), rtol=0, atol=1e-14):
            return False
    return True


def pin_constant_input(impl):
    """A constant has zero detail at every level; the approximation grows by
    sqrt(2) per level in 1D and by 2 per level in 2D."""
    c = 0.3
    for levels in (1, 3, 5):
        y = impl.dwt1d(np.full(64, c), levels)
        na = 64 >> levels
        if np.any(y[na:] != 0.0):
            return False
        if not np.allclose(y[:na], c * 2.0 ** (levels / 2), rtol=1e-14, atol=0):
            return False
        z = impl.dwt2d(np.full((32, 64), c), levels)
        mask = oracle.detail_mask_2d(32, 64, levels)
        if np.any(z[mask] != 0.0):
            return False
        if not np.allclose(z[~mask], c * 2.0 ** levels, rtol=1e-14, atol=0):
            return False
    return True


def pin_alternating_sign(impl):
    """x[n] = (-1)^n is pure high frequency: d0 = 0 and d1 = -sqrt(2)
    (d1 = (x[2n+1] - x[2n]) s with x[2n] = 1, x[2n+1] = -1)."""
    x = np.array([1.0, -1.0] * 16)
    lo, hi = impl.analysis_1d(x)
    return (np.allclose(lo, 0.0, atol=1e-15)
            and np.allclose(hi, -math.sqrt(2.0), rtol=1e-15, atol=0))


def pin_parseval(impl):
    rng = synth.rng(2, 0)
    x1 = rng.standard_normal(1024)
    x2 = rng.standard_normal((64, 128))
    e1 = np.sum(impl.dwt1d(x1, 6) ** 2) / np.sum(x1 ** 2)
    e2 = np.sum(impl.dwt2d(x2, 4) ** 2) / np.sum(x2 ** 2)
    return abs(e1 - 1) < 1e-13 and abs(e2 - 1) < 1e-13


PINS = [pin_paper_pair_formulas, pin_two_sample_matrix, pin_4pt_golden,
        pin_2x2_golden, pin_textbook_1d, pin_textbook_2d, pin_constant_input,
        pin_alternating_sign, pin_parseval]


def _oracle_impl(detail_sign=1):
    return types.SimpleNamespace(
        analysis_1d=lambda x: oracle.analysis_1d(x, detail_sign),
        dwt1d=lambda x, L: oracle.dwt1d(x, L, detail_sign),
        dwt2d=lambda x, L: oracle.dwt2d(x, L, detail_sign),
    )


@pytest.mark.parametrize("pin", PINS, ids=lambda p: p.__name__)
def test_pin_holds(pin):
    assert pin(_oracle_impl())


# --------------------------------------------------------------------------
# Properties that need no implementation object.
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,levels", [(2, 1), (64, 1), (64, 6), (1000, 3),
                                      (4096, 12), (65536, 1)])
def test_perfect_reconstruction_1d(n, levels):
    x = synth.signal_1d(n, seed=7, index=n + levels)
    y = oracle.idwt1d(oracle.dwt1d(x, levels), levels)
    assert np.max(np.abs(y - x)) < 1e-13 * max(1.0, np.max(np.abs(x)))


@pytest.mark.parametrize("h,w,levels", [(2, 2, 1), (8, 16, 3), (64, 32, 5),
                                        (96, 160, 5), (256, 256, 8)])
def test_perfect_reconstruction_2d(h, w, levels):
    x = synth.piecewise_smooth_image(h, w, seed=11, index=h + w + levels)
    y = oracle.idwt2d(oracle.dwt2d(x, levels), levels)
    assert np.max(np.abs(y - x)) < 1e-14


def test_synthesis_is_transpose_of_analysis():
    """The bank is orthonormal (a_i are the time-reversed b_i, Section II):
    the synthesis matrix equals the transpose of the analysis matrix."""
    A = _matrix(lambda e: oracle.dwt2d(e.reshape(8, 8), 3).ravel(), 64)
    Sy = _matrix(lambda e: oracle.idwt2d(e.reshape(8, 8), 3).ravel(), 64)
    assert np.allclose(Sy, A.T, atol=1e-15)
    assert np.allclose(A @ A.T, np.eye(64), atol=1e-14)


def test_mallat_2d_is_not_kron():
    """With two or more levels the Mallat 2D transform is not the tensor
    product of two 1D transforms (it only recurses on LL)."""
    A = _matrix(lambda e: oracle.dwt2d(e.reshape(4, 4), 2).ravel(), 16)
    H4 = _matrix(lambda e: oracle.dwt1d(e, 2), 4)
    assert not np.allclose(A, np.kron(H4, H4))
    A1 = _matrix(lambda e: oracle.dwt2d(e.reshape(4, 4), 1).ravel(), 16)
    assert np.allclose(A1, textbook_2d(4, 4, 1), atol=1e-15)


def test_alias_cancellation_polynomials():
    """Section II / Eq. 13-15: with the oracle's taps (read back by probing it
    with impulses), A0(z)B0(-z) + A1(z)B1(-z) = 0 (alias term cancels) and
    A0(z)B0(z) + A1(z)B1(z) = 2 z^-1 (distortion is a pure delay, undone by
    taking the odd phase)."""
    def analysis_taps(which):
        # d_i[0] = y_i[1] = b_i[0] x[1] + b_i[1] x[0]
        t0 = oracle.analysis_1d([0.0, 1.0])[which][0]
        t1 = oracle.analysis_1d([1.0, 0.0])[which][0]
        return np.array([t0, t1])

    def synthesis_taps(which):
        d = [[1.0], [0.0]] if which == 0 else [[0.0], [1.0]]
        return oracle.synthesis_1d(d[0], d[1])

    b0, b1 = analysis_taps(0), analysis_taps(1)
    a0, a1 = synthesis_taps(0), synthesis_taps(1)
    alt = np.array([1.0, -1.0])  # f(-z) for a 2-tap causal filter
    alias = np.convolve(a0, b0 * alt) + np.convolve(a1, b1 * alt)
    dist = np.convolve(a0, b0) + np.convolve(a1, b1)
    assert np.allclose(alias, 0.0, atol=1e-15)
    assert np.allclose(dist, [0.0, 2.0, 0.0], atol=1e-15)


def test_definition_matches_numpy_convolution():
    """Analysis = np.convolve with the causal taps, then the odd phase;
    synthesis = zero insertion, np.convolve, sum, truncate."""
    rng = synth.rng(3, 0)
    x = rng.standard_normal(50)
    b0, b1 = np.array([S, S]), np.array([S, -S])
    a0, a1 = np.array([S, S]), np.array([-S, S])
    lo, hi = oracle.analysis_1d(x)
    assert np.allclose(lo, np.convolve(x, b0)[1::2][:25], atol=1e-15)
    assert np.allclose(hi, np.convolve(x, b1)[1::2][:25], atol=1e-15)
    u0 = np.zeros(50)
    u1 = np.zeros(50)
    u0[::2], u1[::2] = lo, hi
    xr = (np.convolve(u0, a0) + np.convolve(u1, a1))[:50]
    assert np.allclose(oracle.synthesis_1d(lo, hi), xr, atol=1e-15)


def test_existing_vs_fast_haar():
    """Section V compares the original bank with the fast one.  On the 1D
    signal workload (2^16 samples) the definition and the polyphase form
    agree to rounding; the error in dB (20 log10 of the relative L2 norm)
    is far below the paper's -90 dB / -160 dB figures."""
    x = synth.signal_1d(1 << 16)
    lo, hi = oracle.analysis_1d(x)
    plo, phi = oracle.polyphase_analysis_1d(x)
    for a, b in ((lo, plo), (hi, phi)):
        err = oracle.rel_l2(b, a)
        assert err < 1e-15
        assert 20 * math.log10(max(err, 1e-300)) < -250
    xr = oracle.polyphase_synthesis_1d(plo, phi)
    assert np.max(np.abs(xr - oracle.synthesis_1d(lo, hi))) < 1e-14
    assert np.max(np.abs(xr - x)) < 1e-13


def test_both_sign_conventions_reconstruct():
    """detail_sign = -1 (the Section II taps read as causal) is also a
    perfect-reconstruction bank; it only negates every detail."""
    x = synth.signal_1d(256, seed=5)
    c1 = oracle.dwt1d(x, 4, 1)
    c2 = oracle.dwt1d(x, 4, -1)
    na = 256 >> 4
    assert np.allclose(c1[:na], c2[:na], atol=0)
    assert np.allclose(c1[na:], -c2[na:], atol=0)
    assert np.allclose(oracle.idwt1d(c2, 4, -1), x, atol=1e-13)


@pytest.mark.parametrize("bad", [(6, 2), (10, 2), (8, 4)])
def test_rejects_nondivisible(bad):
    n, levels = bad
    with pytest.raises(ValueError):
        oracle.dwt1d(np.zeros(n), levels)
    with pytest.raises(ValueError):
        oracle.dwt2d(np.zeros((n, n)), levels)


def test_empty_inputs():
    assert oracle.dwt1d(np.zeros((0, 8)), 3).shape == (0, 8)
    assert oracle.dwt2d(np.zeros((0, 4, 4)), 2).shape == (0, 4, 4)


# --------------------------------------------------------------------------
# Gradient of the denoising loss (the differentiation workload).
# --------------------------------------------------------------------------

def test_loss_gradient_matches_finite_differences():
    rng = synth.rng(4, 0)
    x = rng.standard_normal((2, 1, 8, 8)) * 0.2
    t, lam, L = 0.05, 1e-3, 2
    eps = 1e-6
    c = oracle.dwt2d(x, L)
    # a step of eps moves every coefficient by at most eps: stay off the kinks
    assert np.min(np.abs(np.abs(c) - t)) > 10 * eps
    g = oracle.denoise_loss_grad(x, L, t, lam)
    fd = np.zeros_like(x)
    for idx in np.ndindex(x.shape):
        xp = x.copy()
        xm = x.copy()
        xp[idx] += eps
        xm[idx] -= eps
        fd[idx] = (oracle.denoise_loss(xp, L, t, lam)[0]
                   - oracle.denoise_loss(xm, L, t, lam)[0]) / (2 * eps)
    assert np.max(np.abs(g - fd)) < 1e-8


def test_loss_limits():
    """threshold 0 and no L1 term: the round trip is exact, loss and gradient
    vanish.  Huge threshold: everything is zeroed, loss = mean(x^2) and the
    gradient is 2x/n."""
    rng = synth.rng(6, 0)
    x = rng.standard_normal((1, 2, 16, 16))
    loss, _, _ = oracle.denoise_loss(x, 3, 0.0, 0.0)
    assert loss < 1e-28
    assert np.max(np.abs(oracle.denoise_loss_grad(x, 3, 0.0, 0.0))) < 1e-15
    loss, mse, l1 = oracle.denoise_loss(x, 3, 1e6, 1e-3)
    assert l1 == 0.0 and abs(loss - np.mean(x ** 2)) < 1e-14
    g = oracle.denoise_loss_grad(x, 3, 1e6, 1e-3)
    assert np.allclose(g, 2 * x / x.size, atol=1e-16)


def _haar_2x2_from_bands(ll, hx, hy, hh):
    """The 2 x 2 image whose one-level coefficients are the given bands: the
    textbook Haar basis images (box, step along the width, step along the
    height, checkerboard), each of norm 1 after the factor 1/2."""
    box = np.array([[1.0, 1.0], [1.0, 1.0]])
    step_x = np.array([[-1.0, 1.0], [-1.0, 1.0]])
    step_y = np.array([[-1.0, -1.0], [1.0, 1.0]])
    checker = np.array([[1.0, -1.0], [-1.0, 1.0]])
    return 0.5 * (ll * box + hx * step_x + hy * step_y + hh * checker)


# The coefficients of the intermediate-threshold case below and what the
# denoising loss (t = 0.05, lam = 1e-3) must give, derived by hand:
#   c = [[LL, Hx], [Hy, HH]] = [[2, 0.3], [-0.2, 0.03]]
#   soft threshold: s = [[1.95, 0.25], [-0.15, 0]] (LL and Hx shrink toward 0,
#     the negative Hy shrinks toward 0 keeping its sign, HH < t vanishes)
#   mse = |x_r - x|^2 / 4 = |s - c|^2 / 4 (Parseval) = (3 * 0.05^2 + 0.03^2) / 4
#   l1 = (|0.25| + |-0.15| + 0) / 3 (three detail coefficients; LL excluded)
#   gradient, mapped back to coefficients (W g): a coefficient above t
#   contributes only lam * sign(s) / 3 if it is a detail, one below t
#   contributes 2 c / 4: W g = [[0, lam/3], [-lam/3, 0.015]]
_C_MID = (2.0, 0.3, -0.2, 0.03)
_T_MID, _LAM_MID = 0.05, 1e-3
_MSE_MID = (3 * 0.05 ** 2 + 0.03 ** 2) / 4
_L1_MID = (0.25 + 0.15) / 3
_WG_MID = np.array([[0.0, _LAM_MID / 3], [-_LAM_MID / 3, 0.015]])


def pin_loss_at_intermediate_threshold(loss_fn, grad_fn):
    x = _haar_2x2_from_bands(*_C_MID)[None, None]
    if not np.allclose(oracle.dwt2d(x[0, 0], 1), [[2.0, 0.3], [-0.2, 0.03]], atol=1e-15):
        return False
    loss, mse, l1 = loss_fn(x, 1, _T_MID, _LAM_MID)
    if not (abs(mse - _MSE_MID) < 1e-15 and abs(l1 - _L1_MID) < 1e-15
            and abs(loss - (_MSE_MID + _LAM_MID * _L1_MID)) < 1e-15):
        return False
    wg = oracle.dwt2d(grad_fn(x, 1, _T_MID, _LAM_MID)[0, 0], 1)
    return bool(np.allclose(wg, _WG_MID, atol=1e-15))


def test_loss_closed_form_at_intermediate_threshold():
    """Soft threshold between 0 and infinity, on coefficients of both signs
    above and below it, with the loss and gradient derived by hand."""
    assert pin_loss_at_intermediate_threshold(oracle.denoise_loss, oracle.denoise_loss_grad)


@pytest.mark.parametrize("mistake", ["half_threshold", "no_sign", "details_only",
                                     "hard_instead_of_soft"])
def test_planted_soft_threshold_mistake_is_caught(mistake, monkeypatch):
    wrong = {
        "half_threshold": lambda c, t: np.sign(c) * np.maximum(np.abs(c) - t / 2, 0.0),
        "no_sign": lambda c, t: np.maximum(np.abs(np.asarray(c, float)) - t, 0.0),
        "details_only": None,
        "hard_instead_of_soft": lambda c, t: np.where(np.abs(c) > t, c, 0.0),
    }[mistake]
    if wrong is None:
        # threshold every coefficient but the low band (LL kept)
        def wrong(c, t):
            c = np.asarray(c, float)
            out = np.sign(c) * np.maximum(np.abs(c) - t, 0.0)
            out[..., 0, 0] = c[..., 0, 0]
            return out
    monkeypatch.setattr(oracle, "soft_threshold", wrong)
    assert not pin_loss_at_intermediate_threshold(oracle.denoise_loss,
                                                  oracle.denoise_loss_grad)


# --------------------------------------------------------------------------
# Mutation test: mistakes planted in (wrappers around) the oracle, on the
# CPU, must each fail at least one pin.
# --------------------------------------------------------------------------

def _mutants():
    base = _oracle_impl()
    flipped = _oracle_impl(detail_sign=-1)

    # the image handed over transposed (rows and columns swapped)
    transposed = types.SimpleNamespace(
        analysis_1d=base.analysis_1d, dwt1d=base.dwt1d,
        dwt2d=lambda x, L: oracle.dwt2d(np.asarray(x).T, L)
        if np.asarray(x).shape[0] == np.asarray(x).shape[1]
        else oracle.dwt2d(x, L))

    def wrong_phase_analysis(x):
        return oracle.analysis_1d(np.roll(np.asarray(x, float), 1))

    wrong_phase = types.SimpleNamespace(
        analysis_1d=wrong_phase_analysis,
        dwt1d=lambda x, L: oracle.dwt1d(np.roll(np.asarray(x, float), 1), L),
        dwt2d=base.dwt2d)

    dropped_level = types.SimpleNamespace(
        analysis_1d=base.analysis_1d,
        dwt1d=lambda x, L: oracle.dwt1d(x, max(L - 1, 1)),
        dwt2d=lambda x, L: oracle.dwt2d(x, max(L - 1, 1)))

    def scaled(x):
        lo, hi = oracle.analysis_1d(x)
        return lo * math.sqrt(2.0), hi

    wrong_scale = types.SimpleNamespace(
        analysis_1d=scaled,
        dwt1d=base.dwt1d,
        dwt2d=lambda x, L: oracle.dwt2d(x, L) * np.where(
            oracle.detail_mask_2d(*np.asarray(x).shape, L), 1.0, 2.0))

    return {"sign": flipped, "transposed": transposed, "phase": wrong_phase,
            "dropped_level": dropped_level, "scale": wrong_scale}


@pytest.mark.parametrize("name", ["sign", "transposed", "phase",
                                  "dropped_level", "scale"])
def test_planted_mistake_is_caught(name):
    impl = _mutants()[name]
    failed = [p.__name__ for p in PINS if not p(impl)]
    assert failed, f"mutant {name} passed every pin"


# --------------------------------------------------------------------------
# Wavelet shrinkage: closed-form limits.
# --------------------------------------------------------------------------

def test_shrink_limits_are_block_means_and_identity():
    """With an infinite threshold every detail vanishes and the output is the
    mean over each 2^L block (1D) or 2^L x 2^L block (2D) -- the Haar scaling
    function; with threshold 0 the output is the input."""
    rng = synth.rng(8, 0)
    x = rng.standard_normal((3, 256))
    for L in (1, 3, 8):
        y = oracle.denoise1d(x, L, 1e30)
        blocks = x.reshape(3, -1, 1 << L).mean(axis=-1)
        assert np.allclose(y, np.repeat(blocks, 1 << L, axis=-1), atol=1e-13)
        assert np.allclose(oracle.denoise1d(x, L, 0.0), x, atol=1e-13)
    im = rng.standard_normal((2, 64, 96))
    for L in (1, 2, 5):
        y = oracle.denoise2d(im, L, 1e30)
        b = 1 << L
        means = im.reshape(2, 64 // b, b, 96 // b, b).mean(axis=(2, 4))
        assert np.allclose(y, np.repeat(np.repeat(means, b, axis=1), b, axis=2), atol=1e-13)
        assert np.allclose(oracle.denoise2d(im, L, 0.0, hard=True), im, atol=1e-13)


def test_hard_shrink_keeps_large_details_exactly():
    """A step edge has one large level-1 detail; with a threshold between
    the noise-free details (0) and the edge detail, hard shrinkage returns
    the signal unchanged and soft shrinkage moves it by exactly t/sqrt(2) at
    the two samples of the edge pair."""
    x = np.zeros(16)
    x[5:] = 1.0  # edge inside the pair (4, 5)
    y = oracle.denoise1d(x, 1, 0.1, hard=True)
    assert np.allclose(y, x, atol=1e-15)
    ys = oracle.denoise1d(x, 1, 0.1)
    d = ys - x
    assert np.allclose(d[[4, 5]], [0.1 / np.sqrt(2), -0.1 / np.sqrt(2)], atol=1e-15)
    assert np.allclose(np.delete(d, [4, 5]), 0.0, atol=1e-15)


def test_decision_masks_reproduce_the_default_paths():
    """Passing the FP64 decision itself as `keep` changes nothing; a flipped
    decision changes exactly the coefficients it names."""
    rng = synth.rng(15, 0)
    x = rng.standard_normal((2, 256))
    c = oracle.dwt1d(x, 4)
    keep = np.abs(c) > 0.7
    assert np.array_equal(oracle.denoise1d(x, 4, 0.7, True, keep),
                          oracle.denoise1d(x, 4, 0.7, True))
    im = rng.standard_normal((1, 2, 32, 32)) * 0.2
    ci = oracle.dwt2d(im, 3)
    k2 = np.abs(ci) > 0.05
    assert np.array_equal(oracle.denoise_loss_grad(im, 3, 0.05, 1e-3, k2),
                          oracle.denoise_loss_grad(im, 3, 0.05, 1e-3))
    flipped = keep.copy()
    flipped[0, 200] = ~flipped[0, 200]
    d = oracle.dwt1d(oracle.denoise1d(x, 4, 0.7, True, flipped) - oracle.denoise1d(x, 4, 0.7, True), 4)
    assert np.count_nonzero(np.abs(d) > 1e-12) == 1 and abs(abs(d[0, 200]) - abs(c[0, 200])) < 1e-12


# --------------------------------------------------------------------------
# Undecimated (stationary) transform.
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,levels", [(16, 1), (64, 3), (256, 5), (1024, 10)])
def test_swt_decimates_to_the_dwt(n, levels):
    """Keeping every 2^l-th sample of level l of the undecimated transform
    gives the decimated (Mallat) coefficients of the pinned DWT."""
    x = synth.signal_1d(n, seed=9, index=n)
    u = oracle.swt1d(x, levels)
    c = oracle.dwt1d(x, levels)
    for l in range(1, levels + 1):
        assert np.allclose(u[l, :: 1 << l], c[n >> l: n >> (l - 1)], atol=1e-13)
    assert np.allclose(u[0, :: 1 << levels], c[: n >> levels], atol=1e-13)


def test_swt_is_shift_equivariant_energy_and_pr():
    rng = synth.rng(10, 0)
    x = rng.standard_normal((3, 128))
    L = 5
    u = oracle.swt1d(x, L)
    assert np.allclose(oracle.swt1d(np.roll(x, 1, axis=-1), L), np.roll(u, 1, axis=-1),
                       atol=1e-13)
    # sum_l |d_l|^2 / 2^l + |a_L|^2 / 2^L = |x|^2 (each level doubles energy)
    e = sum(np.sum(u[:, l] ** 2, axis=-1) / 2.0 ** l for l in range(1, L + 1))
    e = e + np.sum(u[:, 0] ** 2, axis=-1) / 2.0 ** L
    assert np.allclose(e, np.sum(x ** 2, axis=-1), rtol=1e-13)
    assert np.allclose(oracle.iswt1d(u, L), x, atol=1e-13)


def _frame_matrix(n, levels):
    """The undecimated transform as a ((levels + 1) n) x n matrix, column i
    the (pinned) forward transform of the unit impulse e_i."""
    return np.stack([oracle.swt1d(np.eye(n)[i], levels).reshape(-1) for i in range(n)], axis=1)


def pin_iswt_is_weighted_least_squares(iswt):
    """The undecimated transform F is redundant: most coefficient arrays are
    the transform of no signal.  With weights 2^-l on d_l and 2^-L on a_L the
    energy identity above says F^T W F = I, so the inverse that averages the
    two estimates of a_{l-1} at every level is the weighted least-squares
    solution argmin_x sum_l w_l |F_l x - c_l|^2, computed here by numpy's
    least-squares routine on the explicit matrix, on random (inconsistent)
    coefficients."""
    rng = synth.rng(12, 0)
    for n, L in ((16, 1), (32, 3), (64, 5)):
        F = _frame_matrix(n, L)
        w = np.concatenate([np.full(n, 2.0 ** -L)] + [np.full(n, 2.0 ** -l)
                                                      for l in range(1, L + 1)])
        c = rng.standard_normal((L + 1, n))
        sw = np.sqrt(w)
        x_ls = np.linalg.lstsq(F * sw[:, None], c.reshape(-1) * sw, rcond=None)[0]
        if not np.allclose(iswt(c, L), x_ls, atol=1e-12):
            return False
    return True


def test_iswt_is_the_weighted_least_squares_inverse():
    assert pin_iswt_is_weighted_least_squares(oracle.iswt1d)


def test_iswt_single_detail_perturbation_closed_form():
    """One level, one detail coefficient d_1[k] moved by delta: the two
    estimates of x disagree at k (by -delta/sqrt 2) and at k + 1 (by
    +delta/sqrt 2); their average moves x[k] by -delta/(2 sqrt 2) and
    x[k + 1] by +delta/(2 sqrt 2) and nothing else (with wrap-around)."""
    x = synth.signal_1d(64, seed=13)
    for k, delta in ((10, 0.7), (63, -1.3)):
        u = oracle.swt1d(x, 1)
        u[1, k] += delta
        d = oracle.iswt1d(u, 1) - x
        expect = np.zeros(64)
        expect[k] = -delta * S / 2
        expect[(k + 1) % 64] = delta * S / 2
        assert np.allclose(d, expect, atol=1e-14)


def test_planted_iswt_mistake_is_caught():
    """Keeping one estimate of a_{l-1} (from position k only) reconstructs
    consistent coefficients exactly, but is not the least-squares inverse."""
    def first_estimate_only(c, L):
        a = np.asarray(c[0], float).copy()
        for l in range(L, 0, -1):
            a = (a - c[l]) * S
        return a

    x = synth.signal_1d(32, seed=14)
    assert np.allclose(first_estimate_only(oracle.swt1d(x, 3), 3), x, atol=1e-13)
    assert not pin_iswt_is_weighted_least_squares(first_estimate_only)


# --------------------------------------------------------------------------
# 3D (volumes): textbook separable basis, constant input, Parseval, PR.
# --------------------------------------------------------------------------

def textbook_3d(d, h, w, levels):
    n = d * h * w
    B = np.zeros((n, n))

    def put(z, y, x, vz, vy, vx):
        B[(z * h + y) * w + x] = np.einsum("i,j,k->ijk", vz, vy, vx).ravel()

    for l in range(1, levels + 1):
        dl, hl, wl = d >> l, h >> l, w >> l
        for z in range(dl):
            for y in range(hl):
                for x in range(wl):
                    for bz in (0, 1):
                        for by in (0, 1):
                            for bx in (0, 1):
                                if bz == by == bx == 0:
                                    continue
                                vz = _psi(d, l, z) if bz else _phi(d, l, z)
                                vy = _psi(h, l, y) if by else _phi(h, l, y)
                                vx = _psi(w, l, x) if bx else _phi(w, l, x)
                                put(bz * dl + z, by * hl + y, bx * wl + x, vz, vy, vx)
    dL, hL, wL = d >> levels, h >> levels, w >> levels
    for z in range(dL):
        for y in range(hL):
            for x in range(wL):
                put(z, y, x, _phi(d, levels, z), _phi(h, levels, y), _phi(w, levels, x))
    return B


@pytest.mark.parametrize("d,h,w,levels", [(2, 2, 2, 1), (4, 4, 4, 2), (2, 4, 8, 1),
                                          (8, 4, 4, 2), (4, 8, 8, 2)])
def test_3d_matches_textbook_basis(d, h, w, levels):
    n = d * h * w
    M = _matrix(lambda e: oracle.dwt3d(e.reshape(d, h, w), levels).ravel(), n)
    assert np.allclose(M, textbook_3d(d, h, w, levels), rtol=0, atol=1e-14)


def test_3d_constant_parseval_pr():
    c = 0.5
    for L in (1, 2, 3):
        z = oracle.dwt3d(np.full((8, 16, 8), c), L)
        low = z[: 8 >> L, : 16 >> L, : 8 >> L]
        assert np.allclose(low, c * (2.0 ** 1.5) ** L, rtol=1e-14, atol=0)
        assert np.count_nonzero(z) == low.size
    rng = synth.rng(12, 0)
    x = rng.standard_normal((2, 16, 8, 32))
    y = oracle.dwt3d(x, 3)
    assert abs(np.sum(y ** 2) / np.sum(x ** 2) - 1) < 1e-13
    assert np.max(np.abs(oracle.idwt3d(y, 3) - x)) < 1e-13


# --------------------------------------------------------------------------
# General orthonormal two-channel bank (longer filters, periodic boundary).
# --------------------------------------------------------------------------

def lattice_lowpass(angles):
    """An orthonormal low-pass of length 2 * len(angles) built from a
    paraunitary lattice of plane rotations and delays (an independent
    construction: each stage preserves the double-shift orthogonality)."""
    c, s = np.cos(angles[0]), np.sin(angles[0])
    h0, h1 = np.array([c, s]), np.array([-s, c])
    for th in angles[1:]:
        c, s = np.cos(th), np.sin(th)
        z2h1 = np.concatenate([[0.0, 0.0], h1])
        h0p = np.concatenate([h0, [0.0, 0.0]])
        h0, h1 = c * h0p + s * z2h1, -s * h0p + c * z2h1
    return h0


def _d4():
    r3 = np.sqrt(3.0)
    return np.array([1 + r3, 3 + r3, 3 - r3, 1 - r3]) / (4 * np.sqrt(2.0))


def test_d4_closed_form_identities():
    h = _d4()
    assert abs(h.sum() - np.sqrt(2.0)) < 1e-15          # low pass, DC gain sqrt 2
    assert abs(np.dot(h, h) - 1.0) < 1e-15              # unit norm
    assert abs(h[0] * h[2] + h[1] * h[3]) < 1e-16       # orthogonal to its 2-shift
    k = np.arange(4)
    assert abs(np.dot(oracle.qmf_highpass(h), k)) < 1e-14  # two vanishing moments


@pytest.mark.parametrize("taps", ["haar", "d4", "lattice6", "lattice8"])
def test_filter_bank_is_orthonormal(taps):
    h = {"haar": np.full(2, 1 / np.sqrt(2.0)), "d4": _d4(),
         "lattice6": lattice_lowpass([0.3, -0.7, 1.1]),
         "lattice8": lattice_lowpass([0.2, 0.5, -0.4, 0.9])}[taps]
    n, L = 32, 3
    W = _matrix(lambda e: oracle.filter_dwt1d(e, L, h), n)
    assert np.allclose(W @ W.T, np.eye(n), atol=1e-13)
    x = synth.rng(20, 0).standard_normal((2, n))
    assert np.allclose(oracle.filter_idwt1d(oracle.filter_dwt1d(x, L, h), L, h), x, atol=1e-13)


def test_filter_bank_with_haar_taps_is_the_haar_bank():
    x = synth.signal_1d(256, seed=21)
    h = np.full(2, 1 / np.sqrt(2.0))
    assert np.allclose(oracle.filter_dwt1d(x, 5, h), oracle.dwt1d(x, 5), atol=1e-13)


def test_d4_annihilates_linear_ramps():
    """Daubechies-4 has two vanishing moments: every level-1 detail whose
    four taps do not wrap around is exactly zero on a linear ramp."""
    x = 3.0 + 0.25 * np.arange(64)
    lo, hi = oracle.filter_analysis_1d(x, _d4())
    assert np.allclose(hi[:-1], 0.0, atol=1e-13)
    assert abs(hi[-1]) > 1.0  # the wrapped one sees the jump
