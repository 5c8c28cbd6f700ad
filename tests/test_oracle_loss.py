"""Pins of the oracle's training loss (Sec. 3.3, Eq. 9): L2 + D-SSIM with
lambda = 0.2 and its gradient with respect to the rendered image.

The window is checked against scipy's Gaussian filter (an independent
routine with its own sampling and normalisation), the SSIM map against its
closed forms on constant, shifted and scaled images, the adjoint against the
inner-product identity and the gradient against FP64 central differences.
"""
import numpy as np
import pytest

from oracle import loss as L


def _img(rng, H, W):
    return rng.uniform(0.0, 1.0, size=(H, W, 3))


def test_window_matches_scipy_gaussian_filter():
    ndi = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(0)
    x = rng.uniform(size=(23, 19))
    # truncate * sigma + 0.5 rounds down to radius 5; mode 'constant' = zero padding
    want = ndi.gaussian_filter(x, 1.5, mode="constant", cval=0.0, truncate=5.0 / 1.5)
    assert np.abs(L.window_filter(x) - want).max() < 1e-14
    assert abs(L.gauss_window().sum() - 1.0) < 1e-15
    assert L.gauss_window().shape == (11, 11)


def test_adjoint_identity():
    rng = np.random.default_rng(1)
    x, m = rng.normal(size=(17, 26)), rng.normal(size=(17, 26))
    lhs = float((L.window_filter(x) * m).sum())
    rhs = float((x * L.window_filter_adjoint(m)).sum())
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


def test_identical_images_give_zero_loss_and_a_stationary_point():
    rng = np.random.default_rng(2)
    x = _img(rng, 21, 18)
    assert abs(L.ssim(x, x) - 1.0) < 1e-14
    assert abs(L.loss(x, x)) < 1e-14
    # SSIM(., y) peaks at y, L2 vanishes there: the gradient is zero
    assert np.abs(L.loss_grad(x, x)).max() < 1e-14


def test_constant_images_closed_form_in_the_interior():
    H, W, R = 20, 24, L.RADIUS
    for a, b in ((0.3, 0.7), (0.5, 0.5), (0.0, 0.9)):
        s = L.ssim_map(np.full((H, W), a), np.full((H, W), b))
        want = (2 * a * b + L.C1) / (a * a + b * b + L.C1)
        assert np.abs(s[R:H - R, R:W - R] - want).max() < 1e-12
        # the border sees the zero padding: not the interior value unless a == b
        if a != b:
            assert abs(s[0, 0] - want) > 1e-6


def test_shifted_and_scaled_images_closed_forms():
    ndi = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(3)
    H, W, R = 26, 22, L.RADIUS
    x = rng.uniform(0.2, 0.6, size=(H, W))

    def f(z):
        return ndi.gaussian_filter(z, 1.5, mode="constant", cval=0.0, truncate=5.0 / 1.5)

    mu = f(x)
    var = f(x * x) - mu * mu
    inner = (slice(R, H - R), slice(R, W - R))
    # y = x + d: contrast-structure term is one, luminance term remains
    d = 0.15
    s = L.ssim_map(x, x + d)
    want = (2 * mu * (mu + d) + L.C1) / (mu * mu + (mu + d) ** 2 + L.C1)
    assert np.abs(s - want)[inner].max() < 1e-11
    # y = k x: both terms in closed form of mu and var
    k = 1.7
    s = L.ssim_map(x, k * x)
    want = ((2 * k * mu * mu + L.C1) * (2 * k * var + L.C2)
            / (((1 + k * k) * mu * mu + L.C1) * ((1 + k * k) * var + L.C2)))
    assert np.abs(s - want).max() < 1e-11  # zero padding scales with x: exact everywhere
    # symmetric in its two arguments
    y = rng.uniform(size=(H, W))
    assert np.abs(L.ssim_map(x, y) - L.ssim_map(y, x)).max() < 1e-14


def test_l2_term_closed_form():
    rng = np.random.default_rng(4)
    y = _img(rng, 15, 13)
    d = 0.25
    # lambda = 0 leaves the mean squared error only
    assert abs(L.loss(y + d, y, lam=0.0) - d * d) < 1e-14
    g = L.loss_grad(y + d, y, lam=0.0)
    assert np.abs(g - 2 * d / y.size).max() < 1e-16
    # lambda = 1 leaves 1 - SSIM
    x = _img(rng, 15, 13)
    assert abs(L.loss(x, y, lam=1.0) - (1.0 - L.ssim(x, y))) < 1e-14


@pytest.mark.parametrize("lam", [0.2, 1.0])
def test_gradient_matches_central_differences(lam):
    rng = np.random.default_rng(5)
    H, W = 19, 16
    x, y = _img(rng, H, W), _img(rng, H, W)
    # smooth the target so the two images share structure (covariance terms live)
    y = 0.5 * y + 0.5 * x
    g = L.loss_grad(x, y, lam)
    h = 1e-6
    picks = [(0, 0, 0), (H - 1, W - 1, 2), (0, W - 1, 1), (H // 2, W // 2, 0), (4, 5, 1), (5, 4, 2)]
    picks += [tuple(v) for v in zip(rng.integers(0, H, 30), rng.integers(0, W, 30), rng.integers(0, 3, 30))]
    gmax = np.abs(g).max()
    for i, j, c in picks:
        xp, xm = x.copy(), x.copy()
        xp[i, j, c] += h
        xm[i, j, c] -= h
        num = (L.loss(xp, y, lam) - L.loss(xm, y, lam)) / (2 * h)
        err = abs(g[i, j, c] - num) / max(abs(num), 1e-3 * gmax)
        assert err < 1e-6, (i, j, c, g[i, j, c], num)
