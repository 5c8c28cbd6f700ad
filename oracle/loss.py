"""FP64 oracle of the photometric training loss of Sec. 3.3 (Eq. 9):
L = (1 - lambda) L2 + lambda L_D-SSIM with lambda = 0.2, and its gradient
dL/dC with respect to the rendered image C, the input of the backward pass.

TEST INFRASTRUCTURE: imported only by tests/ and by the CPU legs of bench.py.
The CUDA library never imports it, and it shares no code with it.

The paper names the two terms but not their constants; the readings taken
here (the loss 3DGS trains with, which the paper builds on):
  * L2 is the mean over the image's H * W * 3 values of (C - C_gt)^2;
  * L_D-SSIM = 1 - SSIM, SSIM the mean over pixels and channels of the SSIM
    map of Wang et al. (2004): local means, variances and covariance taken
    with an 11 x 11 Gaussian window (sigma 1.5, weights normalised to sum to
    one), each colour channel on its own, values outside the image counted
    as zero, C1 = 0.01^2 and C2 = 0.03^2 (dynamic range 1).
Images are [H, W, 3] arrays, one per view.

Everything is written straight from those definitions: the windowed sums are
121 shifted, weighted copies of the zero-padded image, and the gradient is
the chain rule through them, the window's adjoint written out as the
scatter it is.
"""
import numpy as np

RADIUS = 5
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2
LAMBDA = 0.2


def gauss_window():
    """The 11 x 11 window: outer product of the sampled, normalised 1-D Gaussian."""
    t = np.arange(-RADIUS, RADIUS + 1, dtype=np.float64)
    g = np.exp(-t * t / (2.0 * SIGMA * SIGMA))
    g /= g.sum()
    return np.outer(g, g)


def window_filter(img):
    """out[p] = sum_d K[d] img[p + d] over the window, img zero outside [H, W]."""
    H, W = img.shape
    K = gauss_window()
    R = RADIUS
    pad = np.zeros((H + 2 * R, W + 2 * R))
    pad[R:R + H, R:R + W] = img
    out = np.zeros((H, W))
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            out += K[dy + R, dx + R] * pad[R + dy:R + dy + H, R + dx:R + dx + W]
    return out


def window_filter_adjoint(m):
    """Adjoint of window_filter: img_bar[q] = sum over p of K[q - p] m[p]."""
    H, W = m.shape
    K = gauss_window()
    R = RADIUS
    pad = np.zeros((H + 2 * R, W + 2 * R))
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            pad[R + dy:R + dy + H, R + dx:R + dx + W] += K[dy + R, dx + R] * m
    return pad[R:R + H, R:R + W]


def _moments(x, y):
    mx, my = window_filter(x), window_filter(y)
    sxx = window_filter(x * x) - mx * mx
    syy = window_filter(y * y) - my * my
    sxy = window_filter(x * y) - mx * my
    return mx, my, sxx, syy, sxy


def ssim_map(x, y):
    """Per-pixel SSIM of two single-channel images [H, W]."""
    mx, my, sxx, syy, sxy = _moments(np.asarray(x, np.float64), np.asarray(y, np.float64))
    return ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))


def ssim(img, gt):
    """Mean SSIM over pixels and channels of two [H, W, 3] images."""
    img, gt = np.asarray(img, np.float64), np.asarray(gt, np.float64)
    return float(np.mean([ssim_map(img[..., c], gt[..., c]).mean() for c in range(img.shape[2])]))


def loss(img, gt, lam=LAMBDA):
    """Eq. 9 for one view: (1 - lam) * L2 + lam * (1 - SSIM)."""
    img, gt = np.asarray(img, np.float64), np.asarray(gt, np.float64)
    l2 = float(np.mean((img - gt) ** 2))
    return (1.0 - lam) * l2 + lam * (1.0 - ssim(img, gt))


def loss_grad(img, gt, lam=LAMBDA):
    """dL/dC of Eq. 9 for one view, [H, W, 3].

    Per channel, with mu_x = F x, B = F x^2 and X = F (x y) (F the window
    filter), SSIM's pixel value s = N / D with
      N = (2 mu_x mu_y + C1) (2 (X - mu_x mu_y) + C2),
      D = (mu_x^2 + mu_y^2 + C1) (B - mu_x^2 + F y^2 - mu_y^2 + C2),
    so ds/dmu_x = (dN/dmu_x - s dD/dmu_x) / D, ds/dB = -s / (B - mu_x^2 + ...),
    ds/dX = 2 (2 mu_x mu_y + C1) / D; the chain rule through F takes them
    back to the pixels: dS/dx = F^T a + 2 x F^T b + y F^T c (over the pixel
    count), and the L2 term adds 2 (x - y) over the value count.
    """
    img, gt = np.asarray(img, np.float64), np.asarray(gt, np.float64)
    H, W, nc = img.shape
    n = H * W * nc
    out = np.empty_like(img)
    for c in range(nc):
        x, y = img[..., c], gt[..., c]
        mx, my, sxx, syy, sxy = _moments(x, y)
        l1, cs1 = 2 * mx * my + C1, 2 * sxy + C2
        l2, cs2 = mx * mx + my * my + C1, sxx + syy + C2
        Nm, D = l1 * cs1, l2 * cs2
        s = Nm / D
        dN = 2 * my * cs1 + l1 * (-2 * my)
        dD = 2 * mx * cs2 + l2 * (-2 * mx)
        a = (dN - s * dD) / D
        b = -s / cs2
        cc = 2 * l1 / D
        dssim = (window_filter_adjoint(a) + 2 * x * window_filter_adjoint(b)
                 + y * window_filter_adjoint(cc)) / n
        out[..., c] = (1.0 - lam) * 2.0 * (x - y) / n - lam * dssim
    return out
