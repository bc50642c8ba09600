"""SSIM term of the mapping loss (Sec. 3.4: L_m = (1 - zeta)(w4 L1(D) + w5 L1(C))
+ zeta L_SSIM, zeta = 0.3 in Table hyper), FP64 numpy.  Test infrastructure only.

The paper does not define its SSIM; this follows the usual structural
similarity index: per colour channel, local statistics under an 11 x 11
Gaussian window of standard deviation 1.5 (normalised to sum 1, zero padding at
the image border, same output size),

    s = (2 mu_x mu_y + C1)(2 sigma_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(sigma_x^2 + sigma_y^2 + C2)),

C1 = 0.01^2, C2 = 0.03^2, and L_SSIM = 1 - mean of s over pixels and channels
of all views.  x is the rendered image, y the target.

Gradient: with g = dL/ds = -weight / (3P) and the window G (symmetric),
    dL/dx = g [ G * ds/dmu_x + 2 x (G * ds/dE[x^2]) + y (G * ds/dE[xy]) ],
    ds/dmu_x   = (2 mu_y (a2 - a1) - 2 mu_x s (b2 - b1)) / (b1 b2),
    ds/dE[x^2] = -s / b2,     ds/dE[xy] = 2 a1 / (b1 b2),
where a1, a2, b1, b2 are the four factors of s and sigma_x^2 = E[x^2] - mu_x^2,
sigma_xy = E[xy] - mu_x mu_y.  Filtering uses scipy's correlate1d (a library
primitive) along rows then columns.
"""
from __future__ import annotations

import numpy as np
from scipy.ndimage import correlate1d

C1 = 0.01 ** 2
C2 = 0.03 ** 2
WIN = 11
SIGMA = 1.5


def window():
    i = np.arange(WIN) - WIN // 2
    g = np.exp(-(i * i) / (2 * SIGMA * SIGMA))
    return g / g.sum()


def _filt(img, g):
    return correlate1d(correlate1d(img, g, axis=0, mode="constant", cval=0.0), g, axis=1, mode="constant", cval=0.0)


def ssim_view(x, y):
    """SSIM map [H,W,3] and the three partial maps for one view (x, y: [H,W,3])."""
    g = window()
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    s = np.zeros_like(x)
    dmu, dx2, dxy = np.zeros_like(x), np.zeros_like(x), np.zeros_like(x)
    for ch in range(3):
        X, Y = x[..., ch], y[..., ch]
        mx, my = _filt(X, g), _filt(Y, g)
        ex2, ey2, exy = _filt(X * X, g), _filt(Y * Y, g), _filt(X * Y, g)
        sx2, sy2, sxy = ex2 - mx * mx, ey2 - my * my, exy - mx * my
        a1, a2 = 2 * mx * my + C1, 2 * sxy + C2
        b1, b2 = mx * mx + my * my + C1, sx2 + sy2 + C2
        sm = a1 * a2 / (b1 * b2)
        s[..., ch] = sm
        dmu[..., ch] = (2 * my * (a2 - a1) - 2 * mx * sm * (b2 - b1)) / (b1 * b2)
        dx2[..., ch] = -sm / b2
        dxy[..., ch] = 2 * a1 / (b1 * b2)
    return s, dmu, dx2, dxy


def loss_ssim(rgb, target_rgb, size, weight=1.0):
    """weight * (1 - mean SSIM) over all views (pixels concatenated as in the
    image layout, size [V,2] = (width, height)); returns (L, dL/drgb [P,3])."""
    rgb = np.asarray(rgb, np.float64)
    tgt = np.asarray(target_rgb, np.float64)
    P = rgb.shape[0]
    g = window()
    grad = np.zeros_like(rgb)
    total = 0.0
    base = 0
    for w, h in np.asarray(size, np.int64):
        w, h = int(w), int(h)
        x = rgb[base:base + w * h].reshape(h, w, 3)
        y = tgt[base:base + w * h].reshape(h, w, 3)
        s, dmu, dx2, dxy = ssim_view(x, y)
        total += s.sum()
        gs = -weight / (3.0 * P)
        gx = np.zeros_like(x)
        for ch in range(3):
            gx[..., ch] = gs * (_filt(dmu[..., ch], g) + 2 * x[..., ch] * _filt(dx2[..., ch], g)
                                + y[..., ch] * _filt(dxy[..., ch], g))
        grad[base:base + w * h] = gx.reshape(-1, 3)
        base += w * h
    L = weight * (1.0 - total / (3.0 * P))
    return L, grad
