"""Pins of the SSIM term of the mapping loss (Sec. 3.4 L_m, zeta = 0.3).

* brute force: the SSIM map of a small image from explicit window sums;
* SSIM(x, x) = 1; constant images give (2ab + C1) / (a^2 + b^2 + C1) away
  from the border;
* the gradient against central finite differences of the loss.
"""
import numpy as np
import pytest

from oracle import ssim as S


def _brute(x, y):
    H, W = x.shape
    g = S.window()
    w2 = np.outer(g, g)
    r = S.WIN // 2
    out = np.zeros((H, W))
    for i in range(H):
        for j in range(W):
            mx = my = ex2 = ey2 = exy = 0.0
            for a in range(-r, r + 1):
                for b in range(-r, r + 1):
                    ii, jj = i + a, j + b
                    if 0 <= ii < H and 0 <= jj < W:
                        wt = w2[a + r, b + r]
                        X, Y = x[ii, jj], y[ii, jj]
                        mx += wt * X
                        my += wt * Y
                        ex2 += wt * X * X
                        ey2 += wt * Y * Y
                        exy += wt * X * Y
            sx2, sy2, sxy = ex2 - mx * mx, ey2 - my * my, exy - mx * my
            out[i, j] = ((2 * mx * my + S.C1) * (2 * sxy + S.C2)) / ((mx * mx + my * my + S.C1) * (sx2 + sy2 + S.C2))
    return out


def test_window_is_normalised_gaussian():
    g = S.window()
    assert len(g) == 11 and abs(g.sum() - 1) < 1e-15
    assert g[5] == g.max() and np.allclose(g, g[::-1])
    assert g[4] / g[5] == pytest.approx(np.exp(-1 / (2 * 1.5 ** 2)), rel=1e-14)


def test_ssim_map_matches_brute_force():
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 1, (13, 17, 3))
    y = np.clip(x + rng.normal(0, 0.1, x.shape), 0, 1)
    s, *_ = S.ssim_view(x, y)
    for ch in range(3):
        np.testing.assert_allclose(s[..., ch], _brute(x[..., ch], y[..., ch]), rtol=1e-10, atol=1e-12)


def test_identity_and_constant_images():
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, (20, 24, 3))
    s, *_ = S.ssim_view(x, x)
    np.testing.assert_allclose(s, 1.0, atol=1e-12)
    a, b = 0.3, 0.7
    s, *_ = S.ssim_view(np.full((30, 30, 3), a), np.full((30, 30, 3), b))
    inner = s[5:-5, 5:-5]
    np.testing.assert_allclose(inner, (2 * a * b + S.C1) / (a * a + b * b + S.C1), rtol=1e-12)


def test_ssim_gradient_matches_central_differences():
    rng = np.random.default_rng(2)
    size = np.array([[9, 7], [6, 5]])
    P = int((size[:, 0] * size[:, 1]).sum())
    x = rng.uniform(0.1, 0.9, (P, 3))
    y = rng.uniform(0.1, 0.9, (P, 3))
    L, g = S.loss_ssim(x, y, size, weight=0.3)
    for _ in range(25):
        p, ch = int(rng.integers(P)), int(rng.integers(3))
        h = 1e-6
        x[p, ch] += h
        Lp = S.loss_ssim(x, y, size, weight=0.3)[0]
        x[p, ch] -= 2 * h
        Lm = S.loss_ssim(x, y, size, weight=0.3)[0]
        x[p, ch] += h
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[p, ch]) <= 1e-7 * max(1.0, abs(g[p, ch])) + 1e-10, (p, ch, fd, g[p, ch])
