"""Pins of the oracle's SH basis, losses, re-projection term, Adam and SE(3) map.

* SH: orthonormality over the sphere by exact quadrature (Gauss-Legendre in
  cos(theta) x uniform in phi); degree 0 is the constant 1/(2 sqrt(pi)).
* L1 losses and the filter gate G(p) (Sec. 3.3): finite differences, and gate
  cases built by hand.
* Re-projection loss, Eq. lba (Sec. 3.2): zero at the true pose without noise,
  twist gradient vs central differences through Exp(xi) E_t.
* Adam against torch.optim.Adam; SE(3) exponential against scipy.linalg.expm.
"""
import math

import numpy as np
import pytest
import scipy.linalg
import torch

import oracle
import scenes


def test_sh_basis_is_orthonormal():
    nt, nphi = 24, 48
    x, wx = np.polynomial.legendre.leggauss(nt)  # cos(theta)
    phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    dirs = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    w = (wx[:, None] * np.full(nphi, 2 * np.pi / nphi)[None, :]).reshape(-1)
    Y = oracle.sh_eval(dirs, 3)
    G = (Y * w[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)
    np.testing.assert_allclose(oracle.sh_eval(dirs[:5], 0)[:, 0], 0.5 / math.sqrt(math.pi))
    # degree 1 is proportional to the direction itself
    Y1 = oracle.sh_eval(dirs[:50], 1)
    np.testing.assert_allclose(Y1[:, [3, 1, 2]] / math.sqrt(3 / (4 * math.pi)), dirs[:50], atol=1e-14)


def test_degree0_colour_is_the_generated_colour():
    c = scenes.config(1, scale=0.1)
    sc = c["scene"]
    geom = oracle.project_geom(sc, c["cams"])
    proj = oracle.project64(sc, c["cams"], geom)
    vis = geom["radius"] > 0
    colour = scenes.SH_C0 * sc["sh"][:, 0, :].astype(np.float64) + 0.5
    np.testing.assert_allclose(proj[vis, 7:10], colour[vis], rtol=1e-6, atol=1e-7)


def test_l1_loss_value_gradient_and_gate():
    rng = np.random.default_rng(0)
    P = 200
    img = dict(rgb=rng.uniform(0, 1, (P, 3)), depth=rng.uniform(0.5, 3, P), alpha=rng.uniform(0.9, 1, P))
    t_rgb, t_depth = rng.uniform(0, 1, (P, 3)), rng.uniform(0.5, 3, P)
    L, dC, dD = oracle.loss_l1(img, t_rgb, t_depth, w_c=0.7, w_d=0.3)
    for k in range(20):
        p, ch = int(rng.integers(P)), int(rng.integers(3))
        h = 1e-7
        for arr, grad, idx in ((img["rgb"], dC, (p, ch)), (img["depth"], dD, (p,))):
            old = arr[idx]
            arr[idx] = old + h
            Lp = oracle.loss_l1(img, t_rgb, t_depth, w_c=0.7, w_d=0.3)[0]
            arr[idx] = old - h
            Lm = oracle.loss_l1(img, t_rgb, t_depth, w_c=0.7, w_d=0.3)[0]
            arr[idx] = old
            assert abs((Lp - Lm) / (2 * h) - grad[idx]) < 1e-7
    # the value is the mean absolute error over pixel-channels and pixels
    assert L == pytest.approx(0.7 * np.abs(img["rgb"] - t_rgb).mean() + 0.3 * np.abs(img["depth"] - t_depth).mean(),
                              rel=1e-12)
    # gate: D^ > 0, D > 0 and A > gamma
    img = dict(rgb=np.full((4, 3), 0.5), depth=np.array([1.0, 0.0, 1.0, 1.0]),
               alpha=np.array([0.995, 0.995, 0.98, 0.995]))
    t_rgb = np.zeros((4, 3))
    t_depth = np.array([2.0, 2.0, 2.0, 0.0])
    L, dC, dD = oracle.loss_l1(img, t_rgb, t_depth, w_c=0.5, w_d=1.0, gate=True, gamma=0.99)
    assert np.all(dC[1:] == 0) and np.all(dD[1:] == 0)
    np.testing.assert_allclose(dC[0], 0.5 / 12)
    assert dD[0] == pytest.approx(-1.0 / 4)
    assert L == pytest.approx(0.5 * 1.5 / 12 + 1.0 / 4)


def _reproj_case(seed, noise):
    rng = np.random.default_rng(seed)
    vm = scenes.look_at((0.3, -0.2, 0.1), (0.0, 0.2, 3.0))
    cams = scenes.cams_from([[525.0, 525.0, 320.0, 240.0]], [[640, 480]], vm[None])
    px, py = scenes.keypoint_pixels(seed, 640, 480, 300)
    depth = rng.uniform(1.0, 4.0, 640 * 480)
    pts, ok = scenes.backproject(vm, cams["intr"][0], px, py, depth, 640)
    obs = np.stack([px + 0.5, py + 0.5], 1) + rng.normal(0, noise, (300, 2))
    return cams, pts[ok].astype(np.float64), obs[ok]


def test_reprojection_zero_at_true_pose():
    cams, pts, obs = _reproj_case(1, 0.0)
    L, g = oracle.reproj(pts, obs, cams)
    assert L < 1e-9


def test_reprojection_gradient_matches_central_differences():
    cams, pts, obs = _reproj_case(2, 1.0)
    L, g = oracle.reproj(pts, obs, cams, weight=1.5)
    E0 = cams["viewmats"][0].astype(np.float64)
    for k in range(6):
        h = 1e-7
        xi = np.zeros(6)
        xi[k] = h
        Lp = oracle.reproj(pts, obs, dict(cams, viewmats=oracle.se3_exp_apply(xi, E0)[None]), weight=1.5)[0]
        xi[k] = -h
        Lm = oracle.reproj(pts, obs, dict(cams, viewmats=oracle.se3_exp_apply(xi, E0)[None]), weight=1.5)[0]
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[0, k]) <= 1e-6 * max(1.0, abs(g[0, k])), (k, fd, g[0, k])


def test_adam_matches_torch():
    rng = np.random.default_rng(4)
    n = 64
    p = rng.standard_normal(n)
    m, v = np.zeros(n), np.zeros(n)
    tp = torch.tensor(p.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-2, betas=(0.9, 0.999), eps=1e-15)
    for t in range(1, 6):
        g = rng.standard_normal(n)
        oracle.adam(p, g, m, v, lr=1e-2, b1=0.9, b2=0.999, eps=1e-15, t=t)
        tp.grad = torch.tensor(g)
        opt.step()
        np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("scale", [1.0, 1e-7])
def test_se3_exp_matches_matrix_exponential(scale):
    rng = np.random.default_rng(5)
    for _ in range(5):
        xi = rng.standard_normal(6) * scale
        rho, ph = xi[:3], xi[3:]
        X = np.zeros((4, 4))
        X[:3, :3] = [[0, -ph[2], ph[1]], [ph[2], 0, -ph[0]], [-ph[1], ph[0], 0]]
        X[:3, 3] = rho
        Tm = scipy.linalg.expm(X)
        E = np.concatenate([np.eye(3), np.zeros((3, 1))], 1)
        np.testing.assert_allclose(oracle.se3_exp_apply(xi, E), Tm[:3], atol=1e-14, rtol=1e-12)
        E2 = rng.standard_normal((3, 4))
        full = Tm @ np.vstack([E2, [0, 0, 0, 1]])
        np.testing.assert_allclose(oracle.se3_exp_apply(xi, E2), full[:3], atol=1e-13, rtol=1e-12)


def test_keyframe_decoding_is_correctly_rounded():
    """Every colour byte maps to the FP32 number nearest c/255 (checked in
    exact rational arithmetic against both FP32 neighbours), and depths to the
    FP32 product, with the closed values 0 -> 0 and 255 -> 1."""
    from fractions import Fraction
    c = np.arange(256, dtype=np.uint8)
    rgb, depth = oracle.decode_keyframes(np.stack([c, c, c], 1), np.array([0, 5000, 65535], np.uint16), 1 / 5000)
    assert rgb.dtype == np.float32 and depth.dtype == np.float32
    assert rgb[0, 0] == 0.0 and rgb[255, 2] == 1.0
    for k in range(256):
        x = rgb[k, 0]
        exact = Fraction(k, 255)
        err = abs(Fraction(float(x)) - exact)
        for nb in (np.nextafter(x, np.float32(-1)), np.nextafter(x, np.float32(2))):
            assert err <= abs(Fraction(float(nb)) - exact), k
    s = np.float32(1 / 5000)
    assert depth[0] == 0.0
    assert depth[1] == np.float32(np.float32(5000) * s) and abs(float(depth[1]) - 1.0) < 1e-6
    assert depth[2] == np.float32(np.float32(65535) * s)
