"""Pins of the oracle's projection and binning against facts fixed outside it.

* Sec. 3.4 "Projection": mu2D = K E_t mu / d and r2D = f r / d for an isotropic
  Gaussian; the EWA footprint reduces to that on the optical axis.
* The EWA covariance J W S W^T J^T is checked against scipy rotations and a
  numerical Jacobian of the pinhole map.
* Support radius and tile rectangle: every excluded tile lies beyond three
  standard deviations; the rectangle is the smallest covering the square.
* Front-to-back order (Sec. 3.4 "Differentiable Rasterization").
"""
import math

import numpy as np
import pytest

import oracle
import scenes
from helpers import pinhole_jacobian_numeric, rotation_from_quat


def test_geom_expf_within_one_ulp():
    rng = np.random.default_rng(0)
    xs = np.concatenate([np.linspace(-80, 80, 4001), rng.uniform(-12, 4, 4000)]).astype(np.float32)
    for x in xs:
        y = oracle.geom_expf(float(x))
        t = math.exp(float(x))
        assert abs(y - t) <= 1.0 * float(np.spacing(np.float32(t))), x
    assert oracle.geom_expf(0.0) == 1.0


def _iso_scene(z, s, o, col, q=(1.0, 0.0, 0.0, 0.0)):
    sh = np.zeros((1, 1, 3), np.float32)
    sh[0, 0] = (np.asarray(col) - 0.5) / scenes.SH_C0
    return dict(means=np.array([[0.0, 0.0, z]], np.float32),
                log_scales=np.full((1, 3), math.log(s), np.float32),
                quats=np.array([q], np.float32), opacity_logit=np.array([math.log(o / (1 - o))], np.float32),
                sh=sh, sh_degree=0)


@pytest.mark.parametrize("blur", [0.0, 0.3])
@pytest.mark.parametrize("q", [(1.0, 0.0, 0.0, 0.0), (0.3, -0.5, 0.7, 0.2)])
def test_isotropic_on_axis_closed_form(blur, q):
    """One isotropic Gaussian on the optical axis renders as
    o exp(-|p - c|^2 / (2 (f^2 s^2 / z^2 + blur))), with r2D = f s / z."""
    f, W, H, z, s, o = 60.0, 64, 48, 3.0, 0.05, 0.8
    col = (0.2, 0.6, 0.9)
    scene = _iso_scene(z, s, o, col, q)
    cams = scenes.pinhole(W, H, f)
    fwd = oracle.forward(scene, cams, blur=blur)
    # the scene stores float32 log-scale and logit: use the values they hold
    s = math.exp(float(scene["log_scales"][0, 0]))
    o = 1.0 / (1.0 + math.exp(-float(scene["opacity_logit"][0])))
    col = scenes.SH_C0 * scene["sh"][0, 0].astype(np.float64) + 0.5
    var = (f * s / z) ** 2 + blur
    assert fwd["geom"]["radius"][0] == math.ceil(3 * math.sqrt(var) - 1e-9)
    px, py = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    d2 = (px - W / 2) ** 2 + (py - H / 2) ** 2
    a = o * np.exp(-d2 / (2 * var))
    a = np.minimum(a, 0.99)
    a[a < 1 / 255] = 0.0
    # only pixels inside the rectangle of touched tiles can be reached
    x0, y0, x1, y1 = fwd["geom"]["rect"][0]
    tx, ty = (px // 16).astype(int), (py // 16).astype(int)
    inside = (tx >= x0) & (tx <= x1) & (ty >= y0) & (ty <= y1)
    a[~inside] = 0.0
    img = fwd["img"]
    keep = (img["flags"] == 0).reshape(H, W)
    assert keep.mean() > 0.98
    np.testing.assert_allclose(img["alpha"].reshape(H, W)[keep], a[keep], rtol=1e-12, atol=1e-13)
    for ch in range(3):
        np.testing.assert_allclose(img["rgb"][:, ch].reshape(H, W)[keep], col[ch] * a[keep],
                                   rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(img["depth"].reshape(H, W)[keep], z * a[keep], rtol=1e-12, atol=1e-12)


def test_ewa_covariance_matches_scipy_rotation_and_numeric_jacobian():
    c = scenes.config(1, scale=0.02)
    scene = c["scene"]
    # an oblique camera so that the world-to-camera rotation matters
    vm = scenes.look_at((0.7, -0.4, -0.5), (0.1, 0.2, 3.0))
    cams = scenes.pinhole(64, 48, 60.0, viewmats=vm[None])
    geom = oracle.project_geom(scene, cams)
    proj = oracle.project64(scene, cams, geom, blur=0.3)
    E = vm.astype(np.float64)
    Wr, t = E[:, :3], E[:, 3]
    R = rotation_from_quat(scene["quats"])
    s = np.exp(scene["log_scales"].astype(np.float64))
    checked = 0
    for i in np.nonzero(geom["radius"])[0]:
        if proj[i, 13] or proj[i, 14]:
            continue
        p = Wr @ scene["means"][i].astype(np.float64) + t
        J = pinhole_jacobian_numeric(p, 60.0, 60.0)
        S2 = J @ Wr @ (R[i] @ np.diag(s[i] ** 2) @ R[i].T) @ Wr.T @ J.T + 0.3 * np.eye(2)
        np.testing.assert_allclose(proj[i, 10:13], [S2[0, 0], S2[0, 1], S2[1, 1]], rtol=1e-7,
                                   atol=1e-9 * S2[0, 0])
        np.testing.assert_allclose(proj[i, 0:3], [60 * p[0] / p[2] + 32, 60 * p[1] / p[2] + 24, p[2]],
                                   rtol=1e-12)
        conic = np.linalg.inv(S2)
        np.testing.assert_allclose(proj[i, 3:6], [conic[0, 0], conic[0, 1], conic[1, 1]], rtol=1e-6,
                                   atol=1e-9 * abs(conic[0, 0]))
        checked += 1
    assert checked >= 20


def test_fp32_geometry_agrees_with_fp64():
    c = scenes.config(1)
    geom = oracle.project_geom(c["scene"], c["cams"])
    proj = oracle.project64(c["scene"], c["cams"], geom)
    vis = geom["radius"] > 0
    np.testing.assert_allclose(geom["uvz"][vis], proj[vis, 0:3], rtol=2e-6, atol=2e-4)
    a, b, cc = proj[vis, 10], proj[vis, 11], proj[vis, 12]
    mid = 0.5 * (a + cc)
    lam = mid + np.sqrt(np.maximum(mid * mid - (a * cc - b * b), 0))
    r64 = 3 * np.sqrt(lam)
    frac = r64 - np.floor(r64)
    clear = (frac > 1e-3) & (frac < 1 - 1e-3)
    assert clear.mean() > 0.95
    np.testing.assert_array_equal(geom["radius"][vis][clear], np.ceil(r64[clear]).astype(np.int32))


def test_excluded_tiles_lie_beyond_three_sigma_and_rect_is_tight():
    c = scenes.config(1, scale=0.05)
    cams = c["cams"]
    geom = oracle.project_geom(c["scene"], cams)
    proj = oracle.project64(c["scene"], cams, geom)
    W, H = 64, 48
    px, py = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    tx, ty = (px // 16).astype(int), (py // 16).astype(int)
    n_checked = 0
    for i in np.nonzero(geom["radius"])[0]:
        a, b, cc = proj[i, 10:13]
        Sinv = np.linalg.inv(np.array([[a, b], [b, cc]]))
        dx, dy = px - proj[i, 0], py - proj[i, 1]
        maha = Sinv[0, 0] * dx * dx + 2 * Sinv[0, 1] * dx * dy + Sinv[1, 1] * dy * dy
        x0, y0, x1, y1 = geom["rect"][i]
        inside = (tx >= x0) & (tx <= x1) & (ty >= y0) & (ty <= y1)
        if (~inside).any():
            assert maha[~inside].min() > 9.0 * (1 - 1e-5)
        # tightness: the unclamped rectangle edges contain u -/+ r and v -/+ r
        u, v = geom["uvz"][i, 0], geom["uvz"][i, 1]
        r = geom["radius"][i]
        if x0 > 0:
            assert x0 * 16 <= u - r < (x0 + 1) * 16
        if x1 < 3:
            assert x1 * 16 <= u + r < (x1 + 1) * 16
        if y0 > 0:
            assert y0 * 16 <= v - r < (y0 + 1) * 16
        if y1 < 2:
            assert y1 * 16 <= v + r < (y1 + 1) * 16
        n_checked += 1
    assert n_checked > 50


def test_culling_rules():
    cams = scenes.pinhole(64, 48, 60.0)
    scene = _iso_scene(3.0, 0.05, 0.5, (0.5, 0.5, 0.5))
    for z, visible in [(0.1, False), (0.2, False), (0.2001, True), (-3.0, False)]:
        sc = dict(scene, means=np.array([[0.0, 0.0, z]], np.float32))
        assert (oracle.project_geom(sc, cams)["radius"][0] > 0) == visible, z
    # far outside the image: no tile touched
    sc = dict(scene, means=np.array([[30.0, 0.0, 3.0]], np.float32))
    assert oracle.project_geom(sc, cams)["radius"][0] == 0
    # a zero quaternion is culled
    sc = dict(scene, quats=np.zeros((1, 4), np.float32))
    assert oracle.project_geom(sc, cams)["radius"][0] == 0


def test_binning_is_front_to_back_per_tile():
    c = scenes.config(1)
    cams = c["cams"]
    geom = oracle.project_geom(c["scene"], cams, tile_cull=False)
    bins = oracle.bin_tiles(cams, geom)
    keys, vals, ranges = bins["keys"], bins["vals"], bins["ranges"]
    assert bins["n_pairs"] == int(geom["tiles_touched"].sum())
    # every (Gaussian, tile) pair of the rectangles appears once, under the right tile
    expect = set()
    for i in np.nonzero(geom["radius"])[0]:
        x0, y0, x1, y1 = geom["rect"][i]
        for ty in range(y0, y1 + 1):
            for tx in range(x0, x1 + 1):
                expect.add((ty * 4 + tx, int(i)))
    got = set(zip((keys >> np.uint64(32)).astype(int).tolist(), vals.astype(int).tolist()))
    assert got == expect and len(got) == len(keys)
    # keys ascending; within a tile depth bits ascending, ties by index
    z = geom["uvz"][:, 2].view(np.uint32)
    for t in range(bins["n_tiles"]):
        b, e = ranges[t]
        ids = vals[b:e]
        assert np.all((keys[b:e] >> np.uint64(32)) == t)
        assert np.all((keys[b:e] & np.uint64(0xFFFFFFFF)) == z[ids])
        order = np.lexsort((ids, z[ids]))
        np.testing.assert_array_equal(order, np.arange(len(ids)))
    assert ranges[-1, 1] == len(keys)


def test_tile_cull_drops_only_tiles_no_pixel_blends():
    """The exact tile test (rectangles of up to 64 tiles) removes a pair only
    where the splat's FP32 log2 alpha is below log2(1/255) at every pixel of
    the tile (checked by brute force over the tile's pixels); the lists keep
    every other pair in the same order, so the FP64 images are bit-identical
    with and without the test; and it removes a good share of the pairs."""
    for tile in [(16, 16), (32, 16), (8, 8)]:
        sc = scenes.cube_scene(1500, seed=44, sh_degree=0, log_scale=(-3.0, 0.6), opacity=(-1.0, 1.5))
        cams = scenes.pinhole(96, 80, 70.0)
        W, H = 96, 80
        full = oracle.forward(sc, cams, tile=tile, tile_cull=False)
        cut = oracle.forward(sc, cams, tile=tile)
        for k in ("rgb", "depth", "alpha", "final_T"):
            np.testing.assert_array_equal(cut["img"][k], full["img"][k])
        pairs = lambda f: set(zip((f["bins"]["keys"] >> np.uint64(32)).astype(int).tolist(),
                                  f["bins"]["vals"].astype(int).tolist()))
        kept, every = pairs(cut), pairs(full)
        assert kept <= every
        dropped = every - kept
        assert len(dropped) > 0.1 * len(every), (len(dropped), len(every))
        ntx = (W + tile[0] - 1) // tile[0]
        drec = cut["drec"]
        for t, i in dropped:
            ty, tx = divmod(t, ntx)
            xs = np.arange(tx * tile[0], min((tx + 1) * tile[0], W))
            ys = np.arange(ty * tile[1], min((ty + 1) * tile[1], H))
            PX, PY = np.meshgrid(xs, ys)
            l2 = oracle.blend_l2(np.repeat(drec[i][None], PX.size, 0), PX.ravel(), PY.ravel())
            assert np.all(l2 < oracle.L2_ALPHA_MIN), (tile, t, i, float(l2.max()))
