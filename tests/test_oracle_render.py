"""Pins of the oracle's compositing (Sec. 3.4 C(p), D(p); Sec. 3.3 M_b(p)).

* invariants: alpha (border mask) and transmittance in [0, 1], transmittance
  never rises along a ray, A = 1 - T, C and D bounded by the blend weights;
* invariance of the image to the input order of the Gaussians;
* brute force: per pixel, the Gaussians whose rectangle covers the pixel's tile,
  sorted by (float32 depth, index), composited in plain Python from an
  independent numpy projection (scipy rotations, numerical Jacobian).
"""
import numpy as np

import oracle
import scenes
from helpers import project_bruteforce


def test_invariants_and_monotone_transmittance():
    c = scenes.config(1, scale=0.25)
    cams = c["cams"]
    fwd = oracle.forward(c["scene"], cams)
    img, bins, proj = fwd["img"], fwd["bins"], fwd["proj"]
    n = fwd["geom"]["n"]
    A, T = img["alpha"], img["final_T"]
    assert np.all((A >= 0) & (A <= 1)) and np.all((T > 0) & (T <= 1))
    np.testing.assert_allclose(A, 1 - T, atol=0)
    assert np.all(T >= oracle.T_MIN)
    # C <= max colour * A and z_min A <= D <= z_max A
    vis = fwd["geom"]["radius"] > 0
    cmax = proj[vis, 7:10].max()
    zmin, zmax = proj[vis, 2].min(), proj[vis, 2].max()
    assert np.all(img["rgb"] <= cmax * A[:, None] + 1e-12)
    assert np.all(img["depth"] <= zmax * A + 1e-12) and np.all(img["depth"] >= zmin * A - 1e-12)
    # transmittance after the first k list entries never rises with k
    ranges = bins["ranges"]
    maxlen = int((ranges[:, 1] - ranges[:, 0]).max())
    prev = np.ones_like(T)
    for k in [1, 2, 3, 5, 8, 13, 21, 34, 55, 89, maxlen]:
        cut = dict(bins, ranges=np.stack([ranges[:, 0], np.minimum(ranges[:, 1], ranges[:, 0] + k)], 1)
                   .astype(np.uint32).copy())
        Tk = oracle.render(cams, proj, fwd["drec"], cut, n)["final_T"]
        assert np.all(Tk <= prev + 1e-15) and np.all((Tk > 0) & (Tk <= 1))
        prev = Tk
    np.testing.assert_array_equal(prev, T)


def test_image_invariant_to_input_order():
    c = scenes.config(1, scale=0.5)
    scene, cams = c["scene"], c["cams"]
    fwd = oracle.forward(scene, cams)
    perm = np.random.default_rng(5).permutation(scene["means"].shape[0])
    ps = {k: (v[perm] if isinstance(v, np.ndarray) else v) for k, v in scene.items()}
    fwd2 = oracle.forward(ps, cams)
    z = fwd["geom"]["uvz"][:, 2][fwd["geom"]["radius"] > 0]
    assert len(np.unique(z)) == len(z)  # distinct depths: order fully fixed
    for k in ("rgb", "depth", "alpha", "final_T"):
        np.testing.assert_allclose(fwd2["img"][k], fwd["img"][k], rtol=0, atol=1e-14)
    np.testing.assert_array_equal(fwd2["img"]["n_contrib"], fwd["img"]["n_contrib"])


def _composite_bruteforce(scene, cams, geom, blur):
    intr, vm = cams["intr"][0], cams["viewmats"][0]
    W, H = (int(v) for v in cams["size"][0])
    pr = project_bruteforce(scene, intr, vm, blur)
    col = scenes.SH_C0 * np.asarray(scene["sh"][:, 0, :], np.float64) + 0.5
    zb = geom["uvz"][:, 2].view(np.uint32)
    rgb = np.zeros((H * W, 3))
    dep = np.zeros(H * W)
    alp = np.zeros(H * W)
    vis = np.nonzero(geom["radius"] > 0)[0]
    for py in range(H):
        for px in range(W):
            tx, ty = px // 16, py // 16
            cand = [i for i in vis if geom["rect"][i, 0] <= tx <= geom["rect"][i, 2]
                    and geom["rect"][i, 1] <= ty <= geom["rect"][i, 3]]
            cand.sort(key=lambda i: (int(zb[i]), int(i)))
            T, C, D = 1.0, np.zeros(3), 0.0
            for i in cand:
                d = np.array([px + 0.5, py + 0.5]) - pr[i]["uv"]
                a = pr[i]["o"] * np.exp(-0.5 * d @ np.linalg.solve(pr[i]["cov"], d))
                a = min(a, 0.99)
                if a < 1 / 255:
                    continue
                if T * (1 - a) < 1e-4:
                    break
                C += col[i] * a * T
                D += pr[i]["z"] * a * T
                T *= 1 - a
            rgb[py * W + px], dep[py * W + px], alp[py * W + px] = C, D, 1 - T
    return rgb, dep, alp


def test_bruteforce_per_pixel_compositing():
    c = scenes.config(1, scale=0.02)  # 40 Gaussians
    scene, cams = c["scene"], c["cams"]
    assert scene["means"].shape[0] <= 50
    # the brute force decides in FP64, the oracle on its FP32 l2 (within
    # 2e-6 (1 + M) of log2 alpha): pixels with an FP64 alpha within 1e-5 of a
    # cut are left out
    fwd = oracle.forward(scene, cams, blur=0.3, margin_alpha=1e-5)
    rgb, dep, alp = _composite_bruteforce(scene, cams, fwd["geom"], 0.3)
    img = fwd["img"]
    keep = img["flags"] == 0
    assert keep.mean() > 0.99
    # the numerical Jacobian in the brute force limits agreement to ~1e-8
    np.testing.assert_allclose(img["rgb"][keep], rgb[keep], atol=1e-7)
    np.testing.assert_allclose(img["depth"][keep], dep[keep], atol=1e-6)
    np.testing.assert_allclose(img["alpha"][keep], alp[keep], atol=1e-7)
    assert np.abs(img["alpha"]).sum() > 10  # the scene is not empty


def test_empty_scene_and_empty_tiles():
    cams = scenes.pinhole(40, 24, 30.0)  # ragged: 3 x 2 tiles, partial edge tiles
    scene = scenes.cube_scene(3, seed=9)
    scene["means"][:] = [0.0, 0.0, -5.0]  # all behind the camera
    fwd = oracle.forward(scene, cams)
    assert fwd["bins"]["n_pairs"] == 0
    assert np.all(fwd["img"]["alpha"] == 0) and np.all(fwd["img"]["final_T"] == 1)
    assert np.all(fwd["img"]["n_contrib"] == 0)
