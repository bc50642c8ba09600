"""Pins of the oracle's FP32 alpha decisions (Sec. 3.4 Eq. gauss and the
compositing's alpha rules: skip below 1/255, clamp at 0.99, stop before
T (1 - alpha) < 1e-4).

The oracle takes the skip and clamp decisions on l2, an FP32 evaluation of
log2 of the raw alpha o exp(-1/2 d^T conic d) by a stated operation order
(orc_blend_records, orc_blend_l2), and bounds the kernel's deviation at the
stop decision by a band.  Pinned here against computations independent of
that code:

* its log2 against numpy's FP64 log2;
* l2 against log2 alpha in FP64 from an independent numpy projection (scipy
  rotations, numerical Jacobian) at random (splat, pixel) points: within
  2e-6 (1 + M), M the magnitude of the quadratic form's terms in base 2;
* the skip and clamp decisions against the FP64 ones, at points placed
  within 3e-5 of both cuts: equal wherever FP64 is farther from its cut than
  that bound;
* l2 against a numpy float32 evaluation of the stated operation order (IEEE
  single precision, no contraction; fused multiply-adds rounded once);
* the transmittance band: the kernel's FP32 transmittance, emulated with the
  approximate exponential's error at its bound in the direction that moves T
  most, stays inside the band the oracle reports for every pixel; the widest
  band is within 2x of the largest such deviation, and on the widest tenth of
  the bands the median ratio to the pixel's own deviation is at most 3.
"""
from fractions import Fraction

import numpy as np

import oracle
import scenes
from helpers import project_bruteforce

LN2 = np.log(2.0)


def test_log2_by_its_own_method():
    rng = np.random.default_rng(3)
    y = np.concatenate([1.0 + rng.uniform(0, 1, 4000), np.exp(rng.uniform(0, 70, 4000)),
                        2.0 ** np.arange(0, 100), [1.0, np.sqrt(2.0), 1.4142134, 1.4142137]]).astype(np.float32)
    got = np.array([oracle.geom_log2f(v) for v in y], np.float64)
    ref = np.log2(y.astype(np.float64))
    ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(got - ref) <= 2 * ulp + 2e-8), np.max(np.abs(got - ref) / ulp)
    assert np.all(got[y == 2.0 ** np.round(np.log2(y))] == np.round(np.log2(y[y == 2.0 ** np.round(np.log2(y))])))


def _points(seed, n_pts, scene, cams):
    """Random (drawn splat, pixel inside its rectangle) pairs."""
    geom = oracle.project_geom(scene, cams)
    vis = np.nonzero(geom["radius"] > 0)[0]
    rng = np.random.default_rng(seed)
    o = rng.choice(vis, n_pts)
    W, H = (int(v) for v in cams["size"][0])
    u, v = geom["uvz"][o, 0].astype(np.float64), geom["uvz"][o, 1].astype(np.float64)
    r = geom["radius"][o]
    px = np.clip(np.floor(u + rng.uniform(-1, 1, n_pts) * r), 0, W - 1).astype(np.int32)
    py = np.clip(np.floor(v + rng.uniform(-1, 1, n_pts) * r), 0, H - 1).astype(np.int32)
    return o, px, py


def _log2_alpha64(scene, cams, o, px, py):
    """log2 of the raw alpha in FP64 from the independent numpy projection, and
    the magnitude M of the base-2 quadratic form's terms."""
    pr = project_bruteforce({k: (v[o] if isinstance(v, np.ndarray) else v) for k, v in scene.items()},
                            cams["intr"][0], cams["viewmats"][0], 0.3)
    l64, mag = np.zeros(len(o)), np.zeros(len(o))
    for k, p in enumerate(pr):
        d = p["uv"] - np.array([px[k] + 0.5, py[k] + 0.5])
        conic = np.linalg.inv(p["cov"])
        terms = np.array([conic[0, 0] * d[0] ** 2, 2 * conic[0, 1] * d[0] * d[1], conic[1, 1] * d[1] ** 2])
        l64[k] = np.log2(p["o"]) - 0.5 * terms.sum() / LN2
        mag[k] = 0.5 * np.abs(terms).sum() / LN2
    return l64, mag


def _scene_cams():
    c = scenes.config(1)
    return c["scene"], c["cams"]


def test_l2_is_log2_alpha_within_its_bound():
    scene, cams = _scene_cams()
    o, px, py = _points(1, 20000, scene, cams)
    drec = oracle.blend_records(scene, cams)
    l2 = oracle.blend_l2(drec[o], px, py).astype(np.float64)
    l64, mag = _log2_alpha64(scene, cams, o, px, py)
    err = np.abs(l2 - l64)
    bound = 2e-6 * (1 + mag)
    assert np.all(err <= bound), float(np.max(err / bound))
    assert np.max(err / bound) > 0.05  # the bound is not vacuous


def _near_cut_scene(seed, n, cut_log2, clamp):
    """n Gaussians, each with the pixel nearest its mean (or a pixel a few
    sigma away) and an opacity that puts log2 alpha64 within 3e-5 of cut."""
    sc = scenes.cube_scene(n, seed=seed, log_scale=(-1.0, 0.1), half=0.6)
    cams = scenes.pinhole(160, 120, 150.0)
    rng = np.random.default_rng(seed)
    pr = project_bruteforce(sc, cams["intr"][0], cams["viewmats"][0], 0.3)
    px, py = np.zeros(n, np.int32), np.zeros(n, np.int32)
    for k, p in enumerate(pr):
        off = np.zeros(2) if clamp else rng.normal(0, 1.5, 2) * np.sqrt(np.diag(p["cov"]))
        q = np.clip(np.floor(p["uv"] + off), [0, 0], [159, 119]).astype(np.int32)
        px[k], py[k] = q
        d = p["uv"] - (q + 0.5)
        qf = d @ np.linalg.solve(p["cov"], d)
        target = cut_log2 + rng.uniform(-3e-5, 3e-5)  # log2(o g) wanted
        lo = target * LN2 + 0.5 * qf  # ln o
        lo = min(lo, -1e-7)
        sc["opacity_logit"][k] = np.float32(lo - np.log1p(-np.exp(lo)))
    return sc, cams, np.arange(n), px, py


def test_decisions_equal_fp64_ones_away_from_the_bound():
    for cut, clamp, fp32_cut in ((np.log2(1 / 255), False, oracle.L2_ALPHA_MIN),
                                 (np.log2(0.99), True, oracle.L2_ALPHA_MAX)):
        sc, cams, o, px, py = _near_cut_scene(11 if clamp else 12, 4000, cut, clamp)
        drec = oracle.blend_records(sc, cams)
        ok = drec[:, 4] != 0
        l2 = oracle.blend_l2(drec[o], px, py).astype(np.float64)
        l64, mag = _log2_alpha64(sc, cams, o, px, py)
        dist = np.abs(l64 - cut)
        near = dist < 3.1e-5
        assert near[ok].mean() > 0.9  # the points really sit at the cut
        decided = dist > 2e-6 * (1 + mag) + abs(fp32_cut - cut)
        assert decided[ok].mean() > 0.5
        np.testing.assert_array_equal((l2 >= fp32_cut)[ok & decided], (l64 >= cut)[ok & decided])


def _f32(x):
    return np.asarray(x, np.float32)


def _fma32(a, b, c):
    """float32 a * b + c rounded once: the product is exact in float64; the
    float64 sum is rounded once more, which can only matter next to a float32
    halfway point, where the exact rational value decides."""
    a, b, c = (np.asarray(v, np.float32) for v in (a, b, c))
    s = a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)
    r = s.astype(np.float32)
    out = r.copy()
    half = np.spacing(np.abs(r)).astype(np.float64) / 2
    risky = np.abs(np.abs(s - r.astype(np.float64)) - half) <= 4 * np.spacing(np.abs(s))
    for k in np.nonzero(risky.ravel())[0]:
        ex = Fraction(float(a.flat[k])) * Fraction(float(b.flat[k])) + Fraction(float(c.flat[k]))
        lo_, hi_ = np.nextafter(r.flat[k], np.float32(-np.inf)), np.nextafter(r.flat[k], np.float32(np.inf))
        cands = [lo_, r.flat[k], hi_]
        dist = [abs(Fraction(float(v)) - ex) for v in cands]
        best = min(range(3), key=lambda i: (dist[i], int(np.float32(cands[i]).view(np.uint32)) & 1))
        out.flat[k] = cands[best]
    return out


def test_l2_follows_its_stated_float32_operation_order():
    scene, cams = _scene_cams()
    o, px, py = _points(5, 50000, scene, cams)
    drec = oracle.blend_records(scene, cams)[o]
    got = oracle.blend_l2(drec, px, py)
    u, v, du, dv, l2o, A, B, C = (drec[:, k] for k in range(8))
    sx, sy = _f32(px) + np.float32(0.5), _f32(py) + np.float32(0.5)
    dx = (u - sx) + du
    base = _fma32(A * dx, dx, l2o)
    bdx = B * dx
    dy = (v - sy) + dv
    ref = _fma32(dy, _fma32(C, dy, bdx), base)
    np.testing.assert_array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_transmittance_band_covers_the_kernels_deviation():
    c = scenes.config(1)
    scene, cams = c["scene"], c["cams"]
    fwd = oracle.forward(scene, cams)
    proj, drec, bins, img = fwd["proj"], fwd["drec"], fwd["bins"], fwd["img"]
    W, H = (int(v) for v in cams["size"][0])
    ranges, vals = bins["ranges"], bins["vals"]
    worst, n_checked = np.zeros(W * H), 0
    for pix in range(W * H):
        py, px = divmod(pix, W)
        tile = (py // 16) * ((W + 15) // 16) + px // 16
        ids = vals[ranges[tile, 0]:ranges[tile, 0] + img["n_contrib"][pix]].astype(np.int64)
        if len(ids) == 0:
            continue
        l2 = oracle.blend_l2(drec[ids], np.full(len(ids), px), np.full(len(ids), py)).astype(np.float64)
        keep = l2 >= oracle.L2_ALPHA_MIN
        ids, l2 = ids[keep], l2[keep]
        for sign in (-1.0, 1.0):
            a32 = np.minimum(np.float32(0.99), _f32(2.0 ** l2 * (1 + sign * oracle.EX2_REL)))
            T = np.float32(1.0)
            for a in a32:
                T = np.float32(T * np.float32(np.float32(1.0) - a))
            worst[pix] = max(worst[pix], abs(np.log(float(T) / img["final_T"][pix])))
        n_checked += 1
    band = img["slack"][:, 3]
    assert n_checked > 1000
    assert np.all(worst <= band)
    # tight where it matters: the widest band is within 2x of the largest
    # deviation, and on the widest tenth of the bands the median ratio to the
    # pixel's own deviation is at most 3 and none exceeds 8 (a pixel's
    # roundings may partly cancel, which the band cannot know)
    assert band.max() <= 2.0 * worst.max()
    top = band > np.quantile(band, 0.9)
    ratio = band[top] / worst[top]
    assert np.median(ratio) <= 3.0 and ratio.max() <= 8.0, (np.median(ratio), ratio.max())
