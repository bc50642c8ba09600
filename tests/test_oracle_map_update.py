"""Pins of densification, pruning and view point selection (Sec. 3.4, 3.3).

* a densified Gaussian projects back onto its own pixel centre, at the sensor
  depth, with a 2D radius of one pixel (Eq. d: d = r f), through the oracle's
  own projection;
* pruning agrees with sigmoid(logit) >= tau away from the cut, keeps order;
* view point selection on hand-built match counts.
"""
import math

import numpy as np

import oracle
import scenes
from oracle import map_update as MU


def test_densified_gaussian_projects_to_its_pixel_with_unit_radius():
    vm = scenes.look_at((0.3, -0.2, 0.1), (0.0, 0.3, 3.0))
    cams = scenes.cams_from([[60.0, 60.0, 32.0, 24.0]], [[64, 48]], vm[None])
    rng = np.random.default_rng(0)
    P = 64 * 48
    alpha = rng.uniform(0, 1, P).astype(np.float32)
    depth = rng.uniform(1.0, 4.0, P).astype(np.float32)
    depth[::7] = 0.0
    rgb = rng.uniform(0, 1, (P, 3))
    idx, g = MU.densify(alpha, rgb, depth, cams, 0.5, 0.0, 0)
    np.testing.assert_array_equal(idx, np.nonzero((alpha < 0.5) & (depth > 0))[0])
    scene = dict(g, sh_degree=0)
    geom = oracle.project_geom(scene, cams, blur=0.0)
    proj = oracle.project64(scene, cams, geom, blur=0.0)
    px, py = idx % 64 + 0.5, idx // 64 + 0.5
    vis = geom["radius"] > 0
    assert vis.mean() > 0.99
    # the float32 pose is orthonormal only to ~1e-7, so R^T undoes R to that level
    np.testing.assert_allclose(proj[vis, 0], px[vis], atol=1e-4)
    np.testing.assert_allclose(proj[vis, 1], py[vis], atol=1e-4)
    np.testing.assert_allclose(proj[vis, 2], depth[idx][vis], rtol=1e-6)
    # isotropic: the 2D covariance is (f r / d)^2 = 1 px^2 on the optical axis and
    # grows by the perspective factor off it; its determinant is >= 1
    a, b, c = proj[vis, 10], proj[vis, 11], proj[vis, 12]
    assert np.all(a * c - b * b >= 1 - 1e-9)
    centre = (np.abs(px - 32) < 2) & (np.abs(py - 24) < 2)
    np.testing.assert_allclose(a[centre[vis]], 1.0, rtol=2e-3)
    np.testing.assert_allclose(proj[vis, 7:10], rgb[idx][vis], atol=1e-12)


def test_prune_matches_sigmoid_threshold_and_keeps_order():
    rng = np.random.default_rng(1)
    logit = rng.normal(-3, 3, 10000).astype(np.float32)
    new_index, n_kept = MU.prune_select(logit, 0.005)
    op = 1 / (1 + np.exp(-logit.astype(np.float64)))
    away = np.abs(op - 0.005) > 1e-6
    np.testing.assert_array_equal((new_index >= 0)[away], (op >= 0.005)[away])
    kept = new_index[new_index >= 0]
    np.testing.assert_array_equal(kept, np.arange(n_kept))


def test_view_selection_interval():
    M = [0, 19, 20, 74, 75, 100, 30]
    T = [0, 100, 100, 100, 100, 100, 40]
    # half-open interval: 30 < 0.75 * 40 = 30 is false
    assert MU.select_views(M, T) == [1, 0, 1, 1, 0, 0, 0]
    assert math.isclose(0.75 * 40, 30) and MU.select_views([0, 30], [0, 40]) == [1, 0]
