"""Pins of the oracle's reverse mode against central finite differences of its
own FP64 forward (which the render and geometry tests pin independently).

The functional is F = sum wC.C + wD D + wA A with random per-pixel weights, so
its gradient is exactly what the reverse pass computes for upstream gradients
(wC, wD, wA).  Tile membership and order are held fixed (they are piecewise
constant), and pixels with a decision within 1e-3 of its threshold get zero
weight so no decision flips inside the difference stencil.  Parameters are
FP64 here; the twist perturbs the pose as Exp(xi) E_t.
"""
import numpy as np
import pytest

import oracle
import scenes
from helpers import grad_cams as _cams, grad_scene as _tiny_scene

H_REL = 1e-6


def _functional(img, w):
    return float((w["C"] * img["rgb"]).sum() + (w["D"] * img["depth"]).sum() + (w["A"] * img["alpha"]).sum())


def _setup(deg, seed, oblique, edge=False):
    scene, cams = _tiny_scene(deg, seed, edge), _cams(oblique)
    fwd = oracle.forward(scene, cams, margin_alpha=1e-3, margin_T=1e-3)
    proj = fwd["proj"]
    vis = fwd["geom"]["radius"] > 0
    assert vis.sum() >= 20
    if edge:
        assert proj[vis, 13:15].any()             # the tangent clamp is exercised
        assert (proj[vis, 6] > 0.99).any()        # so is the alpha clamp
    else:
        assert not proj[vis, 13:15].any()
    assert proj[vis, 7:10].min() > 0.05           # no colour clamp in the stencil
    P = fwd["bins"]["n_pix"]
    rng = np.random.default_rng(seed + 1000)
    keep = (fwd["img"]["flags"] == 0).astype(np.float64)
    assert keep.mean() > 0.9
    w = dict(C=rng.standard_normal((P, 3)) * keep[:, None], D=rng.standard_normal(P) * keep,
             A=rng.standard_normal(P) * keep)
    return scene, cams, fwd, w


def _eval(scene, cams, fwd, w):
    proj = oracle.project64(scene, cams, fwd["geom"])
    drec = oracle.blend_records(scene, cams)
    return _functional(oracle.render(cams, proj, drec, fwd["bins"], fwd["geom"]["n"]), w)


@pytest.mark.parametrize("deg,seed,oblique,edge", [(0, 11, False, False), (3, 12, True, False),
                                                   (3, 13, False, True)])
def test_param_gradients_match_central_differences(deg, seed, oblique, edge):
    scene, cams, fwd, w = _setup(deg, seed, oblique, edge)
    g = oracle.backward(scene, cams, fwd, w["C"], w["D"], w["A"])
    rng = np.random.default_rng(seed)
    vis = np.nonzero(fwd["geom"]["radius"] > 0)[0]
    for name in ("means", "log_scales", "quats", "opacity_logit", "sh"):
        an_all = g[name]
        scale = np.abs(an_all).max()
        assert scale > 0, name
        picks = [int(rng.choice(vis)) for _ in range(12)]
        if edge:
            picks += [i for i in range(10) if i in set(vis.tolist())]
        for i in picks:
            idx = (i,) + tuple(int(rng.integers(0, s)) for s in an_all.shape[1:])
            theta = scene[name][idx]
            h = H_REL * max(1.0, abs(theta))
            sp = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in scene.items()}
            sp[name][idx] = theta + h
            fp = _eval(sp, cams, fwd, w)
            sp[name][idx] = theta - h
            fm = _eval(sp, cams, fwd, w)
            fd = (fp - fm) / (2 * h)
            an = an_all[idx]
            assert abs(fd - an) <= 1e-5 * abs(an) + 1e-6 * scale, (name, idx, fd, an)


@pytest.mark.parametrize("deg,seed,oblique,edge", [(0, 21, True, False), (3, 22, True, False),
                                                   (3, 23, False, True)])
def test_twist_gradient_matches_central_differences(deg, seed, oblique, edge):
    scene, cams, fwd, w = _setup(deg, seed, oblique, edge)
    g = oracle.backward(scene, cams, fwd, w["C"], w["D"], w["A"])
    E0 = cams["viewmats"][0].astype(np.float64)
    scale = np.abs(g["twist"]).max()
    for k in range(6):
        h = 1e-6
        xi = np.zeros(6)
        xi[k] = h
        cp = dict(cams, viewmats=oracle.se3_exp_apply(xi, E0)[None])
        fp = _eval(scene, cp, fwd, w)
        xi[k] = -h
        cm = dict(cams, viewmats=oracle.se3_exp_apply(xi, E0)[None])
        fm = _eval(scene, cm, fwd, w)
        fd = (fp - fm) / (2 * h)
        an = g["twist"][0, k]
        assert abs(fd - an) <= 1e-5 * abs(an) + 1e-6 * scale, (k, fd, an)


def test_multi_view_gradients_sum_over_views():
    scene = _tiny_scene(3, 31)
    vms = np.stack([scenes.look_at((0.2 * k, -0.1, -0.2), (0.0, 0.0, 3.0)) for k in range(3)])
    cams = scenes.pinhole(64, 48, 60.0, n_views=3, viewmats=vms)
    fwd = oracle.forward(scene, cams)
    P = fwd["bins"]["n_pix"]
    rng = np.random.default_rng(3)
    dC, dD, dA = rng.standard_normal((P, 3)), rng.standard_normal(P), rng.standard_normal(P)
    g = oracle.backward(scene, cams, fwd, dC, dD, dA)
    tot = {k: np.zeros_like(v) for k, v in g.items() if k not in ("g2d", "twist")}
    for v in range(3):
        cv = scenes.cams_from(cams["intr"][v:v + 1], cams["size"][v:v + 1], cams["viewmats"][v:v + 1])
        fv = oracle.forward(scene, cv)
        sl = slice(v * 64 * 48, (v + 1) * 64 * 48)
        gv = oracle.backward(scene, cv, fv, dC[sl], dD[sl], dA[sl])
        for k in tot:
            tot[k] += gv[k]
        np.testing.assert_allclose(g["twist"][v], gv["twist"][0], rtol=1e-12, atol=1e-15)
    for k in tot:
        np.testing.assert_allclose(g[k], tot[k], rtol=1e-12, atol=1e-15)
