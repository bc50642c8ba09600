"""The differentiation form of the path: the CUDA backward behind
torch.autograd (``rasterize``), checked against the oracle's analytic gradient
and against central finite differences of the CUDA forward itself.

Scenes are the 40-Gaussian gradient scenes of the oracle's own finite
difference pins (Sec. 3.4 C(p), D(p); Sec. 3.3 M_b(p); the twist perturbs the
pose as Exp(xi) E_t).  Pixels with a decision within 3 % of its threshold get
zero weight, so no decision moves inside a difference stencil (the step sizes
below change alpha by well under 1 %); each stencil is also checked to leave
the oracle's tile rectangles and depth order unchanged.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2405_19614_gb300 as gs
from gpu_util import PARAM_KEYS, make_rast, rel_l2, t
from helpers import grad_cams, grad_scene

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3
# central-difference steps: large enough that FP32 rounding of the render
# (about 5e-6 in the weighted sum) stays below 1 % of the difference, small
# enough that alpha moves by well under the 3 % flag margin
STEP = dict(means=2e-4, log_scales=2e-3, quats=2e-3, opacity_logit=1e-2, sh=1e-2, twist=2e-4)
FD_MARGIN = 3e-2


def _leaf_params(scene, requires_grad=True):
    p = {k: t(scene[k]).requires_grad_(requires_grad) for k in PARAM_KEYS}
    p["sh_degree"] = int(scene["sh_degree"])
    return p


def _vm(cams):
    return t(np.asarray(cams["viewmats"], np.float32).reshape(-1, 12))


def _weights(fwd, seed):
    keep = fwd["img"]["flags"] == 0
    P = keep.size
    rng = np.random.default_rng(seed)
    return dict(C=rng.standard_normal((P, 3)) * keep[:, None], D=rng.standard_normal(P) * keep,
                A=rng.standard_normal(P) * keep), keep


def _functional(out, w):
    rgb, depth, alpha = out
    return ((t(w["C"]).double() * rgb.double()).sum() + (t(w["D"]).double() * depth.double()).sum() +
            (t(w["A"]).double() * alpha.double()).sum())


def _grads_of(p, twist):
    g = {k: p[k].grad.detach().cpu().numpy().astype(np.float64) for k in PARAM_KEYS}
    g["twist"] = twist.grad.detach().cpu().numpy().astype(np.float64)
    return g


@pytest.mark.parametrize("deg,seed,oblique,edge", [(0, 11, False, False), (3, 12, True, False),
                                                   (3, 13, False, True)])
def test_autograd_matches_oracle_gradient(deg, seed, oblique, edge):
    scene, cams = grad_scene(deg, seed, edge), grad_cams(oblique)
    fwd = oracle.forward(scene, cams)
    w, keep = _weights(fwd, seed + 100)
    assert keep.mean() > 0.99
    ref = oracle.backward(scene, cams, fwd, w["C"], w["D"], w["A"])
    rast = make_rast(scene, cams)
    p = _leaf_params(scene)
    twist = torch.zeros(1, 6, device="cuda", requires_grad=True)
    out = gs.rasterize(rast, p, _vm(cams), twist)
    _functional(out, w).backward()
    assert rast.status() == 0
    g = _grads_of(p, twist)
    for k in (*PARAM_KEYS, "twist"):
        e = rel_l2(g[k], ref[k])
        print(f"deg {deg} seed {seed}: autograd {k:14s} rel-L2 err = {e:.3e}")
        assert e <= GRAD_TOL, k


def test_autograd_l1_loss_matches_oracle():
    """L1 on RGB plus L1 on depth against a seeded target render (the small
    plain workload's loss), differentiated by autograd end to end."""
    scene, cams = grad_scene(3, 41), grad_cams(True)
    target = grad_scene(3, 42)
    tgt = oracle.forward(target, cams)["img"]
    fwd = oracle.forward(scene, cams)
    _, dC, dD = oracle.loss_l1(fwd["img"], tgt["rgb"], tgt["depth"], 1.0, 1.0)
    ref = oracle.backward(scene, cams, fwd, dC, dD)
    rast = make_rast(scene, cams)
    p = _leaf_params(scene)
    twist = torch.zeros(1, 6, device="cuda", requires_grad=True)
    rgb, depth, _ = gs.rasterize(rast, p, _vm(cams), twist)
    loss = (rgb - t(tgt["rgb"])).abs().mean() + (depth - t(tgt["depth"])).abs().mean()
    loss.backward()
    g = _grads_of(p, twist)
    for k in (*PARAM_KEYS, "twist"):
        e = rel_l2(g[k], ref[k])
        print(f"L1 loss: autograd {k:14s} rel-L2 err = {e:.3e}")
        assert e <= GRAD_TOL, k


def test_two_renders_before_one_backward():
    """Two calls on one rasterizer (two poses), one backward of their summed
    functional: outputs of the first call are unchanged by the second, and the
    gradients are the sums of each call's oracle gradients."""
    scene = grad_scene(3, 51)
    cams = [grad_cams(False), grad_cams(True)]
    rast = make_rast(scene, cams[0])
    p = _leaf_params(scene)
    twists = [torch.zeros(1, 6, device="cuda", requires_grad=True) for _ in cams]
    outs, refs, total = [], [], None
    for k, c in enumerate(cams):
        fwd = oracle.forward(scene, c)
        w, keep = _weights(fwd, 60 + k)
        refs.append((fwd, w, keep))
        out = gs.rasterize(rast, p, _vm(c), twists[k])
        outs.append(out)
        f = _functional(out, w)
        total = f if total is None else total + f
    # the first call's image still equals its own render, not the second's
    fwd0, _, keep0 = refs[0]
    rgb0 = outs[0][0].detach().cpu().numpy()
    assert np.abs(rgb0 - fwd0["img"]["rgb"])[keep0].max() <= 1e-4
    total.backward()
    assert rast.status() == 0
    g = {k: p[k].grad.detach().cpu().numpy() for k in PARAM_KEYS}
    exp = {k: 0.0 for k in PARAM_KEYS}
    for k, (fwd, w, _) in enumerate(refs):
        r = oracle.backward(scene, cams[k], fwd, w["C"], w["D"], w["A"])
        for name in PARAM_KEYS:
            exp[name] = exp[name] + r[name]
        e = rel_l2(twists[k].grad.cpu().numpy(), r["twist"])
        print(f"two renders: twist of call {k} rel-L2 err = {e:.3e}")
        assert e <= GRAD_TOL
    for name in PARAM_KEYS:
        e = rel_l2(g[name], exp[name])
        print(f"two renders: {name:14s} rel-L2 err = {e:.3e}")
        assert e <= GRAD_TOL, name


@pytest.mark.parametrize("deg,seed,oblique", [(3, 12, True), (0, 11, False)])
def test_autograd_matches_central_differences_of_the_gpu_forward(deg, seed, oblique):
    scene, cams = grad_scene(deg, seed), grad_cams(oblique)
    fwd = oracle.forward(scene, cams, margin_alpha=FD_MARGIN, margin_T=FD_MARGIN)
    w, keep = _weights(fwd, seed + 5)
    assert keep.mean() > 0.95
    rast = make_rast(scene, cams)
    p = _leaf_params(scene)
    twist = torch.zeros(1, 6, device="cuda", requires_grad=True)
    vm = _vm(cams)
    _functional(gs.rasterize(rast, p, vm, twist), w).backward()
    g = _grads_of(p, twist)

    def F(sc, vmat):
        with torch.no_grad():
            return float(_functional(gs.rasterize(rast, _leaf_params(sc, False), vmat), w))

    # the stencil must not change the rectangles or depth order (the tile
    # test only removes pairs no pixel blends, so its lists are not compared)
    full = oracle.forward(scene, cams, tile_cull=False)["bins"]

    def same_lists(sc, c):
        b = oracle.forward(sc, c, tile_cull=False)["bins"]
        return np.array_equal(b["vals"], full["vals"]) and np.array_equal(b["ranges"], full["ranges"])

    rng = np.random.default_rng(seed + 9)
    vis = np.nonzero(fwd["geom"]["radius"] > 0)[0]
    checked = 0
    for name in PARAM_KEYS:
        h = STEP[name]
        scale = np.abs(g[name]).max()
        for _ in range(6):
            i = int(rng.choice(vis))
            idx = (i,) + tuple(int(rng.integers(0, s)) for s in g[name].shape[1:])
            sp = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in scene.items()}
            th = sp[name][idx]
            sp[name][idx] = th + h
            sm = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in scene.items()}
            sm[name][idx] = th - h
            if not (same_lists(sp, cams) and same_lists(sm, cams)):
                continue
            fd = (F(sp, vm) - F(sm, vm)) / (2 * h)
            an = g[name][idx]
            print(f"FD {name}{idx}: fd {fd:.6g} autograd {an:.6g}")
            assert abs(fd - an) <= 1e-2 * abs(an) + 2e-3 * scale, (name, idx, fd, an)
            checked += 1
    E0 = np.asarray(cams["viewmats"][0], np.float64)
    scale = np.abs(g["twist"]).max()
    h = STEP["twist"]
    for k in range(6):
        xi = np.zeros(6)
        xi[k] = h
        cp = dict(cams, viewmats=oracle.se3_exp_apply(xi, E0)[None])
        xi[k] = -h
        cm = dict(cams, viewmats=oracle.se3_exp_apply(xi, E0)[None])
        assert same_lists(scene, cp) and same_lists(scene, cm)
        fd = (F(scene, _vm(cp)) - F(scene, _vm(cm))) / (2 * h)
        an = g["twist"][0, k]
        print(f"FD twist[{k}]: fd {fd:.6g} autograd {an:.6g}")
        assert abs(fd - an) <= 1e-2 * abs(an) + 2e-3 * scale, (k, fd, an)
    assert checked >= 20
