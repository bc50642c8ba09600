"""Parity at the full sizes of the five workloads, in the launch configuration
bench.py times (all views of a workload in one launch per stage, compositing
variants picked by the autotuner), on outputs the oracle computes in seconds:

* workload 2 (300k Gaussians, 1200x680): every key, list and range, the whole
  image and every gradient tensor;
* workload 4 (1M Gaussians, 8 x 1200x680): every key, list and range; images and
  2D gradients of two sampled views; parameter and twist gradients for upstream
  gradients placed on those two views only (zero elsewhere);
* workload 5 (4M Gaussians, 16 views of four sizes): per-view lists, images and
  twist gradients of one view of each size;
* workload 3 (100k Gaussians, 640x480): the joint twist gradient with the gate
  and the re-projection term.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2405_19614_gb300 as gs
import scenes
from gpu_util import (GRAD_TOL, PARAM_KEYS, check_image, check_single_blend_alpha, params_on_device, parity_log,
                      rel_l2, t, viewmats_on_device, zero_grads)
from paper_2405_19614_gb300.autotune import tune

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2405_19614_gb300.build import build
    build()


def _view(cams, v):
    return scenes.cams_from(cams["intr"][v:v + 1], cams["size"][v:v + 1], cams["viewmats"][v:v + 1])


def _f64(scene):
    # the oracle works in FP64; converting once spares it a copy per call
    return {k: (v.astype(np.float64) if isinstance(v, np.ndarray) else v) for k, v in scene.items()}


def _setup(idx):
    c = scenes.config(idx)
    scene, cams = c["scene"], c["cams"]
    n, V = scene["means"].shape[0], len(cams["size"])
    rast = gs.Rasterizer(n, scene["sh_degree"], cams["intr"], cams["size"], pair_capacity=12 * n * V)
    p = params_on_device(scene)
    vm = viewmats_on_device(cams)
    rast.forward(p, vm)
    torch.cuda.synchronize()
    assert rast.status() == 0
    # the variants bench.py would use on this workload
    d_rgb = torch.zeros(rast.n_pix, 3, device="cuda")
    d_depth = torch.zeros(rast.n_pix, device="cuda")
    tune(rast, p, vm, d_rgb, d_depth, use_cache=False)
    rast.forward(p, vm)
    torch.cuda.synchronize()
    return c, _f64(scene), cams, rast, p, vm


def _pix_range(cams, v):
    size = np.asarray(cams["size"], np.int64)
    base = int((size[:v, 0] * size[:v, 1]).sum())
    return base, base + int(size[v, 0] * size[v, 1])


def _tile_range(cams, v):
    size = np.asarray(cams["size"], np.int64)
    nt = ((size[:, 0] + 15) // 16) * ((size[:, 1] + 15) // 16)
    base = int(nt[:v].sum())
    return base, base + int(nt[v])


def _check_view_lists(rast, cams, v, ref_bins):
    t0, t1 = _tile_range(cams, v)
    ranges = rast.bins["ranges"].cpu().numpy().view(np.uint32)[t0:t1]
    ref_r = ref_bins["ranges"]
    starts = ranges[:, 0].astype(np.int64)
    lens = (ranges[:, 1] - ranges[:, 0]).astype(np.int64)
    np.testing.assert_array_equal(lens, (ref_r[:, 1] - ref_r[:, 0]).astype(np.int64))
    nonempty = lens > 0
    if not nonempty.any():
        return
    lo, hi = int(starts[nonempty].min()), int((starts + lens)[nonempty].max())
    keys = rast.bins["keys"][lo:hi].cpu().numpy().view(np.uint64) - np.uint64(t0 << 32)
    vals = rast.bins["vals"][lo:hi].cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(keys, ref_bins["keys"])
    np.testing.assert_array_equal(vals, ref_bins["vals"])


def _check_view_image(rast, cams, v, ref_img, name):
    p0, p1 = _pix_range(cams, v)
    img = {k: val[p0:p1].cpu().numpy() for k, val in rast.img.items()}
    check_image(img, ref_img, f"{name} view {v}")
    return img


def _log_grads(name, errors):
    parity_log(dict(kind="grad", name=name, **errors))


def test_workload2_full_parity():
    c, scene, cams, rast, p, vm = _setup(2)
    geom = oracle.project_geom(scene, cams)
    bins = oracle.bin_tiles(cams, geom)
    assert rast.n_pairs() == bins["n_pairs"]
    K = bins["n_pairs"]
    np.testing.assert_array_equal(rast.bins["keys"][:K].cpu().numpy().view(np.uint64), bins["keys"])
    np.testing.assert_array_equal(rast.bins["vals"][:K].cpu().numpy().view(np.uint32), bins["vals"])
    np.testing.assert_array_equal(rast.bins["ranges"].cpu().numpy().view(np.uint32), bins["ranges"])
    proj = oracle.project64(scene, cams, geom)
    drec = oracle.blend_records(scene, cams)
    img = oracle.render(cams, proj, drec, bins, geom["n"])
    gpu_img = _check_view_image(rast, cams, 0, img, "replica-300k")
    # (in this room every pixel blends several entries: the check may find none)
    check_single_blend_alpha(gpu_img, dict(bins=bins, drec=drec, geom=geom, img=img), cams, "replica-300k")
    # gradients of L1 RGB + 0.1 L1 depth against an oracle render of the target scene
    tgt = oracle.forward(c["target_scene"], cams)["img"]
    L, dC, dD = oracle.loss_l1(img, tgt["rgb"].astype(np.float32), tgt["depth"].astype(np.float32), 1.0, 0.1)
    keep = img["flags"] == 0
    dC[~keep] = 0
    dD[~keep] = 0
    gref = oracle.project_bwd(scene, cams, geom, oracle.render_bwd(cams, proj, drec, bins, geom["n"], dC, dD,
                                                                    np.zeros_like(dD)))
    grads = zero_grads(p)
    d_twist = torch.zeros(1, 6, device="cuda")
    rast.backward(p, vm, t(dC), t(dD), None, grads, d_twist)
    torch.cuda.synchronize()
    out = {k: grads[k].cpu().numpy() for k in PARAM_KEYS}
    out["twist"] = d_twist.cpu().numpy()
    errs = {k: rel_l2(out[k], gref[k]) for k in (*PARAM_KEYS, "twist")}
    _log_grads("replica-300k", errs)
    for k, e in errs.items():
        print(f"replica-300k: grad {k:14s} rel-L2 err = {e:.3e}")
        assert e <= GRAD_TOL, k


def test_workload4_full_parity_sampled_views():
    c, scene, cams, rast, p, vm = _setup(4)
    geom = oracle.project_geom(scene, cams)
    bins = oracle.bin_tiles(cams, geom)
    assert rast.n_pairs() == bins["n_pairs"]
    K = bins["n_pairs"]
    np.testing.assert_array_equal(rast.bins["keys"][:K].cpu().numpy().view(np.uint64), bins["keys"])
    np.testing.assert_array_equal(rast.bins["vals"][:K].cpu().numpy().view(np.uint32), bins["vals"])
    np.testing.assert_array_equal(rast.bins["ranges"].cpu().numpy().view(np.uint32), bins["ranges"])
    del bins
    sampled = [0, 5]
    rng = np.random.default_rng(44)
    P = rast.n_pix
    dC, dD, dA = np.zeros((P, 3)), np.zeros(P), np.zeros(P)
    sub = scenes.cams_from(cams["intr"][sampled], cams["size"][sampled], cams["viewmats"][sampled])
    fsub = oracle.forward(scene, sub)
    sub_dC, sub_dD, sub_dA = [], [], []
    for j, v in enumerate(sampled):
        p0, p1 = _pix_range(cams, v)
        q0, q1 = _pix_range(sub, j)
        ref_img = {k: val[q0:q1] for k, val in fsub["img"].items()}
        _check_view_image(rast, cams, v, ref_img, "batched-1M")
        keep = ref_img["flags"] == 0
        g = rng.normal(0, 1e-6, (p1 - p0, 3)) * keep[:, None]
        gd = rng.normal(0, 1e-6, p1 - p0) * keep
        ga = rng.normal(0, 1e-7, p1 - p0) * keep
        dC[p0:p1], dD[p0:p1], dA[p0:p1] = g, gd, ga
        sub_dC.append(g)
        sub_dD.append(gd)
        sub_dA.append(ga)
    gref = oracle.backward(scene, sub, fsub, np.concatenate(sub_dC), np.concatenate(sub_dD),
                           np.concatenate(sub_dA))
    # 2D gradients of the sampled views
    gs.gs_render_bwd_splats(rast.proj, rast.n, rast.bins, rast.views, rast.img, t(dC), t(dD), t(dA), rast.grad2d,
                            rast.work_counter)
    torch.cuda.synchronize()
    G = rast.grad2d.view(len(cams["size"]), rast.n, 12)
    n = rast.n
    errs = {}
    for j, v in enumerate(sampled):
        e = rel_l2(G[v, :, :10].cpu().numpy(), gref["g2d"][j * n:(j + 1) * n])
        errs[f"g2d_view{v}"] = e
        print(f"batched-1M view {v}: 2D grad rel-L2 err = {e:.3e}")
        assert e <= GRAD_TOL
    rast.grad2d.zero_()
    # parameter and twist gradients through the full batched backward
    grads = zero_grads(p)
    d_twist = torch.zeros(len(cams["size"]), 6, device="cuda")
    rast.backward(p, vm, t(dC), t(dD), t(dA), grads, d_twist)
    torch.cuda.synchronize()
    for k in PARAM_KEYS:
        errs[k] = rel_l2(grads[k].cpu().numpy(), gref[k])
    tw = d_twist.cpu().numpy()
    errs["twist"] = rel_l2(tw[sampled], gref["twist"])
    _log_grads("batched-1M views 0,5", errs)
    for k, e in errs.items():
        print(f"batched-1M: grad {k:14s} rel-L2 err = {e:.3e}")
        assert e <= GRAD_TOL, k
    others = [v for v in range(len(cams["size"])) if v not in sampled]
    assert np.abs(tw[others]).max() == 0.0


def test_workload5_full_parity_one_view_per_size():
    c, scene, cams, rast, p, vm = _setup(5)
    sampled = [1, 6, 9, 14]  # 640x480, 960x540, 1200x680, 1280x720
    rng = np.random.default_rng(55)
    P = rast.n_pix
    dC, dD = np.zeros((P, 3)), np.zeros(P)
    refs = {}
    for v in sampled:
        cv = _view(cams, v)
        f = oracle.forward(scene, cv)
        _check_view_lists(rast, cams, v, f["bins"])
        _check_view_image(rast, cams, v, f["img"], "long-4M")
        keep = f["img"]["flags"] == 0
        p0, p1 = _pix_range(cams, v)
        dC[p0:p1] = rng.normal(0, 1e-6, (p1 - p0, 3)) * keep[:, None]
        dD[p0:p1] = rng.normal(0, 1e-6, p1 - p0) * keep
        g = oracle.backward(scene, cv, f, dC[p0:p1], dD[p0:p1])
        refs[v] = g["twist"][0]
    grads = zero_grads(p)
    d_twist = torch.zeros(len(cams["size"]), 6, device="cuda")
    rast.backward(p, vm, t(dC), t(dD), None, grads, d_twist)
    torch.cuda.synchronize()
    tw = d_twist.cpu().numpy()
    errs = {f"twist_view{v}": rel_l2(tw[v], refs[v]) for v in sampled}
    _log_grads("long-4M", errs)
    for k, e in errs.items():
        print(f"long-4M: {k} grad rel-L2 err = {e:.3e}")
        assert e <= GRAD_TOL


def test_workload3_full_joint_twist_gradient():
    c = scenes.config(3)
    scene, cams = c["scene"], c["cams"]
    scene64 = _f64(scene)
    E_true = cams["viewmats"][0].astype(np.float64)
    E0 = oracle.se3_exp_apply(c["init_offset"], E_true).astype(np.float32)
    true_cams = dict(cams, viewmats=E_true[None].astype(np.float32))
    cams0 = dict(cams, viewmats=E0[None])
    tgt = oracle.forward(scene64, true_cams)["img"]
    rng = np.random.default_rng(c["noise_seed"])
    t_rgb = (tgt["rgb"] + rng.normal(0, 0.02, tgt["rgb"].shape)).astype(np.float32)
    t_depth = tgt["depth"].astype(np.float32)
    px, py = scenes.keypoint_pixels(c["keypoint_seed"], 640, 480, c["n_keypoints"])
    pts, ok = scenes.backproject(E_true, cams0["intr"][0], px, py, tgt["depth"], 640)
    obs = (np.stack([px + 0.5, py + 0.5], 1)[ok] + rng.normal(0, 1.0, (int(ok.sum()), 2))).astype(np.float32)
    pts = pts[ok].astype(np.float32)
    ref = oracle.forward(scene64, cams0)
    keep = ref["img"]["flags"] == 0
    amb = np.abs(ref["img"]["alpha"] - 0.99) < 1e-5
    Lr, dC, dD = oracle.loss_l1(ref["img"], t_rgb, t_depth, 0.5, 1.0, gate=True, gamma=0.99)
    dC[~keep | amb] = 0
    dD[~keep | amb] = 0
    g_ref = oracle.backward(scene64, cams0, ref, dC, dD)["twist"]
    Lk, g_kp = oracle.reproj(pts.astype(np.float64), obs.astype(np.float64), cams0, weight=1.5)
    g_ref = g_ref + g_kp
    p = params_on_device(scene)
    vm = viewmats_on_device(cams0)
    rast = gs.Rasterizer(scene["means"].shape[0], scene["sh_degree"], cams0["intr"], cams0["size"])
    rast.forward(p, vm)
    d_twist = torch.zeros(1, 6, device="cuda")
    rast.backward(p, vm, t(dC), t(dD), None, None, d_twist)
    loss = torch.zeros(1, device="cuda")
    gs.gs_reproj_loss_grad(t(pts), t(obs), None, rast.views, vm, 1.5, loss, d_twist)
    torch.cuda.synchronize()
    e = rel_l2(d_twist.cpu().numpy(), g_ref)
    _log_grads("tum-track-100k joint", dict(twist=e))
    print(f"tum-track-100k: joint twist gradient rel-L2 err = {e:.3e}")
    assert e <= GRAD_TOL
