"""Pose refinement (Sec. 3.3 joint optimisation) on the GPU: the joint twist
gradient w1 dL_rpj + w2 dL_c + w3 dL_d with the filter gate against the oracle,
and the 100-iteration tracking loop of the TUM-shaped workload reducing the pose
error from a perturbed start."""
import numpy as np
import pytest
import torch

import oracle
import paper_2405_19614_gb300 as gs
import scenes
from gpu_util import params_on_device, rel_l2, t, viewmats_on_device
from paper_2405_19614_gb300.pipeline import TrackingStep

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2405_19614_gb300.build import build
    build()


def _setup(scale, seed_noise=0):
    c = scenes.config(3, scale)
    cams = c["cams"]
    E_true = cams["viewmats"][0].astype(np.float64)
    E0 = oracle.se3_exp_apply(c["init_offset"], E_true).astype(np.float32)
    return c, E_true, E0


def test_joint_twist_gradient_parity():
    c, E_true, E0 = _setup(0.1)
    scene = c["scene"]
    true_cams = dict(c["cams"], viewmats=E_true[None].astype(np.float32))
    cams0 = dict(c["cams"], viewmats=E0[None])
    # target: an oracle render at the true pose plus pixel noise (sigma 0.02)
    tgt = oracle.forward(scene, true_cams)["img"]
    rng = np.random.default_rng(c["noise_seed"])
    t_rgb = (tgt["rgb"] + rng.normal(0, 0.02, tgt["rgb"].shape)).astype(np.float32)
    t_depth = tgt["depth"].astype(np.float32)
    px, py = scenes.keypoint_pixels(c["keypoint_seed"], 640, 480, c["n_keypoints"])
    pts, ok = scenes.backproject(E_true, cams0["intr"][0], px, py, tgt["depth"], 640)
    obs = np.stack([px + 0.5, py + 0.5], 1)[ok] + rng.normal(0, 1.0, (int(ok.sum()), 2))
    pts = pts[ok].astype(np.float32)
    obs = obs.astype(np.float32)
    # oracle joint gradient at the perturbed pose
    ref = oracle.forward(scene, cams0)
    keep = ref["img"]["flags"] == 0
    Lr, dC, dD = oracle.loss_l1(ref["img"], t_rgb, t_depth, 0.5, 1.0, gate=True, gamma=0.99)
    # pixels whose gate input sits at its threshold are ambiguous too
    amb = np.abs(ref["img"]["alpha"] - 0.99) < 1e-5
    dC[~keep | amb] = 0
    dD[~keep | amb] = 0
    g_img = oracle.backward(scene, cams0, ref, dC, dD)["twist"]
    Lk, g_kp = oracle.reproj(pts.astype(np.float64), obs.astype(np.float64), cams0, weight=1.5)
    g_ref = g_img + g_kp
    # GPU, through the same calls the tracking step makes
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
    print(f"joint twist gradient rel-L2 err = {e:.3e}; L_rpj = {float(loss):.4f} (oracle {Lk:.4f})")
    assert e <= 1e-3
    assert abs(float(loss) - Lk) <= 1e-4 * Lk


def _pose_error(E, E_true):
    R, tv = E[:, :3].astype(np.float64), E[:, 3].astype(np.float64)
    Rt, tt = E_true[:, :3], E_true[:, 3]
    c, ct = -R.T @ tv, -Rt.T @ tt
    dR = R @ Rt.T
    ang = np.degrees(np.arccos(np.clip((np.trace(dR) - 1) / 2, -1, 1)))
    return float(np.linalg.norm(c - ct)), float(ang)


def test_tracking_loop_reduces_pose_error():
    c, E_true, E0 = _setup(0.5)
    scene = c["scene"]
    p = params_on_device(scene)
    cams = c["cams"]
    n = scene["means"].shape[0]
    # motion-blurred target: mean of 7 renders along a 2 cm / 1 deg twist, + noise
    r = gs.Rasterizer(n, scene["sh_degree"], cams["intr"], cams["size"])
    acc_rgb = torch.zeros(640 * 480, 3, device="cuda")
    acc_d = torch.zeros(640 * 480, device="cuda")
    for s in np.linspace(-0.5, 0.5, c["n_sub"]):
        Es = oracle.se3_exp_apply(s * c["motion"], E_true).astype(np.float32)
        r.forward(p, t(Es.reshape(1, 12)))
        acc_rgb += r.img["rgb"]
        acc_d += r.img["depth"]
    acc_rgb /= c["n_sub"]
    acc_d /= c["n_sub"]
    g = torch.Generator(device="cuda").manual_seed(c["noise_seed"])
    t_rgb = (acc_rgb + 0.02 * torch.randn(acc_rgb.shape, device="cuda", generator=g)).contiguous()
    t_depth = acc_d.contiguous()
    px, py = scenes.keypoint_pixels(c["keypoint_seed"], 640, 480, c["n_keypoints"])
    pts, ok = scenes.backproject(E_true, cams["intr"][0], px, py, acc_d.cpu().numpy(), 640)
    rng = np.random.default_rng(c["noise_seed"])
    obs = np.stack([px + 0.5, py + 0.5], 1)[ok] + rng.normal(0, 1.0, (int(ok.sum()), 2))
    kp = dict(points=t(pts[ok].astype(np.float32)), obs=t(obs.astype(np.float32)))
    step = TrackingStep(p, cams["intr"], cams["size"], E0[None], t_rgb, t_depth, keypoints=kp)
    e_t0, e_r0 = _pose_error(E0, E_true)
    for _ in range(c["iters"]):
        step.run()
    torch.cuda.synchronize()
    E = step.viewmats.view(3, 4).cpu().numpy()
    e_t, e_r = _pose_error(E, E_true)
    print(f"tracking: centre error {100 * e_t0:.2f} -> {100 * e_t:.2f} cm, rotation {e_r0:.3f} -> {e_r:.3f} deg")
    assert step.rast.status() == 0
    assert e_t < 0.5 * e_t0 and e_r < 0.5 * e_r0
