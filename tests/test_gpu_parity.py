"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bars: radii, tile rectangles, depths, keys, per-tile lists and ranges
bit-exact; the records' decision quantities (2D mean and its remainder,
log2 o, base-2 conic) bit-exact, so the alpha skip and clamp decisions agree
bit for bit; RGB, depth and alpha within 1e-4 absolute of the FP64 oracle on
pixels whose stop decision is outside the transmittance band (at most 0.01 %
of pixels are in it, each within 1e-4 plus that one entry's contribution);
gradients within 1e-3 relative L2 per parameter tensor (logged per output),
with the upstream gradient of the banded pixels zeroed on both sides.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2405_19614_gb300 as gs
import scenes
from gpu_util import (GRAD_TOL, IMG_TOL, PARAM_KEYS, check_image, check_single_blend_alpha, gpu_bins, gpu_geom,
                      make_rast, oracle_targets, params_on_device, parity_log, rel_l2, t, viewmats_on_device,
                      zero_grads)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2405_19614_gb300.build import build
    build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def _cases():
    # (name, scene, cams): small, several tiles, ragged edges, uneven multi-view
    c1 = scenes.config(1)
    yield "plain-2k-64x48", c1["scene"], c1["cams"]
    sc = scenes.cube_scene(3000, seed=77, sh_degree=3, log_scale=(-3.2, 0.5))
    vms = np.stack([scenes.look_at((0.3 * k - 0.3, -0.2, -0.4), (0.0, 0.1, 3.0)) for k in range(3)])
    cams = scenes.cams_from([[70, 70, 50, 30], [90, 80, 61.5, 40], [40, 40, 18, 17]],
                            [[100, 61], [123, 77], [37, 35]], vms)
    yield "sh3-3views-ragged", sc, cams


CASES = list(_cases())


def _run(scene, cams, capacity=None):
    rast = make_rast(scene, cams, capacity)
    p = params_on_device(scene)
    vm = viewmats_on_device(cams)
    rast.forward(p, vm)
    torch.cuda.synchronize()
    return rast, p, vm


@pytest.mark.parametrize("name,scene,cams", CASES, ids=[c[0] for c in CASES])
def test_projection_and_binning_bit_exact(name, scene, cams):
    rast, p, vm = _run(scene, cams)
    assert rast.status() == 0
    geom = oracle.project_geom(scene, cams)
    rec, radii, tt, rect = gpu_geom(rast)
    np.testing.assert_array_equal(radii, geom["radius"])
    vis = geom["radius"] > 0
    np.testing.assert_array_equal(tt, geom["kept"])
    np.testing.assert_array_equal(rect[vis], geom["rect"][vis])
    np.testing.assert_array_equal(rec[vis][:, 0:3].view(np.uint32), geom["uvz"][vis].view(np.uint32))
    # the tiles each splat keeps (exact tile test), bit for bit
    mask = rast.proj["tile_mask"].cpu().numpy().view(np.uint64)
    small = vis & ((rect[:, 2] - rect[:, 0] + 1) * (rect[:, 3] - rect[:, 1] + 1) <= 64)
    np.testing.assert_array_equal(mask[small], geom["tile_mask"][small])
    assert int(geom["kept"].sum()) < int(geom["tiles_touched"].sum())
    bins = oracle.bin_tiles(cams, geom)
    keys, vals, ranges = gpu_bins(rast)
    assert rast.n_pairs() == bins["n_pairs"]
    np.testing.assert_array_equal(keys, bins["keys"])
    np.testing.assert_array_equal(vals, bins["vals"])
    np.testing.assert_array_equal(ranges, bins["ranges"])
    # the decision quantities, bit for bit: (u, v), remainders (du, dv), log2 o
    # and the base-2 conic (A', B', C')
    drec = oracle.blend_records(scene, cams)
    cols = [0, 1, 7, 11, 3, 4, 5, 6]  # record columns of (u, v, du, dv, log2 o, A', B', C')
    np.testing.assert_array_equal(rec[vis][:, cols].view(np.uint32), drec[vis].view(np.uint32))
    # colour is ordinary FP32 against FP64
    proj = oracle.project64(scene, cams, geom)
    np.testing.assert_allclose(rec[vis][:, 8:11], proj[vis][:, 7:10], rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("name,scene,cams", CASES, ids=[c[0] for c in CASES])
def test_render_forward_parity(name, scene, cams):
    rast, p, vm = _run(scene, cams)
    fwd = oracle.forward(scene, cams)
    img = {k: v.cpu().numpy() for k, v in rast.img.items()}
    check_image(img, fwd["img"], name)
    assert check_single_blend_alpha(img, fwd, cams, name) > 0


def _backward_case(scene, cams, target_scene=None, twist=True):
    rast, p, vm = _run(scene, cams)
    ref = oracle.forward(scene, cams)
    keep = ref["img"]["flags"] == 0
    if target_scene is not None:
        t_rgb, t_depth = oracle_targets(target_scene, cams)
    else:
        rng = np.random.default_rng(0)
        t_rgb = rng.uniform(0, 1, ref["img"]["rgb"].shape).astype(np.float32)
        t_depth = rng.uniform(0, 5, ref["img"]["depth"].shape).astype(np.float32)
    L, dC, dD = oracle.loss_l1(ref["img"], t_rgb, t_depth, 1.0, 1.0)
    # an extra alpha term exercises the border-mask gradient
    dA = np.random.default_rng(1).normal(0, 1e-4, ref["img"]["alpha"].shape)
    dC[~keep] = 0.0
    dD[~keep] = 0.0
    dA[~keep] = 0.0
    gref = oracle.backward(scene, cams, ref, dC, dD, dA)
    grads = zero_grads(p)
    d_twist = torch.zeros(len(cams["size"]), 6, device=vm.device) if twist else None
    rast.backward(p, vm, t(dC), t(dD), t(dA), grads, d_twist)
    torch.cuda.synchronize()
    assert rast.status() == 0
    assert float(rast.grad2d.abs().max()) == 0.0  # left zeroed for the next call
    out = {k: grads[k].cpu().numpy() for k in PARAM_KEYS}
    if twist:
        out["twist"] = d_twist.cpu().numpy()
    return out, gref


def check_grads(out, gref, name, keys=(*PARAM_KEYS, "twist")):
    rec = dict(kind="grad", name=name)
    for k in keys:
        e = rel_l2(out[k], gref[k])
        rec[k] = e
        print(f"{name}: grad {k:14s} rel-L2 err = {e:.3e}")
    parity_log(rec)
    for k in keys:
        assert rec[k] <= GRAD_TOL, k


@pytest.mark.parametrize("name,scene,cams", CASES, ids=[c[0] for c in CASES])
def test_backward_parity(name, scene, cams):
    out, gref = _backward_case(scene, cams)
    check_grads(out, gref, name)


def test_splat_gradients_parity():
    c = scenes.config(1)
    scene, cams = c["scene"], c["cams"]
    rast, p, vm = _run(scene, cams)
    ref = oracle.forward(scene, cams)
    keep = ref["img"]["flags"] == 0
    rng = np.random.default_rng(2)
    P = ref["bins"]["n_pix"]
    dC, dD, dA = rng.normal(0, 1, (P, 3)), rng.normal(0, 1, P), rng.normal(0, 1, P)
    dC[~keep] = 0
    dD[~keep] = 0
    dA[~keep] = 0
    g2d = oracle.render_bwd(cams, ref["proj"], ref["drec"], ref["bins"], ref["geom"]["n"], dC, dD, dA)
    gs.gs_render_bwd_splats(rast.proj, rast.n, rast.bins, rast.views, rast.img, t(dC), t(dD), t(dA), rast.grad2d,
                            rast.work_counter)
    torch.cuda.synchronize()
    G = rast.grad2d.view(-1, 12).cpu().numpy()[:, :10]
    names = ("u", "v", "conicA", "conicB", "conicC", "opacity", "r", "g", "b", "z")
    for k, nm in enumerate(names):
        e = rel_l2(G[:, k], g2d[:, k])
        print(f"2D grad {nm:8s} rel-L2 err = {e:.3e}")
        assert e <= GRAD_TOL, nm


@pytest.mark.parametrize("deg", [1, 2])
def test_backward_parity_sh_degrees_1_and_2(deg):
    """Degrees 1 (3K = 12 floats a row, 16-byte copies) and 2 (27 floats,
    4-byte copies) of the colour backward, with a ragged last block (n = 1001)."""
    sc = scenes.cube_scene(1001, seed=80 + deg, sh_degree=deg, log_scale=(-3.2, 0.5))
    out, gref = _backward_case(sc, CASES[1][2])
    check_grads(out, gref, f"sh{deg}-1001")


def test_colour_backward_unaligned_sh_equals_aligned():
    """The SH rows travel 16 bytes at a time when the coefficient and gradient
    pointers are 16-byte aligned, 4 bytes at a time otherwise: both give the
    same gradients bit for bit."""
    _, scene, cams = CASES[1]
    rast, p, vm = _run(scene, cams)
    rng = np.random.default_rng(10)
    P = rast.n_pix
    gs.gs_render_bwd_splats(rast.proj, rast.n, rast.bins, rast.views, rast.img, t(rng.normal(0, 1, (P, 3))),
                            t(rng.normal(0, 1, P)), None, rast.grad2d, rast.work_counter)
    g2d = rast.grad2d.clone()

    def shifted(x):  # the same values, 4 bytes past a 16-byte boundary
        buf = torch.zeros(x.numel() + 1, device=x.device)
        y = buf[1:].view(x.shape)
        y.copy_(x)
        assert y.data_ptr() % 16 == 4
        return y

    out = {}
    for mode in ("aligned", "unaligned"):
        rast.grad2d.copy_(g2d)
        q = dict(p)
        g = zero_grads(p)
        if mode == "unaligned":
            q["sh"] = shifted(p["sh"])
            g["sh"] = shifted(g["sh"])
        gs.gs_project_bwd(q, rast.views, vm, rast.proj, rast.grad2d, g, None)
        torch.cuda.synchronize()
        out[mode] = {k: g[k].cpu().numpy() for k in PARAM_KEYS}
    for k in PARAM_KEYS:
        assert np.abs(out["aligned"][k]).max() > 0, k
        np.testing.assert_array_equal(out["unaligned"][k], out["aligned"][k], err_msg=k)


@pytest.mark.parametrize("name,scene,cams", CASES, ids=[c[0] for c in CASES])
def test_overwrite_grads_equals_accumulating_into_zeros(name, scene, cams):
    """With overwrite_grads the projection backward writes every Gaussian's
    gradients: a buffer full of garbage ends equal to zeros plus the
    accumulated gradients (SH degrees with and without view dependence).  Both
    calls chain the same 2D gradients (the compositing backward adds with
    atomics, so two runs of it may differ in the last bit)."""
    rast, p, vm = _run(scene, cams)
    rng = np.random.default_rng(9)
    P = rast.n_pix
    gs.gs_render_bwd_splats(rast.proj, rast.n, rast.bins, rast.views, rast.img, t(rng.normal(0, 1, (P, 3))),
                            t(rng.normal(0, 1, P)), None, rast.grad2d, rast.work_counter)
    g2d = rast.grad2d.clone()
    out = {}
    for mode in ("add", "overwrite"):
        rast.grad2d.copy_(g2d)
        g = zero_grads(p) if mode == "add" else {k: torch.full_like(p[k], 1e30) for k in PARAM_KEYS}
        gs.gs_project_bwd(p, rast.views, vm, rast.proj, rast.grad2d, g, None, overwrite_grads=(mode == "overwrite"))
        torch.cuda.synchronize()
        out[mode] = {k: g[k].cpu().numpy() for k in PARAM_KEYS}
    for k in PARAM_KEYS:
        assert np.abs(out["add"][k]).max() > 0, k
        np.testing.assert_array_equal(out["overwrite"][k], out["add"][k], err_msg=k)


@pytest.mark.parametrize("n", [1, 5, 1_000_003])
def test_keyframe_decoding_matches_oracle(n):
    """Sensor-format keyframes decode bit for bit as the oracle's FP32
    definition, over a ragged pixel count (the last n mod 4 pixels take the
    scalar path)."""
    rng = np.random.default_rng(n)
    rgb8 = rng.integers(0, 256, (n, 3), dtype=np.uint8)
    d16 = rng.integers(0, 65536, n, dtype=np.uint32).astype(np.uint16)
    d16[: min(n, 2)] = (0, 65535)[: min(n, 2)]
    ref_rgb, ref_depth = oracle.decode_keyframes(rgb8, d16, 1 / 5000)
    rgb = torch.empty(n, 3, device="cuda")
    depth = torch.empty(n, device="cuda")
    gs.gs_decode_keyframes(torch.from_numpy(rgb8).cuda(), torch.from_numpy(d16.view(np.int16)).cuda(), 1 / 5000, rgb,
                           depth)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(rgb.cpu().numpy().view(np.uint32), ref_rgb.view(np.uint32))
    np.testing.assert_array_equal(depth.cpu().numpy().view(np.uint32), ref_depth.view(np.uint32))


@pytest.mark.parametrize("gate", [False, True])
@pytest.mark.parametrize("name,scene,cams", CASES, ids=[c[0] for c in CASES])
def test_fused_forward_l1_equals_separate_calls(name, scene, cams, gate):
    """gs_render_fwd_l1 gives the images of gs_render_fwd and the gradients of
    gs_loss_l1 bit for bit, and its loss up to summation order."""
    rast, p, vm = _run(scene, cams)
    P = rast.n_pix
    rng = np.random.default_rng(12)
    t_rgb = t(rng.uniform(0, 1, (P, 3)))
    t_depth = t(rng.uniform(0, 4, P) * (rng.uniform(0, 1, P) > 0.1))  # some pixels without a sensor reading
    img_ref = {k: v.clone() for k, v in rast.img.items()}
    loss_a, loss_b = torch.zeros(1, device="cuda"), torch.zeros(1, device="cuda")
    dr_a, dd_a = torch.empty(P, 3, device="cuda"), torch.empty(P, device="cuda")
    dr_b, dd_b = torch.full((P, 3), 7.0, device="cuda"), torch.full((P,), 7.0, device="cuda")
    gs.gs_loss_l1(rast.img["rgb"], rast.img["depth"], rast.img["alpha"], t_rgb, t_depth, 0.7, 0.3, gate, 0.5, loss_a,
                  dr_a, dd_a)
    gs.gs_render_fwd_l1(rast.proj, rast.n, rast.bins, rast.views, rast.img, rast.work_counter, t_rgb, t_depth, 0.7, 0.3,
                        gate, 0.5, loss_b, dr_b, dd_b)
    torch.cuda.synchronize()
    for k, v in img_ref.items():
        assert torch.equal(rast.img[k], v), k
    assert torch.equal(dr_a, dr_b) and torch.equal(dd_a, dd_b)
    assert abs(float(loss_a) - float(loss_b)) <= 1e-5 * abs(float(loss_a))


def test_batched_views_equal_plain_views():
    """Rendering several views in one launch gives the same images as one view per launch."""
    name, scene, cams = CASES[1]
    rast, p, vm = _run(scene, cams)
    batched = {k: v.cpu().numpy() for k, v in rast.img.items()}
    base = 0
    for v in range(len(cams["size"])):
        cv = scenes.cams_from(cams["intr"][v:v + 1], cams["size"][v:v + 1], cams["viewmats"][v:v + 1])
        r1, _, _ = _run(scene, cv)
        P = int(cams["size"][v][0] * cams["size"][v][1])
        for k in ("rgb", "depth", "alpha", "final_T", "n_contrib"):
            np.testing.assert_array_equal(r1.img[k].cpu().numpy(), batched[k][base:base + P])
        base += P


def test_loss_l1_and_gate_parity():
    rng = np.random.default_rng(3)
    P = 5000
    img = dict(rgb=rng.uniform(0, 1, (P, 3)).astype(np.float32), depth=rng.uniform(0, 3, P).astype(np.float32),
               alpha=rng.uniform(0.95, 1.0, P).astype(np.float32))
    img["depth"][:100] = 0.0
    t_rgb = rng.uniform(0, 1, (P, 3)).astype(np.float32)
    t_depth = rng.uniform(0, 3, P).astype(np.float32)
    t_depth[100:200] = 0.0
    for gate in (False, True):
        L, dC, dD = oracle.loss_l1(img, t_rgb, t_depth, 0.5, 1.0, gate=gate, gamma=0.99)
        loss = torch.zeros(1, device="cuda")
        d_rgb = torch.empty(P, 3, device="cuda")
        d_depth = torch.empty(P, device="cuda")
        gs.gs_loss_l1(t(img["rgb"]), t(img["depth"]), t(img["alpha"]), t(t_rgb), t(t_depth), 0.5, 1.0, gate, 0.99,
                      loss, d_rgb, d_depth)
        torch.cuda.synchronize()
        assert abs(float(loss) - L) <= 1e-5 * abs(L)
        np.testing.assert_allclose(d_rgb.cpu().numpy(), dC, rtol=1e-6, atol=1e-12)
        np.testing.assert_allclose(d_depth.cpu().numpy(), dD, rtol=1e-6, atol=1e-12)


@pytest.mark.parametrize("order", ["mixed", "grouped"])
def test_reprojection_parity(order):
    """Keypoints of mixed views (every warp adds lane by lane) and grouped by
    view, as a frame's keypoints come (whole warps of one view add up their
    terms first), with a ragged last warp."""
    rng = np.random.default_rng(4)
    vms = np.stack([scenes.look_at((0.2 * k, -0.1, 0.0), (0.1, 0.2, 3.0)) for k in range(2)])
    cams = scenes.cams_from([[525, 525, 320, 240]] * 2, [[640, 480]] * 2, vms)
    n = 1000
    pts = rng.uniform(-1, 1, (n, 3)) + [0, 0, 3]
    pts[:5, 2] = -2.0  # behind the cameras: left out
    pts = pts.astype(np.float32)
    vid = rng.integers(0, 2, n).astype(np.int32)
    if order == "grouped":
        vid = np.sort(vid)
    obs = rng.uniform(0, 640, (n, 2)).astype(np.float32)
    L, g = oracle.reproj(pts.astype(np.float64), obs.astype(np.float64), cams, weight=1.5, view_ids=vid)
    loss = torch.zeros(1, device="cuda")
    d_twist = torch.zeros(2, 6, device="cuda")
    gs.gs_reproj_loss_grad(t(pts), t(obs), t(vid, torch.int32), gs.make_views(cams["intr"], cams["size"]),
                           viewmats_on_device(cams), 1.5, loss, d_twist)
    torch.cuda.synchronize()
    assert abs(float(loss) - L) <= 1e-5 * L
    e = rel_l2(d_twist.cpu().numpy(), g)
    print(f"re-projection twist grad rel-L2 err = {e:.3e}")
    assert e <= GRAD_TOL


def test_adam_and_step_counter():
    rng = np.random.default_rng(5)
    n = 10_001
    p0 = rng.standard_normal(n)
    groups = [(0, 3001, 1e-3), (3001, 5000, 2e-2), (8001, 2000, 5e-4)]
    P, M, Vv = p0.copy(), np.zeros(n), np.zeros(n)
    tp, tm, tv = t(p0), torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    step = torch.zeros(2, dtype=torch.int32, device="cuda")
    for it in range(1, 4):
        gr = rng.standard_normal(n)
        for off, cnt, lr in groups:
            sl = slice(off, off + cnt)
            pp, mm, vv = P[sl].copy(), M[sl].copy(), Vv[sl].copy()
            oracle.adam(pp, np.ascontiguousarray(gr[sl]), mm, vv, lr=lr, t=it)
            P[sl], M[sl], Vv[sl] = pp, mm, vv
        gs.gs_adam_step(tp, t(gr), tm, tv, groups, step)
        torch.cuda.synchronize()
        assert int(step[0]) == it and int(step[1]) == 0
        np.testing.assert_allclose(tp.cpu().numpy(), P, rtol=1e-5, atol=1e-6)


def test_pose_update_matches_oracle_exp():
    rng = np.random.default_rng(6)
    vms = np.stack([scenes.look_at((0.1 * k, 0.0, 0.0), (0.0, 0.0, 3.0)) for k in range(3)])
    xi = rng.normal(0, 0.05, (3, 6))
    xi[2] = 1e-8
    vm = viewmats_on_device(dict(viewmats=vms))
    tw = t(xi)
    gs.gs_pose_update(vm, tw)
    torch.cuda.synchronize()
    for v in range(3):
        ref = oracle.se3_exp_apply(xi[v].astype(np.float32).astype(np.float64), vms[v].astype(np.float64))
        np.testing.assert_allclose(vm[v].view(3, 4).cpu().numpy(), ref, atol=2e-6)
    assert float(tw.abs().max()) == 0.0


def test_edge_cases_empty_and_tiny():
    cams = scenes.pinhole(37, 23, 30.0)  # ragged 3 x 2 tiles
    # all Gaussians behind the camera
    sc = scenes.cube_scene(50, seed=8)
    sc["means"][:, 2] = -3.0
    rast, p, vm = _run(sc, cams)
    assert rast.n_pairs() == 0 and rast.status() == 0
    assert float(rast.img["alpha"].abs().max()) == 0.0 and float(rast.img["final_T"].min()) == 1.0
    grads = zero_grads(p)
    rast.backward(p, vm, torch.ones(37 * 23, 3, device="cuda"), None, None, grads)
    torch.cuda.synchronize()
    assert all(float(g.abs().max()) == 0.0 for g in grads.values())
    # a single Gaussian
    sc1 = scenes.cube_scene(1, seed=9, log_scale=(-2.0, 0.0))
    sc1["means"][:] = [0.05, -0.02, 2.0]
    rast, p, vm = _run(sc1, cams)
    ref = oracle.forward(sc1, cams)["img"]
    check_image({k: v.cpu().numpy() for k, v in rast.img.items()}, ref, "single-gaussian-37x23", log=False)


def test_capacity_overflow_is_reported_not_fatal():
    c = scenes.config(1)
    rast, p, vm = _run(c["scene"], c["cams"], capacity=500)
    geom = oracle.project_geom(c["scene"], c["cams"])
    assert rast.status() & (1 << 3)
    assert rast.n_pairs() == int(geom["kept"].sum()) > 500
    # the pipeline still completes with in-bounds output
    assert torch.isfinite(rast.img["rgb"]).all()


def test_every_compositing_variant_matches():
    """All forward variants give bit-identical images; every backward variant
    meets the gradient bar against the oracle."""
    name, scene, cams = CASES[1]
    fwd0, bwd0, n_fwd, n_bwd = gs.gs_get_render_variants()
    try:
        ref_img = None
        for fv in range(n_fwd):
            gs.gs_set_render_variants(fv, bwd0)
            rast, p, vm = _run(scene, cams)
            img = {k: v.cpu().numpy() for k, v in rast.img.items()}
            if ref_img is None:
                ref_img = img
            for k in img:
                np.testing.assert_array_equal(img[k], ref_img[k], err_msg=f"fwd variant {fv} {k}")
        for bv in range(n_bwd):
            gs.gs_set_render_variants(fwd0, bv)
            out, gref = _backward_case(scene, cams)
            for k in (*PARAM_KEYS, "twist"):
                e = rel_l2(out[k], gref[k])
                assert e <= GRAD_TOL, (bv, k, e)
            print(f"bwd variant {bv}: max rel-L2 {max(rel_l2(out[k], gref[k]) for k in out):.2e}")
    finally:
        gs.gs_set_render_variants(fwd0, bwd0)


SSIM_SIZES = {
    # odd widths: the gradient pass stages with 4-byte copies
    "odd": [[45, 37], [64, 48], [19, 23], [131, 101]],
    # widths a multiple of 4: the gradient pass stages with the tensor memory accelerator
    "aligned": [[44, 37], [64, 48], [20, 23], [132, 101], [200, 120]],
    # full-size views (the mapping workloads' 1200x680 and 1280x720; one odd width)
    "fullsize": [[1200, 680], [1280, 720]],
    "fullsize-odd": [[962, 541]],
}


@pytest.mark.parametrize("sizes", list(SSIM_SIZES))
def test_ssim_term_parity(sizes):
    """The SSIM term of L_m against the FP64 oracle on uneven views (several
    tiles and ragged edges), added on top of an existing gradient."""
    from oracle import ssim as S
    rng = np.random.default_rng(7)
    size = np.array(SSIM_SIZES[sizes])
    P = int((size[:, 0] * size[:, 1]).sum())
    x = rng.uniform(0, 1, (P, 3)).astype(np.float32)
    y = np.clip(x + rng.normal(0, 0.15, x.shape), 0, 1).astype(np.float32)
    L, g = S.loss_ssim(x.astype(np.float64), y.astype(np.float64), size, weight=0.3)
    views = gs.make_views([[50, 50, 20, 20]] * len(size), size)
    loss = torch.full((1,), 0.25, device="cuda")
    base = rng.normal(0, 1e-5, (P, 3)).astype(np.float32)
    d_rgb = t(base)
    ws = torch.empty(gs.gs_ssim_workspace_size(P), dtype=torch.uint8, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    gs.gs_loss_ssim(t(x), t(y), views, 0.3, loss, d_rgb, ws, status)
    torch.cuda.synchronize()
    assert gs.gs_get_device_status(status) == 0
    e = rel_l2(d_rgb.cpu().numpy() - base, g)
    le = abs(float(loss) - 0.25 - L)
    print(f"SSIM gradient rel-L2 err = {e:.3e}, loss {float(loss) - 0.25:.6f} vs {L:.6f}")
    parity_log(dict(kind="ssim", name=f"ssim-{sizes}", pixels=P, views=len(size), loss_abs_err=le, grad_rel_l2=e))
    assert le <= 2e-6 * max(1.0, L)
    assert e <= GRAD_TOL


TILES = [(8, 8), (16, 8), (32, 16), (16, 32), (32, 32), (64, 32)]


@pytest.mark.parametrize("tile", TILES, ids=[f"{a}x{b}" for a, b in TILES])
def test_tile_shapes_match_oracle(tile):
    """Every tile shape the autotuner may pick, against the oracle run with the
    same tiles: rectangles, keys, lists and ranges bit for bit; the images of
    every compositing variant whose band fits the tile (32- and 64-entry
    chunks) identical to each other and within the image bar; the gradients of
    every fitting backward variant within the gradient bar."""
    name, scene, cams = CASES[1]
    fwd0, bwd0, n_fwd, n_bwd = gs.gs_get_render_variants()
    try:
        rast = make_rast(scene, cams, tile=tile)
        p = params_on_device(scene)
        vm = viewmats_on_device(cams)
        rast.forward(p, vm)
        torch.cuda.synchronize()
        assert rast.status() == 0
        geom = oracle.project_geom(scene, cams, tile=tile)
        _, radii, _, rect = gpu_geom(rast)
        vis = geom["radius"] > 0
        np.testing.assert_array_equal(rect[vis], geom["rect"][vis])
        bins = oracle.bin_tiles(cams, geom, tile)
        keys, vals, ranges = gpu_bins(rast)
        assert rast.n_pairs() == bins["n_pairs"]
        np.testing.assert_array_equal(keys, bins["keys"])
        np.testing.assert_array_equal(vals, bins["vals"])
        np.testing.assert_array_equal(ranges, bins["ranges"])
        ref = oracle.forward(scene, cams, tile=tile)
        first = None
        fitting = [v for v in range(n_fwd) if gs.variant_fits(v, tile)]
        assert len(fitting) >= 4
        for fv in fitting:
            gs.gs_set_render_variants(fv, bwd0)
            gs.gs_render_fwd(rast.proj, rast.n, rast.bins, rast.views, rast.img, rast.work_counter)
            img = {k: v.cpu().numpy() for k, v in rast.img.items()}
            if first is None:
                first = img
                check_image(img, ref["img"], f"{name} tile {tile[0]}x{tile[1]}")
                check_single_blend_alpha(img, ref, cams, f"{name} tile {tile[0]}x{tile[1]}", tile)
            for k in img:
                np.testing.assert_array_equal(img[k], first[k], err_msg=f"fwd variant {fv} {k}")
        keep = ref["img"]["flags"] == 0
        rng = np.random.default_rng(21)
        P = rast.n_pix
        dC, dD, dA = rng.normal(0, 1, (P, 3)), rng.normal(0, 1, P), rng.normal(0, 1e-2, P)
        dC[~keep], dD[~keep], dA[~keep] = 0, 0, 0
        g2d = oracle.render_bwd(cams, ref["proj"], ref["drec"], ref["bins"], ref["geom"]["n"], dC, dD, dA, tile)
        worst = 0.0
        for bv in range(n_bwd):
            if not gs.variant_fits(bv, tile):
                continue
            gs.gs_set_render_variants(fwd0, bv)
            rast.grad2d.zero_()
            gs.gs_render_bwd_splats(rast.proj, rast.n, rast.bins, rast.views, rast.img, t(dC), t(dD), t(dA),
                                    rast.grad2d, rast.work_counter)
            torch.cuda.synchronize()
            G = rast.grad2d.view(-1, 12).cpu().numpy()[:, :10]
            e = rel_l2(G, g2d)
            worst = max(worst, e)
            assert e <= GRAD_TOL, (bv, e)
        parity_log(dict(kind="grad", name=f"{name} tile {tile[0]}x{tile[1]} all bwd variants", g2d=worst))
    finally:
        gs.gs_set_render_variants(fwd0, bwd0)
