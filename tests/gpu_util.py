"""Helpers shared by the GPU parity tests: move seeded inputs to the device, run
the CUDA path through the C ABI, and compare with the oracle.

Image bar: RGB, depth, alpha and final T within IMG_TOL absolute of the FP64
oracle on every pixel whose stop decision (T (1 - alpha) < 1e-4) is not in the
oracle's transmittance band; at most MAX_FLAGGED of the pixels in the band,
each within IMG_TOL plus the exact contribution of the entry at that decision
(a result stopping one entry earlier or later differs by that much); last
indices equal on the unflagged pixels.  The alpha skip and clamp decisions are
bit-exact on both sides, so they flag nothing.  Each comparison's figures
(per-output max abs error, rel-L2 per gradient tensor, flagged count) are
appended as JSON lines to the file named by GS_PARITY_LOG, when set."""
import json
import os

import numpy as np
import torch

import oracle
import paper_2405_19614_gb300 as gs

PARAM_KEYS = ("means", "log_scales", "quats", "opacity_logit", "sh")
IMG_TOL = 1e-4
GRAD_TOL = 1e-3
MAX_FLAGGED = 1e-4  # 0.01 % of the pixels


def parity_log(record):
    path = os.environ.get("GS_PARITY_LOG")
    if path:
        with open(path, "a") as fh:
            fh.write(json.dumps(record) + "\n")


def check_image(img, ref, name, log=True):
    """img: the CUDA path's images (numpy, the same pixels as ref); ref: the
    oracle's render of them."""
    keep = ref["flags"] == 0
    n_flag = int((~keep).sum())
    rec = dict(kind="image", name=name, pixels=int(keep.size), flagged=n_flag)
    print(f"{name}: {n_flag} of {keep.size} pixels with the stop decision in the transmittance band")
    assert n_flag <= MAX_FLAGGED * keep.size, (n_flag, keep.size)
    slack = ref["slack"]
    extra = {"rgb": slack[:, 1:2], "depth": slack[:, 2], "alpha": slack[:, 0], "final_T": slack[:, 0]}
    for k in ("rgb", "depth", "alpha", "final_T"):
        diff = np.abs(np.asarray(img[k], np.float64) - ref[k])
        err = float(diff[keep].max()) if keep.any() else 0.0
        rec[f"max_abs_{k}"] = err
        print(f"{name}: max |{k} err| = {err:.3e}")
        assert err <= IMG_TOL, k
        if n_flag:
            allowed = IMG_TOL + np.broadcast_to(extra[k], diff.shape) * (1 + 1e-6)
            assert np.all(diff[~keep] <= allowed[~keep]), k
            rec[f"max_abs_{k}_flagged"] = float(diff[~keep].max())
    np.testing.assert_array_equal(np.asarray(img["n_contrib"])[keep], ref["n_contrib"][keep])
    if log:
        parity_log(rec)
    return rec


def check_single_blend_alpha(img, fwd, cams, name, tile=(16, 16)):
    """Where a pixel blends only the first entry of its list, its depth is
    z * alpha with alpha the kernel's 2^l2 (T = 1): relative to 2^l2 on the
    oracle's FP32 l2 it must stay within the approximate exponential's bound
    that the oracle's transmittance band assumes, plus the depth's rounding.
    Returns the number of pixels checked."""
    from oracle import EX2_REL, L2_ALPHA_MAX, blend_l2
    bins, drec, geom = fwd["bins"], fwd["drec"], fwd["geom"]
    n = geom["n"]
    sel = np.nonzero((fwd["img"]["flags"] == 0) & (fwd["img"]["n_contrib"] == 1))[0]
    if len(sel) == 0:
        return 0
    width = np.asarray(cams["size"], np.int64)[:, 0]
    v = np.searchsorted(bins["pix_base"], sel, side="right") - 1
    local = sel - bins["pix_base"][v]
    py, px = local // width[v], local % width[v]
    tile_id = bins["tile_base"][v] + (py // tile[1]) * bins["ntx"][v] + px // tile[0]
    o = v * n + bins["vals"][bins["ranges"][tile_id, 0]].astype(np.int64)
    l2 = blend_l2(drec[o], px, py)
    a_ref = np.where(l2 >= L2_ALPHA_MAX, float(np.float32(0.99)), 2.0 ** l2.astype(np.float64))
    z = geom["uvz"][o, 2].astype(np.float64)
    a_gpu = np.asarray(img["depth"], np.float64)[sel] / z
    rel = np.abs(a_gpu / a_ref - 1.0)
    print(f"{name}: {len(sel)} single-blend pixels, max relative alpha error {rel.max():.3e} "
          f"(bound {EX2_REL + 2.0 ** -23:.3e})")
    assert np.all(rel <= EX2_REL + 2.0 ** -23)
    parity_log(dict(kind="ex2", name=name, pixels=int(len(sel)), max_rel_alpha_err=float(rel.max())))
    return len(sel)


def dev():
    return torch.device("cuda:0")


def t(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=dev())


def params_on_device(scene):
    p = {k: t(scene[k]) for k in PARAM_KEYS}
    p["sh_degree"] = int(scene["sh_degree"])
    return p


def viewmats_on_device(cams):
    return t(np.asarray(cams["viewmats"], np.float32).reshape(-1, 12))


def make_rast(scene, cams, capacity=None, tile=(16, 16)):
    return gs.Rasterizer(scene["means"].shape[0], scene["sh_degree"], cams["intr"], cams["size"],
                         pair_capacity=capacity, tile=tile)


def zero_grads(p):
    return {k: torch.zeros_like(p[k]) for k in PARAM_KEYS}


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def gpu_geom(rast):
    rec = rast.proj["rec"].view(-1, 12).cpu().numpy()
    radii = rast.proj["radii"].cpu().numpy()
    tt = rast.proj["tiles_touched"].cpu().numpy().view(np.uint32)
    rr = rast.proj["rect"].cpu().numpy().view(np.uint32)
    r0, r1 = rr[:, 0], rr[:, 1]
    rect = np.stack([r0 & 0xFFFF, r0 >> 16, r1 & 0xFFFF, r1 >> 16], 1).astype(np.int32)
    return rec, radii, tt, rect


def gpu_bins(rast):
    K = min(rast.n_pairs(), rast.capacity)
    keys = rast.bins["keys"][:K].cpu().numpy().view(np.uint64)
    vals = rast.bins["vals"][:K].cpu().numpy().view(np.uint32)
    ranges = rast.bins["ranges"].cpu().numpy().view(np.uint32)
    return keys, vals, ranges


def oracle_targets(target_scene, cams):
    tgt = oracle.forward(target_scene, cams)["img"]
    return tgt["rgb"].astype(np.float32), tgt["depth"].astype(np.float32)
