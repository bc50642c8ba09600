"""Helpers shared by the GPU parity tests: move seeded inputs to the device, run
the CUDA path through the C ABI, and compare with the oracle."""
import numpy as np
import torch

import oracle
import paper_2405_19614_gb300 as gs

PARAM_KEYS = ("means", "log_scales", "quats", "opacity_logit", "sh")


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


def make_rast(scene, cams, capacity=None):
    return gs.Rasterizer(scene["means"].shape[0], scene["sh_degree"], cams["intr"], cams["size"],
                         pair_capacity=capacity)


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
