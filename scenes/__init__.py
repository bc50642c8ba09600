"""Seeded synthetic inputs shaped like the RGB-D workloads of arXiv 2405.19614.

This module is shared by the tests, the oracle legs and the CUDA legs.  It
holds none of the method's arithmetic (no projection, no compositing, no loss):
only random Gaussian parameters, camera intrinsics and poses, keypoint pixel
positions and noise.  Targets that need a render are made by the caller.

The paper evaluates on TUM RGB-D (640x480 handheld sequences, Sec. 4.1); that
dataset is not available here, so these seeded scenes stand in for its shapes:
indoor box rooms with objects, Gaussians on surfaces, 640x480 and Replica-like
1200x680 views.

Conventions: world -> camera matrices are row-major 3x4 [R | t] with the camera
looking along +z, x right, y down; the world is z-up.  Quaternions are (w, x, y, z).
"""
from __future__ import annotations

import math

import numpy as np

SH_C0 = 0.28209479177387814  # 1 / (2 sqrt(pi)): degree-0 basis value


def _sh_count(deg: int) -> int:
    return (deg + 1) ** 2


def random_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def look_at(eye, target, up=(0.0, 0.0, 1.0)):
    """World -> camera 3x4 matrix for a camera at eye looking at target."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    if np.linalg.norm(r) < 1e-8:
        r = np.cross(f, np.array([0.0, 1.0, 0.0]))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f])
    t = -R @ eye
    return np.concatenate([R, t[:, None]], axis=1).astype(np.float32)


def cams_from(intr, size, viewmats):
    return dict(intr=np.asarray(intr, np.float32).reshape(-1, 4),
                size=np.asarray(size, np.int32).reshape(-1, 2),
                viewmats=np.asarray(viewmats, np.float32).reshape(-1, 3, 4))


def pinhole(width, height, f, n_views=1, viewmats=None):
    intr = np.tile(np.array([f, f, width / 2.0, height / 2.0], np.float32), (n_views, 1))
    size = np.tile(np.array([width, height], np.int32), (n_views, 1))
    if viewmats is None:
        viewmats = np.tile(np.concatenate([np.eye(3), np.zeros((3, 1))], 1), (n_views, 1, 1))
    return cams_from(intr, size, viewmats)


# --------------------------------------------------------------------------
# Gaussian clouds
# --------------------------------------------------------------------------

def cube_scene(n, seed, sh_degree=0, centre=(0.0, 0.0, 3.0), half=1.0, log_scale=(-3.5, 0.5),
               opacity=(0.0, 1.0)):
    """Means uniform in a cube (default 2 m, 3 m ahead of an identity camera),
    log-scales N(mu, sd), uniform random rotations, opacity logits N(mu, sd),
    colours U(0,1) stored as the degree-0 SH coefficient, higher bands N(0, 0.1)."""
    rng = np.random.default_rng(seed)
    means = (rng.uniform(-half, half, (n, 3)) + np.asarray(centre)).astype(np.float32)
    ls = rng.normal(log_scale[0], log_scale[1], (n, 3)).astype(np.float32)
    quats = random_quats(rng, n)
    ol = rng.normal(opacity[0], opacity[1], n).astype(np.float32)
    K = _sh_count(sh_degree)
    sh = np.zeros((n, K, 3), np.float32)
    colours = rng.uniform(0.0, 1.0, (n, 3))
    sh[:, 0, :] = (colours - 0.5) / SH_C0
    if K > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.1, (n, K - 1, 3))
    return dict(means=means, log_scales=ls, quats=quats, opacity_logit=ol, sh=sh, sh_degree=sh_degree)


def _box_faces(lo, hi, inward):
    """Six faces of an axis-aligned box as (origin, edge_u, edge_v, normal)."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    d = hi - lo
    faces = []
    for ax in range(3):
        a1, a2 = [a for a in range(3) if a != ax]
        for side in (0, 1):
            o = lo.copy()
            o[ax] = hi[ax] if side else lo[ax]
            eu = np.zeros(3)
            eu[a1] = d[a1]
            ev = np.zeros(3)
            ev[a2] = d[a2]
            nrm = np.zeros(3)
            nrm[ax] = 1.0 if side else -1.0
            if inward:
                nrm = -nrm
            faces.append((o, eu, ev, nrm))
    return faces


def room_layout(seed, room=(6.0, 5.0, 3.0), n_cuboids=20, walls=()):
    """Box room [-X/2, X/2] x [-Y/2, Y/2] x [0, Z] with cuboids on the floor.
    walls: extra thin boxes (lo, hi) for multi-room floors."""
    rng = np.random.default_rng(seed)
    X, Y, Z = room
    faces = _box_faces((-X / 2, -Y / 2, 0.0), (X / 2, Y / 2, Z), inward=True)
    boxes = []
    for _ in range(n_cuboids):
        sx, sy, sz = rng.uniform(0.2, 1.0), rng.uniform(0.2, 1.0), rng.uniform(0.2, 1.2)
        cx = rng.uniform(-X / 2 + 0.3 + sx / 2, X / 2 - 0.3 - sx / 2)
        cy = rng.uniform(-Y / 2 + 0.3 + sy / 2, Y / 2 - 0.3 - sy / 2)
        lo, hi = (cx - sx / 2, cy - sy / 2, 0.0), (cx + sx / 2, cy + sy / 2, sz)
        boxes.append((lo, hi))
    for lo, hi in list(walls):
        boxes.append((tuple(lo), tuple(hi)))
    for lo, hi in boxes:
        for f in _box_faces(lo, hi, inward=False):
            if f[3][2] < -0.5:  # the face resting on the floor is hidden
                continue
            faces.append(f)
    return dict(room=room, faces=faces, boxes=boxes)


def surface_scene(n, seed, layout, sh_degree=3, median_scale=0.015, scale_sd=0.3,
                  normal_sd=0.01, sh_sd=0.1, opacity=(1.0, 1.0)):
    """Gaussians sampled area-weighted on the layout's faces, offset N(0, normal_sd)
    along the normal; per-axis log-scales N(ln median_scale, scale_sd^2); SH
    coefficients N(0, sh_sd) with the degree-0 band centred on a per-face colour."""
    rng = np.random.default_rng(seed)
    faces = layout["faces"]
    areas = np.array([np.linalg.norm(np.cross(eu, ev)) for _, eu, ev, _ in faces])
    fid = rng.choice(len(faces), size=n, p=areas / areas.sum())
    uv = rng.uniform(0.0, 1.0, (n, 2))
    O = np.stack([f[0] for f in faces])[fid]
    EU = np.stack([f[1] for f in faces])[fid]
    EV = np.stack([f[2] for f in faces])[fid]
    NR = np.stack([f[3] for f in faces])[fid]
    means = O + uv[:, :1] * EU + uv[:, 1:] * EV + rng.normal(0.0, normal_sd, (n, 1)) * NR
    ls = rng.normal(math.log(median_scale), scale_sd, (n, 3))
    quats = random_quats(rng, n)
    ol = rng.normal(opacity[0], opacity[1], n)
    K = _sh_count(sh_degree)
    sh = rng.normal(0.0, sh_sd, (n, K, 3))
    face_col = rng.uniform(0.15, 0.85, (len(faces), 3))
    sh[:, 0, :] += (face_col[fid] - 0.5) / SH_C0
    return dict(means=means.astype(np.float32), log_scales=ls.astype(np.float32), quats=quats,
                opacity_logit=ol.astype(np.float32), sh=sh.astype(np.float32), sh_degree=sh_degree)


def _clear_of_boxes(p, boxes, margin):
    for lo, hi in boxes:
        if all(lo[k] - margin <= p[k] <= hi[k] + margin for k in range(3)):
            return False
    return True


def room_poses(seed, layout, n_views, smooth=False, margin=0.8):
    """Camera poses inside the room at 1.2-1.8 m height.  smooth=True places them
    along an arc (a keyframe trajectory); otherwise independent random poses."""
    rng = np.random.default_rng(seed)
    X, Y, Z = layout["room"]
    mats = []
    if smooth:
        c = np.array([rng.uniform(-0.3, 0.3) * X / 2, rng.uniform(-0.3, 0.3) * Y / 2])
        rad = 0.25 * min(X, Y)
        a0 = rng.uniform(0, 2 * math.pi)
        for k in range(n_views):
            a = a0 + 0.35 * k
            eye = np.array([c[0] + rad * math.cos(a), c[1] + rad * math.sin(a), 1.5 + 0.1 * math.sin(a)])
            yaw = a + math.pi / 2 + 0.3 * math.sin(0.7 * k)
            pitch = -0.1 + 0.05 * math.cos(k)
            tgt = eye + np.array([math.cos(yaw) * math.cos(pitch), math.sin(yaw) * math.cos(pitch),
                                  math.sin(pitch)])
            mats.append(look_at(eye, tgt))
        return np.stack(mats)
    for _ in range(n_views):
        for _attempt in range(1000):
            eye = np.array([rng.uniform(-X / 2 + margin, X / 2 - margin),
                            rng.uniform(-Y / 2 + margin, Y / 2 - margin), rng.uniform(1.2, 1.8)])
            if _clear_of_boxes(eye, layout["boxes"], 0.4):
                break
        yaw = rng.uniform(0, 2 * math.pi)
        pitch = rng.normal(0.0, math.radians(10.0))
        tgt = eye + np.array([math.cos(yaw) * math.cos(pitch), math.sin(yaw) * math.cos(pitch),
                              math.sin(pitch)])
        mats.append(look_at(eye, tgt))
    return np.stack(mats)


def multi_room_layout(seed, floor=(30.0, 20.0, 3.0), rooms=(3, 2), n_cuboids=60):
    """A floor split into rooms by interior walls with door gaps."""
    X, Y, Z = floor
    walls = []
    t = 0.1
    for i in range(1, rooms[0]):
        x = -X / 2 + i * X / rooms[0]
        for j in range(rooms[1]):
            y0 = -Y / 2 + j * Y / rooms[1]
            y1 = y0 + Y / rooms[1]
            ym = 0.5 * (y0 + y1)
            walls.append(((x - t, y0, 0.0), (x + t, ym - 0.6, Z)))
            walls.append(((x - t, ym + 0.6, 0.0), (x + t, y1, Z)))
    for j in range(1, rooms[1]):
        y = -Y / 2 + j * Y / rooms[1]
        for i in range(rooms[0]):
            x0 = -X / 2 + i * X / rooms[0]
            x1 = x0 + X / rooms[0]
            xm = 0.5 * (x0 + x1)
            walls.append(((x0, y - t, 0.0), (xm - 0.6, y + t, Z)))
            walls.append(((xm + 0.6, y - t, 0.0), (x1, y + t, Z)))
    return room_layout(seed, floor, n_cuboids, walls)


# --------------------------------------------------------------------------
# tracking inputs
# --------------------------------------------------------------------------

def twist_perturbation(seed, trans_m, rot_deg):
    """A random twist (rho, phi) with |rho| = trans_m metres, |phi| = rot_deg degrees."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(3)
    b = rng.standard_normal(3)
    return np.concatenate([a / np.linalg.norm(a) * trans_m,
                           b / np.linalg.norm(b) * math.radians(rot_deg)])


def keypoint_pixels(seed, width, height, n, border=8):
    rng = np.random.default_rng(seed)
    px = rng.integers(border, width - border, n)
    py = rng.integers(border, height - border, n)
    return px, py


def backproject(viewmat, intr, px, py, depth_img, width):
    """World points for pixel centres (px + 0.5, py + 0.5) at the given depths
    (depth_img flattened row-major).  Returns FP64 points and a validity mask."""
    fx, fy, cx, cy = (float(v) for v in intr)
    d = np.asarray(depth_img, np.float64).reshape(-1)[py * width + px]
    xc = ((px + 0.5) - cx) / fx * d
    yc = ((py + 0.5) - cy) / fy * d
    pc = np.stack([xc, yc, d], 1)
    E = np.asarray(viewmat, np.float64)
    R, t = E[:, :3], E[:, 3]
    pw = np.linalg.solve(R, (pc - t).T).T  # float32 poses are not exactly orthonormal
    return pw, d > 0.3


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------

CONFIG_NAMES = {
    1: "plain-2k-sh0-64x48",
    2: "replica-300k-sh3-1200x680",
    3: "tum-track-100k-sh3-640x480",
    4: "batched-1M-sh3-8x1200x680",
    5: "long-4M-sh3-16-uneven",
}


def config(idx: int, scale: float = 1.0):
    """Scene, cameras and loss settings of workload idx (1..5).  scale < 1 shrinks
    the Gaussian count (for tests), keeping everything else."""
    if idx == 1:
        n = max(1, int(2000 * scale))
        scene = cube_scene(n, seed=1, sh_degree=0)
        target_scene = cube_scene(n, seed=101, sh_degree=0)
        cams = pinhole(64, 48, 60.0)
        return dict(name=CONFIG_NAMES[1], scene=scene, cams=cams, target_scene=target_scene,
                    w_c=1.0, w_d=1.0, gate=False)
    if idx == 2:
        n = max(1, int(300_000 * scale))
        lay = room_layout(2)
        scene = surface_scene(n, 2, lay)
        target_scene = surface_scene(n, 202, lay)
        vm = room_poses(2, lay, 1)
        cams = cams_from([[600.0, 600.0, 600.0, 340.0]], [[1200, 680]], vm)
        return dict(name=CONFIG_NAMES[2], scene=scene, cams=cams, target_scene=target_scene,
                    w_c=1.0, w_d=0.1, gate=False)
    if idx == 3:
        n = max(1, int(100_000 * scale))
        lay = room_layout(3, room=(4.0, 4.0, 3.0), n_cuboids=12)
        scene = surface_scene(n, 3, lay)
        vm = room_poses(3, lay, 1)
        cams = cams_from([[525.0, 525.0, 320.0, 240.0]], [[640, 480]], vm)
        return dict(name=CONFIG_NAMES[3], scene=scene, cams=cams, layout=lay,
                    motion=twist_perturbation(33, 0.02, 1.0), init_offset=twist_perturbation(34, 0.01, 0.5),
                    noise_seed=35, keypoint_seed=36, n_keypoints=1000, n_sub=7, iters=100,
                    w_rpj=1.5, w_c=0.5, w_d=1.0, gate=True, gamma=0.99)
    if idx == 4:
        n = max(1, int(1_000_000 * scale))
        lay = room_layout(4)
        scene = surface_scene(n, 4, lay)
        target_scene = surface_scene(n, 404, lay)
        vm = room_poses(4, lay, 8, smooth=True)
        intr = np.tile([600.0, 600.0, 600.0, 340.0], (8, 1))
        cams = cams_from(intr, np.tile([1200, 680], (8, 1)), vm)
        return dict(name=CONFIG_NAMES[4], scene=scene, cams=cams, target_scene=target_scene,
                    w_c=1.0, w_d=0.5, zeta=0.3, gate=False, iters=20)
    if idx == 5:
        n = max(1, int(4_000_000 * scale))
        lay = multi_room_layout(5)
        scene = surface_scene(n, 5, lay)
        target_scene = surface_scene(n, 505, lay)
        sizes = [(640, 480)] * 4 + [(960, 540)] * 4 + [(1200, 680)] * 4 + [(1280, 720)] * 4
        vm = room_poses(5, lay, 16, smooth=True)
        intr = [[0.5 * w, 0.5 * w, 0.5 * w, 0.5 * h] for (w, h) in sizes]
        cams = cams_from(intr, sizes, vm)
        return dict(name=CONFIG_NAMES[5], scene=scene, cams=cams, target_scene=target_scene,
                    w_c=1.0, w_d=0.5, zeta=0.3, gate=False, iters=20)
    raise ValueError(f"unknown workload {idx}")


def flat_params(scene):
    """All Gaussian parameters packed in one float32 buffer (means, log_scales,
    quats, opacity_logit, sh), with the slices of each tensor."""
    n = scene["means"].shape[0]
    parts = [("means", 3), ("log_scales", 3), ("quats", 4), ("opacity_logit", 1),
             ("sh", 3 * _sh_count(scene["sh_degree"]))]
    total = sum(w for _, w in parts) * n
    buf = np.zeros(total, np.float32)
    off = 0
    slices = {}
    for name, w in parts:
        buf[off:off + w * n] = np.asarray(scene[name], np.float32).reshape(-1)
        slices[name] = (off, w * n)
        off += w * n
    return buf, slices
