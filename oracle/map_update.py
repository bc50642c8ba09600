"""Map maintenance and keyframe choice (test infrastructure only), numpy.

* Densification (Sec. 3.4, Eq. d: d = r f): for each pixel, in pixel order, with
  border mask alpha below a threshold and positive sensor depth d, a Gaussian at
  the back-projection of the pixel centre (world = R^T (p_c - t) for the pose
  [R | t]), isotropic with radius r = d / f, identity rotation, the pixel's
  colour as the degree-0 SH band and a given opacity logit.
* Pruning (Sec. 3.4, tau = 0.005): keep a Gaussian when sigmoid(logit) >= tau;
  the decision is taken on the FP32 logit against log(tau / (1 - tau)) rounded
  to FP32, as the kernel takes it.
* View point selection (Sec. 3.3): keyframe i >= 1 is selected when
  beta <= M_{i-1,i} < alpha T_{i-1,i}; the first keyframe always is.
"""
from __future__ import annotations

import math

import numpy as np

SH_C0 = 0.5 / math.sqrt(math.pi)


def densify(alpha, t_rgb, t_depth, cams, threshold, opacity_logit, sh_degree):
    alpha = np.asarray(alpha, np.float32)
    depth = np.asarray(t_depth, np.float32)
    rgb = np.asarray(t_rgb, np.float64)
    sel = (alpha < np.float32(threshold)) & (depth > 0)
    idx = np.nonzero(sel)[0]
    size = np.asarray(cams["size"], np.int64)
    pix_base = np.concatenate([[0], np.cumsum(size[:, 0] * size[:, 1])[:-1]])
    v = np.searchsorted(pix_base, idx, side="right") - 1
    K = (sh_degree + 1) ** 2
    out = dict(means=np.zeros((len(idx), 3)), log_scales=np.zeros((len(idx), 3)), quats=np.zeros((len(idx), 4)),
               opacity_logit=np.full(len(idx), float(opacity_logit)), sh=np.zeros((len(idx), K, 3)))
    for j, (p, vv) in enumerate(zip(idx, v)):
        fx, fy, cx, cy = (float(x) for x in cams["intr"][vv])
        W = int(size[vv, 0])
        lp = p - pix_base[vv]
        px, py = lp % W + 0.5, lp // W + 0.5
        d = float(depth[p])
        pc = np.array([(px - cx) / fx * d, (py - cy) / fy * d, d])
        E = np.asarray(cams["viewmats"][vv], np.float64).reshape(3, 4)
        out["means"][j] = E[:, :3].T @ (pc - E[:, 3])
        out["log_scales"][j] = math.log(d / fx)
        out["quats"][j] = [1.0, 0.0, 0.0, 0.0]
        out["sh"][j, 0] = (rgb[p] - 0.5) / SH_C0
    return idx, out


def prune_select(opacity_logit, tau):
    logit = np.asarray(opacity_logit, np.float32)
    cut = np.float32(math.log(tau / (1.0 - tau)))
    keep = logit >= cut
    new_index = np.where(keep, np.cumsum(keep) - 1, -1).astype(np.int32)
    return new_index, int(keep.sum())


def select_views(matches, totals, alpha=0.75, beta=20):
    out = []
    for i, (m, t) in enumerate(zip(matches, totals)):
        out.append(1 if i == 0 else int(beta <= m < alpha * t))
    return out
