"""Test-only helpers: an independent FP64 numpy restatement of the projection
for tiny scenes (used as brute force against the oracle), and masks."""
import numpy as np
from scipy.spatial.transform import Rotation

import scenes


def rotation_from_quat(q):
    """Rotation matrices from (w, x, y, z) quaternions, through scipy (scalar last)."""
    q = np.asarray(q, np.float64)
    return Rotation.from_quat(np.concatenate([q[:, 1:], q[:, :1]], 1)).as_matrix()


def pinhole_jacobian_numeric(p, fx, fy, h=1e-6):
    """Central-difference Jacobian of (fx x/z, fy y/z) with respect to p."""
    J = np.zeros((2, 3))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h * max(1.0, abs(p[k]))
        a, b = p + e, p - e
        J[:, k] = (np.array([fx * a[0] / a[2], fy * a[1] / a[2]]) -
                   np.array([fx * b[0] / b[2], fy * b[1] / b[2]])) / (2 * e[k])
    return J


def project_bruteforce(scene, intr, viewmat, blur):
    """FP64 2D mean, covariance, depth, opacity of each Gaussian (no clamping of
    the Jacobian; callers keep Gaussians inside 1.3x the field of view)."""
    fx, fy, cx, cy = (float(v) for v in intr)
    E = np.asarray(viewmat, np.float64)
    W, t = E[:, :3], E[:, 3]
    mu = np.asarray(scene["means"], np.float64)
    R = rotation_from_quat(scene["quats"])
    s = np.exp(np.asarray(scene["log_scales"], np.float64))
    out = []
    for i in range(mu.shape[0]):
        p = W @ mu[i] + t
        S3 = R[i] @ np.diag(s[i] ** 2) @ R[i].T
        J = pinhole_jacobian_numeric(p, fx, fy)
        S2 = J @ W @ S3 @ W.T @ J.T + blur * np.eye(2)
        uv = np.array([fx * p[0] / p[2] + cx, fy * p[1] / p[2] + cy])
        o = 1.0 / (1.0 + np.exp(-float(scene["opacity_logit"][i])))
        out.append(dict(uv=uv, cov=S2, z=p[2], o=o, p=p))
    return out


def flagged_weights(flags, *arrays):
    """Zero the per-pixel weights at flagged pixels."""
    keep = (np.asarray(flags) == 0)
    res = []
    for a in arrays:
        a = np.array(a, np.float64, copy=True)
        if a.ndim == 2:
            a[~keep] = 0.0
        else:
            a[~keep] = 0.0
        res.append(a)
    return res


def grad_scene(deg, seed, edge=False):
    """40 Gaussians 3 m ahead for gradient checks; with edge, some are near
    opaque (alpha clamp active) and some lie beyond 1.3x the half field of
    view (tangent clamp active)."""
    sc = scenes.cube_scene(40, seed=seed, sh_degree=deg, centre=(0.1, -0.05, 3.0), half=0.8,
                           log_scale=(-2.8, 0.3))
    if edge:
        # near-opaque Gaussians (alpha clamp at 0.99 active near their centres) and
        # large ones beyond 1.3x the half field of view (tangent clamp active)
        sc["opacity_logit"][:6] = 6.0
        sc["means"][6:10] = [[3.0, 0.2, 3.0], [-3.1, -0.3, 3.0], [0.3, 2.4, 3.0], [-0.2, -2.5, 3.1]]
        sc["log_scales"][6:10] = -0.9
    # keep colours inside (0, 1) so that no channel sits near the clamp at 0
    rng = np.random.default_rng(seed + 7)
    sc["sh"][:, 0, :] = (rng.uniform(0.3, 0.7, (40, 3)) - 0.5) / scenes.SH_C0
    sc["sh"][:, 1:, :] *= 0.5
    return {k: (v.astype(np.float64) if isinstance(v, np.ndarray) else v) for k, v in sc.items()}


def grad_cams(oblique):
    """64x48 pinhole (f = 60), straight ahead or oblique."""
    if oblique:
        vm = scenes.look_at((0.25, -0.2, -0.3), (0.05, 0.1, 3.0))
        return scenes.pinhole(64, 48, 60.0, viewmats=vm[None])
    return scenes.pinhole(64, 48, 60.0)
