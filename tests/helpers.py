"""Test-only helpers: an independent FP64 numpy restatement of the projection
for tiny scenes (used as brute force against the oracle), and masks."""
import numpy as np
from scipy.spatial.transform import Rotation


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
