"""CPU oracle for the differentiable Gaussian splatting hot path (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` and
``--impl reference`` legs of ``bench.py`` may import this package.  It shares no
code with the CUDA path and never imports it.

The arithmetic lives in ``gs_oracle.c`` (plain C: FP64, plus the FP32 geometry
that decides tile membership and order).  This module compiles it with gcc and
wraps each function with numpy marshalling only.

Paper passages followed (arXiv 2405.19614):
  * Sec. 3.4 "Gaussian Representation", Eq. gauss: f(x) = o exp(-|x-mu|^2 / 2r^2),
    generalised to the anisotropic EWA footprint of the rasteriser of Sec. 4.1.
  * Sec. 3.4 "Projection" / "Differentiable Rasterization": mu2D = K E_t mu / d,
    front-to-back sorting, C(p) = sum c_i f_i prod_{j<i} (1 - f_j), D(p) likewise.
  * Sec. 3.3 border mask M_b(p) (= accumulated opacity) and filter gates G(p).
  * Sec. 3.3 joint loss L = w1 L_rpj + w2 L_c + w3 L_d; Sec. 3.2 Eq. lba (L_rpj).
  * Sec. 3.4 mapping loss L_m (L1 parts), gradient-based optimisation.
  * Sec. 4 RGB-D keyframes (TUM RGB-D: 8-bit colour, 16-bit depth) decoded to
    the FP32 loss targets (decode_keyframes).

Parity pins for every function are in tests/test_oracle_*.py; none is unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

ALPHA_MIN = 1.0 / 255.0
ALPHA_MAX = 0.99
T_MIN = 1e-4
FLAG_ALPHA_MIN, FLAG_T_MIN, FLAG_ALPHA_MAX = 1, 2, 4
# the FP32 cuts of the decisions on l2 = log2(raw alpha): log2(1/255) and
# log2(0.99), each rounded to the nearest float32
L2_ALPHA_MIN = float(np.float32(-7.994353436858858))
L2_ALPHA_MAX = float(np.float32(-0.014499569695115089))
# relative error bound the transmittance band assumes for the kernel's 2^x
# (two units in the last place; measured over every FP32 input in [-8, 0): 2^-22.73)
EX2_REL = 2.0 ** -22


def build(force: bool = False) -> str:
    """Compile gs_oracle.c into liboracle.so next to it (gcc, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class View(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_double), ("fy", ctypes.c_double), ("cx", ctypes.c_double),
                ("cy", ctypes.c_double), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("viewmat", ctypes.c_double * 12)]


class Margins(ctypes.Structure):
    _fields_ = [("margin_alpha", ctypes.c_double), ("margin_T", ctypes.c_double)]


_lib = None


def _L():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i32, i64, f32, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double
        _lib.orc_geom_expf.argtypes = [f32]
        _lib.orc_geom_expf.restype = f32
        _lib.orc_geom_log2f.argtypes = [f32]
        _lib.orc_geom_log2f.restype = f32
        _lib.orc_blend_records.argtypes = [i32, P, i64, P, P, P, P, f32, f32, i32, i32, P]
        _lib.orc_blend_l2_many.argtypes = [i64, P, P, P, P]
        _lib.orc_project_geom.argtypes = [i32, P, i64, P, P, P, f32, f32, i32, i32, P, P, P, P]
        _lib.orc_bin.argtypes = [i32, P, i64, i32, i32, P, P, P, P, i64, P, P, P]
        _lib.orc_tile_cull.argtypes = [i32, P, i64, P, P, i32, i32, P, P]
        _lib.orc_sh_eval.argtypes = [P, i64, i32, P]
        _lib.orc_project64.argtypes = [i32, P, i64, P, P, P, P, P, i32, f64, P, P]
        _lib.orc_render.argtypes = [i32, P, i64, P, P, i32, i32, P, P, P, P, Margins, P, P, P, P, P, P, P]
        _lib.orc_render_bwd.argtypes = [i32, P, i64, P, P, i32, i32, P, P, P, P, P, P, P, P]
        _lib.orc_project_bwd.argtypes = [i32, P, i64, P, P, P, P, P, i32, f64, P, P, P, P, P, P, P, P]
        _lib.orc_loss_l1.argtypes = [i64, P, P, P, P, P, f64, f64, i32, f64, P, P]
        _lib.orc_loss_l1.restype = f64
        _lib.orc_reproj.argtypes = [i64, P, P, P, P, f64, f64, P]
        _lib.orc_reproj.restype = f64
        _lib.orc_adam.argtypes = [i64, P, P, P, P, f64, f64, f64, f64, i32]
        _lib.orc_se3_exp_apply.argtypes = [P, P, P]
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# --------------------------------------------------------------------------
# cameras and layout
# --------------------------------------------------------------------------

def make_views(cams) -> ctypes.Array:
    """cams: dict with intr [V,4] (fx, fy, cx, cy), size [V,2] (width, height),
    viewmats [V,3,4] (world -> camera).  Values are taken as FP64 (float32
    inputs convert exactly)."""
    intr = np.asarray(cams["intr"], np.float64)
    size = np.asarray(cams["size"], np.int32)
    vm = np.asarray(cams["viewmats"], np.float64).reshape(-1, 12)
    V = intr.shape[0]
    arr = (View * V)()
    for v in range(V):
        arr[v].fx, arr[v].fy, arr[v].cx, arr[v].cy = (float(x) for x in intr[v])
        arr[v].width, arr[v].height = int(size[v, 0]), int(size[v, 1])
        for k in range(12):
            arr[v].viewmat[k] = float(vm[v, k])
    return arr


def layout(cams, tile=(16, 16)):
    """Tile and pixel bases of the concatenated views."""
    size = np.asarray(cams["size"], np.int64)
    tw, th = tile
    ntx = (size[:, 0] + tw - 1) // tw
    nty = (size[:, 1] + th - 1) // th
    ntiles = ntx * nty
    tile_base = np.concatenate([[0], np.cumsum(ntiles)[:-1]]).astype(np.int32)
    npix = size[:, 0] * size[:, 1]
    pix_base = np.concatenate([[0], np.cumsum(npix)[:-1]]).astype(np.int64)
    return dict(tile_base=tile_base, n_tiles=int(ntiles.sum()), pix_base=pix_base,
                n_pix=int(npix.sum()), ntx=ntx, nty=nty)


# --------------------------------------------------------------------------
# forward
# --------------------------------------------------------------------------

def geom_expf(x: float) -> float:
    return float(np.float32(_L().orc_geom_expf(float(np.float32(x)))))


def geom_log2f(x: float) -> float:
    return float(np.float32(_L().orc_geom_log2f(float(np.float32(x)))))


DREC_COLS = ("u", "v", "du", "dv", "log2o", "A2", "B2", "C2")


def blend_records(params, cams, near_z=0.2, blur=0.3, tile=(16, 16)):
    """FP32 decision records [V*n, 8] (u, v, du, dv, log2 o, A', B', C') of
    every drawn (view, Gaussian), zeros elsewhere."""
    L = _L()
    means, ls, q, ol = (_c(params[k], np.float64) for k in ("means", "log_scales", "quats", "opacity_logit"))
    n = means.shape[0]
    views = make_views(cams)
    out = np.zeros((len(views) * n, 8), np.float32)
    L.orc_blend_records(len(views), views, n, _p(means), _p(ls), _p(q), _p(ol), float(near_z), float(blur),
                        tile[0], tile[1], _p(out))
    return out


def blend_l2(drec_rows, px, py):
    """FP32 l2 = log2(raw alpha) of decision records [m, 8] at pixels (px, py)."""
    d = _c(drec_rows, np.float32).reshape(-1, 8)
    px, py = _c(px, np.int32).ravel(), _c(py, np.int32).ravel()
    out = np.zeros(d.shape[0], np.float32)
    _L().orc_blend_l2_many(d.shape[0], _p(d), _p(px), _p(py), _p(out))
    return out


def project_geom(params, cams, near_z=0.2, blur=0.3, tile=(16, 16), tile_cull=True):
    """FP32 geometry (binning contract) for every (view, Gaussian): radius,
    tile rectangle and its tile count (tiles_touched), (u, v, z), the decision
    records (drec), and the tiles each drawn Gaussian keeps (tile_mask, and
    their number in kept; every tile of the rectangle without tile_cull)."""
    L = _L()
    means, ls, q = (_c(params[k], np.float64) for k in ("means", "log_scales", "quats"))
    n = means.shape[0]
    views = make_views(cams)
    V = len(views)
    radius = np.zeros(V * n, np.int32)
    rect = np.zeros((V * n, 4), np.int32)
    uvz = np.zeros((V * n, 3), np.float32)
    tt = np.zeros(V * n, np.uint32)
    L.orc_project_geom(V, views, n, _p(means), _p(ls), _p(q), float(near_z), float(blur),
                       tile[0], tile[1], _p(radius), _p(rect), _p(uvz), _p(tt))
    drec = blend_records(params, cams, near_z, blur, tile)
    mask = np.zeros(V * n, np.uint64)
    kept = tt.copy()
    if tile_cull:
        L.orc_tile_cull(V, views, n, _p(drec), _p(rect), tile[0], tile[1], _p(mask), _p(kept))
    return dict(radius=radius, rect=rect, uvz=uvz, tiles_touched=tt, n=n, n_views=V, drec=drec,
                tile_mask=mask if tile_cull else None, kept=kept)


def bin_tiles(cams, geom, tile=(16, 16)):
    """Sorted (key, value) pairs and per-tile ranges, by definition (library sort)."""
    L = _L()
    lay = layout(cams, tile)
    views = make_views(cams)
    K = int(geom["kept"].astype(np.int64).sum())
    keys = np.zeros(max(K, 1), np.uint64)
    vals = np.zeros(max(K, 1), np.uint32)
    ranges = np.zeros((lay["n_tiles"], 2), np.uint32)
    mask = geom.get("tile_mask")
    L.orc_bin(len(views), views, geom["n"], tile[0], tile[1], _p(geom["rect"]),
              None if mask is None else _p(mask), _p(geom["uvz"]), _p(lay["tile_base"]), lay["n_tiles"], _p(keys),
              _p(vals), _p(ranges))
    return dict(keys=keys[:K], vals=vals[:K], ranges=ranges, n_pairs=K, **lay)


def sh_eval(dirs, deg):
    dirs = _c(dirs, np.float64).reshape(-1, 3)
    K = (deg + 1) ** 2
    Y = np.zeros((dirs.shape[0], K), np.float64)
    _L().orc_sh_eval(_p(dirs), dirs.shape[0], deg, _p(Y))
    return Y


PROJ_COLS = ("u", "v", "z", "conicA", "conicB", "conicC", "opacity", "r", "g", "b",
             "cov_a", "cov_b", "cov_c", "clampx", "clampy", "valid")


def project64(params, cams, geom, blur=0.3):
    """FP64 2D quantities for every (view, Gaussian) that touches a tile; [V*n, 16]."""
    L = _L()
    means, ls, q, ol, sh = (_c(params[k], np.float64) for k in
                            ("means", "log_scales", "quats", "opacity_logit", "sh"))
    n = means.shape[0]
    views = make_views(cams)
    out = np.zeros((len(views) * n, 16), np.float64)
    L.orc_project64(len(views), views, n, _p(means), _p(ls), _p(q), _p(ol), _p(sh),
                    int(params["sh_degree"]), float(blur), _p(geom["radius"]), _p(out))
    return out


def render(cams, proj, drec, bins, n, tile=(16, 16), margin_alpha=0.0, margin_T=0.0):
    """FP64 compositing of RGB, depth and alpha (border mask) for all views,
    with the alpha decisions taken on the FP32 decision records drec.
    flags marks pixels whose stop decision lies within the transmittance band
    (FLAG_T_MIN); slack [P, 4] = (w, w * max colour, w * depth) of the entry at
    that decision, w its blend weight, and the relative band of the final T.  margin_alpha > 0 additionally flags
    FP64 alphas within that relative margin of a cut, and margin_T widens the
    band (test knobs for finite differences)."""
    L = _L()
    views = make_views(cams)
    P = bins["n_pix"]
    out = dict(rgb=np.zeros((P, 3)), depth=np.zeros(P), alpha=np.zeros(P), final_T=np.zeros(P),
               n_contrib=np.zeros(P, np.int32), flags=np.zeros(P, np.int32), slack=np.zeros((P, 4)))
    L.orc_render(len(views), views, n, _p(proj), _p(_c(drec, np.float32)), tile[0], tile[1],
                 _p(bins["tile_base"]), _p(bins["pix_base"]), _p(_c(bins["vals"], np.uint32)),
                 _p(bins["ranges"]), Margins(margin_alpha, margin_T), _p(out["rgb"]), _p(out["depth"]),
                 _p(out["alpha"]), _p(out["final_T"]), _p(out["n_contrib"]), _p(out["flags"]),
                 _p(out["slack"]))
    return out


def render_bwd(cams, proj, drec, bins, n, dC, dD, dA, tile=(16, 16)):
    """Per-(view, Gaussian) 2D gradients [V*n, 10] (u, v, conicA, conicB, conicC,
    opacity, r, g, b, z) for upstream image gradients."""
    L = _L()
    views = make_views(cams)
    g2d = np.zeros((len(views) * n, 10), np.float64)
    L.orc_render_bwd(len(views), views, n, _p(proj), _p(_c(drec, np.float32)), tile[0], tile[1],
                     _p(bins["tile_base"]),
                     _p(bins["pix_base"]), _p(_c(bins["vals"], np.uint32)), _p(bins["ranges"]),
                     _p(_c(dC, np.float64)), _p(_c(dD, np.float64)), _p(_c(dA, np.float64)),
                     _p(g2d))
    return g2d


def project_bwd(params, cams, geom, g2d, blur=0.3):
    """Parameter gradients summed over views, and per-view twist gradients [V, 6]."""
    L = _L()
    means, ls, q, ol, sh = (_c(params[k], np.float64) for k in
                            ("means", "log_scales", "quats", "opacity_logit", "sh"))
    n = means.shape[0]
    views = make_views(cams)
    g = dict(means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
             opacity_logit=np.zeros(n), sh=np.zeros(sh.shape, np.float64),
             twist=np.zeros((len(views), 6)))
    L.orc_project_bwd(len(views), views, n, _p(means), _p(ls), _p(q), _p(ol), _p(sh),
                      int(params["sh_degree"]), float(blur), _p(geom["radius"]),
                      _p(_c(g2d, np.float64)), _p(g["means"]), _p(g["log_scales"]),
                      _p(g["quats"]), _p(g["opacity_logit"]), _p(g["sh"]), _p(g["twist"]))
    return g


def loss_l1(img, t_rgb, t_depth, w_c=1.0, w_d=1.0, gate=False, gamma=0.99):
    """L1 colour + depth loss with the optional filter gate; returns (L, dC, dD)."""
    P = img["depth"].shape[0]
    dC = np.zeros((P, 3))
    dD = np.zeros(P)
    Lv = _L().orc_loss_l1(P, _p(_c(img["rgb"], np.float64)), _p(_c(img["depth"], np.float64)),
                          _p(_c(img["alpha"], np.float64)), _p(_c(t_rgb, np.float64)),
                          _p(_c(t_depth, np.float64)), float(w_c), float(w_d), int(gate),
                          float(gamma), _p(dC), _p(dD))
    return Lv, dC, dD


def reproj(points, obs, cams, weight=1.0, view_ids=None, near_z=0.2):
    """Re-projection loss (Eq. lba) and its twist gradient [V, 6]."""
    views = make_views(cams)
    pts = _c(points, np.float64)
    ob = _c(obs, np.float64)
    vid = None if view_ids is None else _c(view_ids, np.int32)
    g = np.zeros((len(views), 6))
    Lv = _L().orc_reproj(pts.shape[0], _p(pts), _p(ob), None if vid is None else _p(vid), views,
                         float(weight), float(near_z), _p(g))
    return Lv, g


def decode_keyframes(rgb8, depth16, depth_scale):
    """Sec. 4 keyframes (TUM RGB-D: 8-bit colour, 16-bit depth) to the FP32
    loss targets by their definition: colour c / 255 and depth d * scale, each
    one IEEE FP32 operation (numpy float32 arithmetic is correctly rounded)."""
    rgb = np.asarray(rgb8, np.uint8).astype(np.float32) / np.float32(255.0)
    depth = np.asarray(depth16, np.uint16).astype(np.float32) * np.float32(depth_scale)
    return rgb.astype(np.float32), depth.astype(np.float32)


def adam(param, grad, m, v, lr, b1=0.9, b2=0.999, eps=1e-15, t=1):
    """One FP64 Adam step in place on float64 arrays."""
    for a in (param, grad, m, v):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    _L().orc_adam(param.size, _p(param), _p(grad), _p(m), _p(v), float(lr), float(b1), float(b2),
                  float(eps), int(t))


def se3_exp_apply(xi, E):
    """Exp(xi) * E for xi = (rho, phi), E a 3x4 world->camera matrix (FP64)."""
    xi = _c(xi, np.float64).reshape(6)
    E = _c(E, np.float64).reshape(12)
    out = np.zeros(12)
    _L().orc_se3_exp_apply(_p(xi), _p(E), _p(out))
    return out.reshape(3, 4)


# --------------------------------------------------------------------------
# whole pipeline conveniences
# --------------------------------------------------------------------------

def forward(params, cams, near_z=0.2, blur=0.3, tile=(16, 16), tile_cull=True, **margins):
    geom = project_geom(params, cams, near_z, blur, tile, tile_cull)
    bins = bin_tiles(cams, geom, tile)
    proj = project64(params, cams, geom, blur)
    drec = geom["drec"]
    img = render(cams, proj, drec, bins, geom["n"], tile, **margins)
    return dict(geom=geom, bins=bins, proj=proj, drec=drec, img=img)


def backward(params, cams, fwd, dC, dD, dA=None, blur=0.3, tile=(16, 16)):
    n = fwd["geom"]["n"]
    if dA is None:
        dA = np.zeros_like(np.asarray(dD, np.float64))
    g2d = render_bwd(cams, fwd["proj"], fwd["drec"], fwd["bins"], n, dC, dD, dA, tile)
    grads = project_bwd(params, cams, fwd["geom"], g2d, blur)
    grads["g2d"] = g2d
    return grads
