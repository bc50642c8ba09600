"""GB300 (sm_103a) differentiable Gaussian splatting for the mapping and pose
refinement hot path of TAMBRIDGE (arXiv 2405.19614).

The compute runs in libgs.so (hand-written CUDA behind the C ABI of
include/gs.h).  This package only marshals arguments: the ``gs_*`` functions
below have the names of the C entry points and take torch tensors that already
live on the GPU; ``Rasterizer`` owns the buffers of one configuration and
``rasterize`` is the autograd entry point.  PyTorch provides device memory and
streams only.
"""
from __future__ import annotations

import ctypes
import math

import torch

from . import _lib
from ._lib import (GS_MAX_ADAM_GROUPS, GS_MAX_VIEWS, GS_TILE, GsAdamGroup, GsBins, GsError, GsImage, GsOptions,
                   GsParamGrads, GsParams, GsProjected, GsView, check)

__all__ = ["gs_get_device_status", "gs_workspace_size", "gs_check_lookback_timeout", "gs_project", "gs_bin_sort", "gs_bin_sort_noalloc", "gs_render_fwd", "gs_render_fwd_l1", "gs_render_stats", "gs_set_render_variants",
           "gs_get_render_variants", "gs_loss_l1", "gs_loss_ssim", "gs_check_ssim_timeout", "gs_render_bwd", "gs_render_bwd_splats",
           "gs_project_bwd", "gs_decode_keyframes", "gs_reproj_loss_grad", "gs_adam_step", "gs_pose_update", "gs_densify",
           "gs_prune_select", "gs_compact_rows", "gs_spatial_order_workspace_size", "gs_spatial_order",
           "gs_select_views", "Rasterizer", "rasterize", "make_views", "variant_fits",
           "GsError", "lib"]


def lib():
    return _lib.load()


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise GsError("tensor must be on the GPU")
    if not t.is_contiguous():
        raise GsError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def make_views(intr, size, tile=None):
    """ctypes array of gs_view_t from intr [V,4] (fx, fy, cx, cy), size [V,2]
    and the tile shape (tile_w, tile_h) of every view (None: the default)."""
    intr = [[float(x) for x in row] for row in (intr.tolist() if hasattr(intr, "tolist") else intr)]
    size = [[int(x) for x in row] for row in (size.tolist() if hasattr(size, "tolist") else size)]
    tw, th = (0, 0) if tile is None else (int(tile[0]), int(tile[1]))
    V = len(intr)
    arr = (GsView * V)()
    for v in range(V):
        arr[v].fx, arr[v].fy, arr[v].cx, arr[v].cy = intr[v]
        arr[v].width, arr[v].height = size[v]
        arr[v].tile_w, arr[v].tile_h = tw, th
    return arr


def variant_fits(variant, tile):
    """Whether a compositing variant's band divides the tile (else the library
    uses the (2, 8) band with the variant's chunk size)."""
    base = variant % _lib.N_BAND_VARIANTS
    bw = _lib.VARIANT_BW[base]
    bh = _lib.VARIANT_PPT[base] * (32 // bw)
    return tile[0] % bw == 0 and tile[1] % bh == 0


def _params(p):
    return GsParams(_ptr(p["means"]), _ptr(p["log_scales"]), _ptr(p["quats"]), _ptr(p["opacity_logit"]),
                    _ptr(p["sh"]), int(p["means"].shape[0]), int(p["sh_degree"]))


def _grads(g):
    if g is None:
        return None
    return GsParamGrads(_ptr(g["means"]), _ptr(g["log_scales"]), _ptr(g["quats"]), _ptr(g["opacity_logit"]),
                        _ptr(g["sh"]))


def _gref(grads):
    return None if grads is None else ctypes.byref(_grads(grads))


# --------------------------------------------------------------------------
# one wrapper per C entry point
# --------------------------------------------------------------------------

def gs_get_device_status(status, stream=None):
    """Host value of a device uint32 error word after the stream's work (synchronises)."""
    out = ctypes.c_uint32()
    check(lib().gs_get_device_status(_ptr(status), ctypes.byref(out), _stream(stream)), "gs_get_device_status")
    return int(out.value)


def gs_workspace_size(op, n=0, n_views=0, pair_capacity=0, n_pixels=0):
    return int(lib().gs_workspace_size(int(op), int(n), int(n_views), int(pair_capacity), int(n_pixels)))


def gs_check_lookback_timeout(spin_limit, withhold_first_tile, status, workspace, stream=None):
    """One two-tile onesweep pass; with withhold_first_tile its look-back wait
    must expire and set the timeout bit of status (device uint32)."""
    check(lib().gs_check_lookback_timeout(int(spin_limit), int(bool(withhold_first_tile)), _ptr(status),
                                          _ptr(workspace), workspace.numel(), _stream(stream)),
          "gs_check_lookback_timeout")


def gs_project(params, views, viewmats, proj, near_z=0.2, blur=0.3, stream=None):
    opt = GsOptions(near_z, blur)
    pj = _proj(proj)
    check(lib().gs_project(ctypes.byref(_params(params)), views, _ptr(viewmats), len(views), ctypes.byref(opt),
                           ctypes.byref(pj), _stream(stream)), "gs_project")


def _proj(proj):
    return GsProjected(_ptr(proj["rec"]), _ptr(proj["rect"]), _ptr(proj["radii"]), _ptr(proj["tiles_touched"]),
                       _ptr(proj["tile_mask"]))


def _bins(bins):
    return GsBins(_ptr(bins["keys"]), _ptr(bins["vals"]), _ptr(bins["ranges"]), _ptr(bins["n_pairs"]),
                  _ptr(bins["status"]), int(bins["keys"].shape[0]))


def _img(img):
    return GsImage(_ptr(img["rgb"]), _ptr(img["depth"]), _ptr(img["alpha"]), _ptr(img["final_T"]),
                   _ptr(img["n_contrib"]))


def gs_bin_sort_workspace_size(n_records, capacity, n_tiles):
    return int(lib().gs_bin_sort_workspace_size(n_records, capacity, n_tiles))


def gs_bin_sort(proj, n, views, bins, workspace, stream=None):
    check(lib().gs_bin_sort(ctypes.byref(_proj(proj)), n, views, len(views), ctypes.byref(_bins(bins)),
                            _ptr(workspace), workspace.numel(), _stream(stream)), "gs_bin_sort")


def gs_bin_sort_noalloc(proj, n, views, bins, stream=None):
    """gs_bin_sort without a caller workspace: for callers that cannot
    allocate device memory (mid graph capture, fixed-rate loops, hosts that own
    all device memory).  Uses a fixed scratch array inside the library (about
    65 MiB); at most 2,097,152 records (views x Gaussians) and a pair capacity
    of at most 2,097,152.  Calls must not overlap on the GPU."""
    check(lib().gs_bin_sort_noalloc(ctypes.byref(_proj(proj)), n, views, len(views), ctypes.byref(_bins(bins)),
                                    _stream(stream)), "gs_bin_sort_noalloc")


def gs_render_fwd(proj, n, bins, views, img, work_counter, stream=None):
    check(lib().gs_render_fwd(ctypes.byref(_proj(proj)), n, ctypes.byref(_bins(bins)), views, len(views),
                              ctypes.byref(_img(img)), _ptr(work_counter), _stream(stream)), "gs_render_fwd")


def gs_render_fwd_l1(proj, n, bins, views, img, work_counter, target_rgb, target_depth, w_c, w_d, use_gate, gamma,
                     loss, d_rgb, d_depth, stream=None):
    """gs_render_fwd with gs_loss_l1 evaluated on each pixel as it finishes."""
    check(lib().gs_render_fwd_l1(ctypes.byref(_proj(proj)), n, ctypes.byref(_bins(bins)), views, len(views),
                                 ctypes.byref(_img(img)), _ptr(work_counter), _ptr(target_rgb), _ptr(target_depth),
                                 w_c, w_d, int(use_gate), gamma, _ptr(loss), _ptr(d_rgb), _ptr(d_depth),
                                 _stream(stream)), "gs_render_fwd_l1")


def gs_render_stats(proj, n, bins, views, n_eval, n_blend, work_counter, stream=None):
    check(lib().gs_render_stats(ctypes.byref(_proj(proj)), n, ctypes.byref(_bins(bins)), views, len(views),
                                _ptr(n_eval), _ptr(n_blend), _ptr(work_counter), _stream(stream)), "gs_render_stats")


def gs_set_render_variants(fwd, bwd):
    check(lib().gs_set_render_variants(int(fwd), int(bwd)), "gs_set_render_variants")


def gs_get_render_variants():
    """(fwd, bwd, n_fwd, n_bwd): variants in use and how many exist."""
    out = [ctypes.c_int32() for _ in range(4)]
    check(lib().gs_get_render_variants(*[ctypes.byref(o) for o in out]), "gs_get_render_variants")
    return tuple(o.value for o in out)


def gs_decode_keyframes(rgb8, depth16, depth_scale, rgb, depth, stream=None):
    """Sensor-format keyframes (uint8 [P,3] colour, 16-bit [P] depth, as
    uint16 or int16 storage) to the FP32 targets rgb [P,3] and depth [P]."""
    if rgb8.dtype != torch.uint8 or depth16.dtype not in (torch.int16, getattr(torch, "uint16", torch.int16)):
        raise GsError("rgb8 must be uint8 and depth16 16-bit")
    P = depth16.numel()
    if rgb8.numel() != 3 * P or rgb.numel() != 3 * P or depth.numel() != P:
        raise GsError("keyframe sizes disagree")
    check(lib().gs_decode_keyframes(_ptr(rgb8), _ptr(depth16), P, float(depth_scale), _ptr(rgb), _ptr(depth),
                                    _stream(stream)), "gs_decode_keyframes")


def gs_loss_l1(rgb, depth, alpha, target_rgb, target_depth, w_c, w_d, use_gate, gamma, loss, d_rgb, d_depth,
               stream=None):
    check(lib().gs_loss_l1(_ptr(rgb), _ptr(depth), _ptr(alpha), _ptr(target_rgb), _ptr(target_depth),
                           depth.numel(), w_c, w_d, int(use_gate), gamma, _ptr(loss), _ptr(d_rgb), _ptr(d_depth),
                           _stream(stream)), "gs_loss_l1")


def gs_ssim_workspace_size(n_pixels):
    return int(lib().gs_ssim_workspace_size(int(n_pixels)))


def gs_loss_ssim(rgb, target_rgb, views, weight, loss, d_rgb, workspace, status=None, stream=None):
    """Adds weight * (1 - mean SSIM) to loss and its gradient to d_rgb (+=);
    status: optional device error word (uint32) for a staged copy that timed out."""
    check(lib().gs_loss_ssim(_ptr(rgb), _ptr(target_rgb), views, len(views), float(weight), _ptr(loss), _ptr(d_rgb),
                             _ptr(workspace), workspace.numel(), _ptr(status) if status is not None else None,
                             _stream(stream)), "gs_loss_ssim")


def gs_check_ssim_timeout(rgb, target_rgb, views, loss, d_rgb, workspace, status, stream=None):
    """The SSIM pass with a staged copy whose barrier never completes (see
    include/gs.h): every block's bounded wait gives up and sets GS_ERR_TIMEOUT
    in status."""
    check(lib().gs_check_ssim_timeout(_ptr(rgb), _ptr(target_rgb), views, len(views), _ptr(loss), _ptr(d_rgb),
                                      _ptr(workspace), workspace.numel(), _ptr(status), _stream(stream)),
          "gs_check_ssim_timeout")


def gs_render_bwd_splats(proj, n, bins, views, img, d_rgb, d_depth, d_alpha, grad2d, work_counter, stream=None):
    check(lib().gs_render_bwd_splats(ctypes.byref(_proj(proj)), n, ctypes.byref(_bins(bins)), views, len(views),
                                     ctypes.byref(_img(img)), _ptr(d_rgb), _ptr(d_depth), _ptr(d_alpha),
                                     _ptr(grad2d), _ptr(work_counter), _stream(stream)), "gs_render_bwd_splats")


def gs_project_bwd(params, views, viewmats, proj, grad2d, grads, d_twist, near_z=0.2, blur=0.3, stream=None,
                   overwrite_grads=False):
    opt = GsOptions(near_z, blur, int(bool(overwrite_grads)))
    check(lib().gs_project_bwd(ctypes.byref(_params(params)), views, _ptr(viewmats), len(views), ctypes.byref(opt),
                               ctypes.byref(_proj(proj)), _ptr(grad2d), _gref(grads), _ptr(d_twist),
                               _stream(stream)), "gs_project_bwd")


def gs_render_bwd(params, views, viewmats, proj, bins, img, d_rgb, d_depth, d_alpha, grad2d, grads, d_twist,
                  work_counter, near_z=0.2, blur=0.3, stream=None, overwrite_grads=False):
    opt = GsOptions(near_z, blur, int(bool(overwrite_grads)))
    check(lib().gs_render_bwd(ctypes.byref(_params(params)), views, _ptr(viewmats), len(views), ctypes.byref(opt),
                              ctypes.byref(_proj(proj)), ctypes.byref(_bins(bins)), ctypes.byref(_img(img)),
                              _ptr(d_rgb), _ptr(d_depth), _ptr(d_alpha), _ptr(grad2d), _gref(grads),
                              _ptr(d_twist), _ptr(work_counter), _stream(stream)), "gs_render_bwd")


def gs_reproj_loss_grad(points, obs, view_ids, views, viewmats, weight, loss, d_twist, near_z=0.2, stream=None):
    check(lib().gs_reproj_loss_grad(_ptr(points), _ptr(obs), _ptr(view_ids), points.shape[0], views,
                                    _ptr(viewmats), len(views), weight, near_z, _ptr(loss), _ptr(d_twist),
                                    _stream(stream)), "gs_reproj_loss_grad")


def gs_adam_step(param, grad, m, v, groups, step, beta1=0.9, beta2=0.999, eps=1e-15, stream=None):
    """groups: list of (offset, count, lr)."""
    if not 1 <= len(groups) <= GS_MAX_ADAM_GROUPS:
        raise GsError("between 1 and 8 Adam groups")
    arr = (GsAdamGroup * len(groups))(*[GsAdamGroup(int(o), int(c), float(lr)) for o, c, lr in groups])
    check(lib().gs_adam_step(_ptr(param), _ptr(grad), _ptr(m), _ptr(v), arr, len(groups), beta1, beta2, eps,
                             _ptr(step), _stream(stream)), "gs_adam_step")


def gs_pose_update(viewmats, twist, stream=None):
    check(lib().gs_pose_update(_ptr(viewmats), _ptr(twist), viewmats.shape[0], _stream(stream)), "gs_pose_update")


def gs_select_workspace_size(n_items):
    return int(lib().gs_select_workspace_size(int(n_items)))


def gs_densify(alpha, target_rgb, target_depth, views, viewmats, threshold, opacity_logit, params, n_old, capacity,
               n_added, workspace, status=None, stream=None):
    """Appends one Gaussian per pixel with alpha < threshold and positive depth
    (Sec. 3.4 densification); params: dict of arrays with room for capacity rows."""
    pg = _grads(params)
    check(lib().gs_densify(_ptr(alpha), _ptr(target_rgb), _ptr(target_depth), views, _ptr(viewmats), len(views),
                           float(threshold), float(opacity_logit), ctypes.byref(pg), int(params["sh_degree"]),
                           int(n_old), int(capacity), _ptr(n_added), _ptr(status), _ptr(workspace),
                           workspace.numel(), _stream(stream)), "gs_densify")


def gs_prune_select(opacity_logit, tau, new_index, n_kept, workspace, stream=None):
    check(lib().gs_prune_select(_ptr(opacity_logit), opacity_logit.numel(), float(tau), _ptr(new_index),
                                _ptr(n_kept), _ptr(workspace), workspace.numel(), _stream(stream)),
          "gs_prune_select")


def gs_compact_rows(new_index, pairs, stream=None):
    """pairs: list of (src, dst) tensors with rows along dim 0."""
    arr = (_lib.GsRows * len(pairs))()
    for k, (src, dst) in enumerate(pairs):
        arr[k].src = _ptr(src)
        arr[k].dst = _ptr(dst)
        arr[k].row_floats = int(src.numel() // max(src.shape[0], 1))
    check(lib().gs_compact_rows(_ptr(new_index), new_index.numel(), arr, len(pairs), _stream(stream)),
          "gs_compact_rows")


def gs_spatial_order_workspace_size(n):
    return int(lib().gs_spatial_order_workspace_size(int(n)))


def gs_spatial_order(means, new_index, workspace, status=None, stream=None):
    """Rank of every Gaussian in the Morton order of its mean (int32 [n])."""
    check(lib().gs_spatial_order(_ptr(means), means.shape[0], _ptr(new_index), _ptr(workspace), workspace.numel(),
                                 _ptr(status), _stream(stream)), "gs_spatial_order")


def gs_select_views(matches, totals, alpha=0.75, beta=20):
    """Host: 0/1 selection of keyframes (Sec. 3.3 view point selection)."""
    n = len(matches)
    M = (ctypes.c_int32 * n)(*[int(x) for x in matches])
    T = (ctypes.c_int32 * n)(*[int(x) for x in totals])
    out = (ctypes.c_int32 * n)()
    check(lib().gs_select_views(M, T, n, float(alpha), int(beta), out), "gs_select_views")
    return [int(x) for x in out]


# --------------------------------------------------------------------------
# buffer owner for one configuration
# --------------------------------------------------------------------------

def _layout(size, tile=(GS_TILE, GS_TILE)):
    ntx = [(int(w) + tile[0] - 1) // tile[0] for w, _ in size]
    nty = [(int(h) + tile[1] - 1) // tile[1] for _, h in size]
    n_tiles = sum(a * b for a, b in zip(ntx, nty))
    n_pix = sum(int(w) * int(h) for w, h in size)
    return n_tiles, n_pix


class Rasterizer:
    """Device buffers and launches for n Gaussians rendered into a fixed set of
    views (sizes and intrinsics fixed; poses are device tensors and may change).
    ``forward`` leaves its outputs in the rasterizer's buffers until the next
    forward; ``generation`` counts the forwards run, so a caller holding an
    older result can tell that the buffers no longer hold it."""

    def __init__(self, n, sh_degree, intr, size, pair_capacity=None, device="cuda", near_z=0.2, blur=0.3,
                 tile=(GS_TILE, GS_TILE)):
        self.n, self.sh_degree = int(n), int(sh_degree)
        self.size = [(int(w), int(h)) for w, h in (size.tolist() if hasattr(size, "tolist") else size)]
        self.intr = [[float(x) for x in row] for row in (intr.tolist() if hasattr(intr, "tolist") else intr)]
        self.tile = (int(tile[0]), int(tile[1]))
        if self.tile[0] not in _lib.TILE_SIDES or self.tile[1] not in _lib.TILE_SIDES or \
                self.tile[0] * self.tile[1] > 2048:
            raise GsError(f"tile sides must be 8, 16, 32 or 64 with at most 2048 pixels, not {self.tile}")
        self.views = make_views(self.intr, self.size, self.tile)
        self.V = len(self.size)
        if not 1 <= self.V <= GS_MAX_VIEWS:
            raise GsError(f"between 1 and {GS_MAX_VIEWS} views")
        self.near_z, self.blur = float(near_z), float(blur)
        self.device = device
        self.n_tiles, self.n_pix = _layout(self.size, self.tile)
        if pair_capacity is None:
            pair_capacity = max(1 << 16, 8 * self.n * self.V)
        self.capacity = int(min(pair_capacity, (1 << 30) - 1))
        self.pair_capacity = pair_capacity
        d = torch.device(device)
        R = self.V * self.n
        i32, f32 = torch.int32, torch.float32
        self.proj = dict(rec=torch.empty(R * 12, dtype=f32, device=d), rect=torch.empty(R, 2, dtype=i32, device=d),
                         radii=torch.empty(R, dtype=i32, device=d), tiles_touched=torch.empty(R, dtype=i32, device=d),
                         tile_mask=torch.empty(R, dtype=torch.int64, device=d))
        self.bins = dict(keys=torch.empty(self.capacity, dtype=torch.int64, device=d),
                         vals=torch.empty(self.capacity, dtype=i32, device=d),
                         ranges=torch.zeros(self.n_tiles, 2, dtype=i32, device=d),
                         n_pairs=torch.zeros(1, dtype=i32, device=d), status=torch.zeros(1, dtype=i32, device=d))
        ws = gs_bin_sort_workspace_size(R, self.capacity, self.n_tiles)
        self.workspace = torch.empty(ws, dtype=torch.uint8, device=d)
        P = self.n_pix
        self.img = dict(rgb=torch.empty(P, 3, dtype=f32, device=d), depth=torch.empty(P, dtype=f32, device=d),
                        alpha=torch.empty(P, dtype=f32, device=d), final_T=torch.empty(P, dtype=f32, device=d),
                        n_contrib=torch.empty(P, dtype=i32, device=d))
        self.grad2d = torch.zeros(R * 12, dtype=f32, device=d)
        self.work_counter = torch.zeros(1, dtype=i32, device=d)
        self.generation = 0

    def forward(self, params, viewmats, stream=None):
        """Project, bin and composite; results in self.img (device, async)."""
        gs_project(params, self.views, viewmats, self.proj, self.near_z, self.blur, stream)
        gs_bin_sort(self.proj, self.n, self.views, self.bins, self.workspace, stream)
        gs_render_fwd(self.proj, self.n, self.bins, self.views, self.img, self.work_counter, stream)
        self.generation += 1
        return self.img

    def backward(self, params, viewmats, d_rgb, d_depth, d_alpha, grads, d_twist=None, stream=None,
                 overwrite_grads=False):
        """Accumulate parameter gradients (or write them, with
        overwrite_grads) and per-view twist gradients for upstream image
        gradients; self.grad2d is left zeroed."""
        gs_render_bwd(params, self.views, viewmats, self.proj, self.bins, self.img, d_rgb, d_depth, d_alpha,
                      self.grad2d, grads, d_twist, self.work_counter, self.near_z, self.blur, stream,
                      overwrite_grads)

    def status(self):
        """Host read of the asynchronous error word (synchronises)."""
        return int(self.bins["status"].item())

    def n_pairs(self):
        return int(self.bins["n_pairs"].item())


class _RasterizeFn(torch.autograd.Function):
    """Forward and backward of the compositing behind autograd.

    The outputs are copies, so a later forward on the same rasterizer cannot
    change tensors autograd still holds.  The backward needs this call's
    projected records, tile lists, final transmittance and last indices; if
    another forward has run on the rasterizer since (two renders in one joint
    loss), it runs this call's forward again first.  The forward is
    deterministic (fixed-order arithmetic, stable sorts), so the recomputed
    state is the one this call's outputs came from, bit for bit."""

    @staticmethod
    def forward(ctx, rast, sh_degree, viewmats, twist, means, log_scales, quats, opacity_logit, sh):
        params = dict(means=means, log_scales=log_scales, quats=quats, opacity_logit=opacity_logit, sh=sh,
                      sh_degree=sh_degree)
        img = rast.forward(params, viewmats)
        ctx.rast = rast
        ctx.generation = rast.generation
        ctx.sh_degree = sh_degree
        ctx.save_for_backward(viewmats, means, log_scales, quats, opacity_logit, sh)
        ctx.want_twist = twist is not None and twist.requires_grad
        return img["rgb"].clone(), img["depth"].clone(), img["alpha"].clone()

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_alpha):
        viewmats, means, log_scales, quats, opacity_logit, sh = ctx.saved_tensors
        params = dict(means=means, log_scales=log_scales, quats=quats, opacity_logit=opacity_logit, sh=sh,
                      sh_degree=ctx.sh_degree)
        rast = ctx.rast
        if rast.generation != ctx.generation:
            rast.forward(params, viewmats)
            ctx.generation = rast.generation
        grads = dict(means=torch.empty_like(means), log_scales=torch.empty_like(log_scales),
                     quats=torch.empty_like(quats), opacity_logit=torch.empty_like(opacity_logit),
                     sh=torch.empty_like(sh))
        d_twist = torch.zeros(viewmats.shape[0], 6, device=means.device) if ctx.want_twist else None
        c = lambda t: None if t is None else t.contiguous()
        rast.backward(params, viewmats, c(g_rgb), c(g_depth), c(g_alpha), grads, d_twist, overwrite_grads=True)
        return (None, None, None, d_twist, grads["means"], grads["log_scales"], grads["quats"],
                grads["opacity_logit"], grads["sh"])


def rasterize(rast, params, viewmats, twist=None):
    """Differentiable render: returns (rgb [P,3], depth [P], alpha [P]), new
    tensors owned by the caller.  Several calls on one rasterizer may share a
    graph before one backward.  twist: optional [V,6] leaf standing for the
    left perturbation Exp(xi) E of each pose at xi = 0 (its value is not read);
    its .grad receives dL/dxi."""
    return _RasterizeFn.apply(rast, int(params["sh_degree"]), viewmats, twist, params["means"],
                              params["log_scales"], params["quats"], params["opacity_logit"], params["sh"])
