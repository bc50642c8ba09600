"""One mapping / pose-refinement iteration over a batch of keyframes, built from
the C-ABI calls (Sec. 3.4 online mapping; Sec. 3.3 joint optimisation).

A step is: project (a1) -> bin + sort (a2-a4) -> composite (a5) -> mapping
loss L_m = (1 - zeta)(w4 L1(D) + w5 L1(C)) + zeta L_SSIM with the optional gate
(a6 and the SSIM term) -> backward of the compositing and projection, with
per-view twist gradients (a7, a8) -> keypoint re-projection term (a9) -> Adam on
all Gaussian parameters (a10).  Everything is enqueued on one stream without a host
synchronisation, so a step can be captured in a CUDA graph and replayed.
"""
from __future__ import annotations

import numpy as np
import torch

from . import (Rasterizer, gs_adam_step, gs_loss_l1, gs_loss_ssim, gs_reproj_loss_grad, gs_ssim_workspace_size)

PARAM_ORDER = ("means", "log_scales", "quats", "opacity_logit", "sh")
DEFAULT_LR = dict(means=1.6e-4, log_scales=5e-3, quats=1e-3, opacity_logit=5e-2, sh=2.5e-3)


def _seg_widths(n, sh_degree):
    K = (sh_degree + 1) ** 2
    return dict(means=3 * n, log_scales=3 * n, quats=4 * n, opacity_logit=n, sh=3 * K * n)


class FlatParams:
    """All Gaussian parameters in one float32 device buffer (segments 256-byte
    aligned), with tensor views for each kind, so the optimiser is one launch."""

    def __init__(self, scene, device):
        n = int(scene["means"].shape[0])
        deg = int(scene["sh_degree"])
        widths = _seg_widths(n, deg)
        self.offsets, off = {}, 0
        for k in PARAM_ORDER:
            self.offsets[k] = off
            off += (widths[k] + 63) // 64 * 64
        self.total = off
        self.n, self.sh_degree, self.widths = n, deg, widths
        self.buf = torch.zeros(self.total, dtype=torch.float32, device=device)
        host = np.zeros(self.total, np.float32)
        for k in PARAM_ORDER:
            host[self.offsets[k]:self.offsets[k] + widths[k]] = np.asarray(scene[k], np.float32).reshape(-1)
        self.buf.copy_(torch.from_numpy(host))

    def views(self, buf=None):
        b = self.buf if buf is None else buf
        K = (self.sh_degree + 1) ** 2
        shapes = dict(means=(self.n, 3), log_scales=(self.n, 3), quats=(self.n, 4), opacity_logit=(self.n,),
                      sh=(self.n, K, 3))
        out = {k: b[self.offsets[k]:self.offsets[k] + self.widths[k]].view(*shapes[k]) for k in PARAM_ORDER}
        out["sh_degree"] = self.sh_degree
        return out


class MappingStep:
    """Buffers and launches of one joint mapping / tracking iteration."""

    def __init__(self, scene, intr, size, viewmats, target_rgb, target_depth, w_c=1.0, w_d=0.5,
                 use_gate=False, gamma=0.99, keypoints=None, w_rpj=1.5, lrs=None, pair_capacity=None,
                 zeta=0.0, device="cuda", tile=(16, 16)):
        dev = torch.device(device)
        self.flat = FlatParams(scene, dev)
        self.params = self.flat.views()
        self.grad_buf = torch.zeros_like(self.flat.buf)
        self.grads = self.flat.views(self.grad_buf)
        self.m = torch.zeros_like(self.flat.buf)
        self.v = torch.zeros_like(self.flat.buf)
        self.step_count = torch.zeros(2, dtype=torch.int32, device=dev)
        lrs = dict(DEFAULT_LR, **(lrs or {}))
        self.groups = [(self.flat.offsets[k], self.flat.widths[k], lrs[k]) for k in PARAM_ORDER]
        self.rast = Rasterizer(self.flat.n, self.flat.sh_degree, intr, size, pair_capacity, dev, tile=tile)
        self.viewmats = torch.as_tensor(np.asarray(viewmats, np.float32).reshape(-1, 12), device=dev).contiguous()
        self.target_rgb = target_rgb
        self.target_depth = target_depth
        P = self.rast.n_pix
        self.d_rgb = torch.zeros(P, 3, device=dev)
        self.d_depth = torch.zeros(P, device=dev)
        # the loss and the twist gradients share one buffer, cleared by one fill a step
        self.acc = torch.zeros(4 + 6 * self.rast.V, device=dev)
        self.loss = self.acc[0:1]
        self.d_twist = self.acc[4:].view(self.rast.V, 6)
        self.w_c, self.w_d, self.use_gate, self.gamma = float(w_c), float(w_d), bool(use_gate), float(gamma)
        self.zeta = float(zeta)
        self.ssim_ws = (torch.empty(gs_ssim_workspace_size(P), dtype=torch.uint8, device=dev)
                        if self.zeta > 0 else None)
        self.keypoints = keypoints  # dict(points [n,3], obs [n,2], view_ids [n]) on the device
        self.w_rpj = float(w_rpj)
        self.optimise_params = True
        # the keypoint re-projection term needs only the poses and keypoints:
        # it runs on a second stream, beside the render (it is a small,
        # latency-bound launch)
        self.side = torch.cuda.Stream(device=dev) if dev.type == "cuda" else None

    def run(self, timers=None, stream=None, part=0):
        """Enqueue one iteration.  timers: optional dict stage -> list to which
        (start, end) CUDA events are appended.  part 1 enqueues the step up to
        the losses (the only launches that read the keyframe targets), part 2
        the rest; 0 both."""
        if part == 0:
            self.run(timers, stream, 1)
            self.run(timers, stream, 2)
            return

        def mark(name):
            if timers is None:
                return None
            e = torch.cuda.Event(enable_timing=True)
            e.record()
            return (name, e)

        def close(tok):
            if tok is None:
                return
            e = torch.cuda.Event(enable_timing=True)
            e.record()
            timers.setdefault(tok[0], []).append((tok[1], e))

        r = self.rast
        main = stream if stream is not None else torch.cuda.current_stream()
        from . import gs_bin_sort, gs_project, gs_render_fwd_l1
        side = self.keypoints is not None and self.side is not None
        if part == 2:
            self._run_backward(mark, close, stream, side)
            return
        tok = mark("zero")
        # grad_buf needs no clearing: the projection backward writes every entry
        self.acc.zero_()  # the loss and the twist gradients
        close(tok)
        if side:
            # after the accumulators are cleared; its atomic adds to the loss and
            # the twist gradients mix with the render's in any order
            self.side.wait_stream(main)
            with torch.cuda.stream(self.side):
                tok = mark("reproj")
                kp = self.keypoints
                gs_reproj_loss_grad(kp["points"], kp["obs"], kp.get("view_ids"), r.views, self.viewmats, self.w_rpj,
                                    self.loss, self.d_twist, r.near_z, self.side)
                close(tok)
        tok = mark("project")
        gs_project(self.params, r.views, self.viewmats, r.proj, r.near_z, r.blur, stream)
        close(tok)
        tok = mark("bin_sort")
        gs_bin_sort(r.proj, r.n, r.views, r.bins, r.workspace, stream)
        close(tok)
        # a5 + a6: the compositing evaluates the L1 terms as each pixel finishes
        tok = mark("render_fwd")
        k1 = 1.0 - self.zeta
        gs_render_fwd_l1(r.proj, r.n, r.bins, r.views, r.img, r.work_counter, self.target_rgb, self.target_depth,
                         k1 * self.w_c, k1 * self.w_d, self.use_gate, self.gamma, self.loss, self.d_rgb, self.d_depth,
                         stream)
        close(tok)
        if self.zeta > 0:
            tok = mark("ssim")
            gs_loss_ssim(r.img["rgb"], self.target_rgb, r.views, self.zeta, self.loss, self.d_rgb, self.ssim_ws,
                         r.bins["status"], stream)
            close(tok)
        if side:
            main.wait_stream(self.side)  # the re-projection has overlapped the render

    def _run_backward(self, mark, close, stream, side):
        """Part 2 of run(): the backward, the re-projection term (when it has no
        second stream) and the optimiser step."""
        from . import gs_project_bwd, gs_render_bwd_splats
        r = self.rast
        tok = mark("render_bwd")
        gs_render_bwd_splats(r.proj, r.n, r.bins, r.views, r.img, self.d_rgb, self.d_depth, None, r.grad2d,
                             r.work_counter, stream)
        close(tok)
        tok = mark("project_bwd")
        gs_project_bwd(self.params, r.views, self.viewmats, r.proj, r.grad2d, self.grads, self.d_twist, r.near_z,
                       r.blur, stream, overwrite_grads=True)
        close(tok)
        if self.keypoints is not None and not side:
            tok = mark("reproj")
            kp = self.keypoints
            gs_reproj_loss_grad(kp["points"], kp["obs"], kp.get("view_ids"), r.views, self.viewmats, self.w_rpj,
                                self.loss, self.d_twist, r.near_z, stream)
            close(tok)
        if self.optimise_params:
            tok = mark("adam")
            gs_adam_step(self.flat.buf, self.grad_buf, self.m, self.v, self.groups, self.step_count, stream=stream)
            close(tok)

    def reorder_spatially(self, stream=None):
        """Stores the Gaussians (parameters and Adam state) in the Morton order
        of their means, as a map grown by densification is stored; rendering
        results do not depend on the order.  Map maintenance, not part of a
        step."""
        from . import gs_compact_rows, gs_spatial_order, gs_spatial_order_workspace_size
        n = self.flat.n
        new_index = torch.empty(n, dtype=torch.int32, device=self.flat.buf.device)
        ws = torch.empty(gs_spatial_order_workspace_size(n), dtype=torch.uint8, device=self.flat.buf.device)
        gs_spatial_order(self.params["means"], new_index, ws, stream=stream)
        bufs = [self.flat.buf, self.m, self.v]
        news = [torch.empty_like(b) for b in bufs]
        pairs = []
        for b, nb in zip(bufs, news):
            src, dst = self.flat.views(b), self.flat.views(nb)
            pairs += [(src[k].reshape(n, -1), dst[k].reshape(n, -1)) for k in PARAM_ORDER]
        gs_compact_rows(new_index, pairs, stream=stream)
        self.flat.buf.copy_(news[0])
        self.m.copy_(news[1])
        self.v.copy_(news[2])

    def kernels_per_step(self):
        """Kernels of this library launched by one run() (memsets excluded)."""
        # bin: record count, scan, compaction, 4 depth passes, pair count, scan, emission, the tile-id
        # passes (8 bits each) and the ranges
        tile_passes = max(1, (max(self.rast.n_tiles - 1, 0).bit_length() + 7) // 8)
        k_bin = 3 + 4 + 3 + tile_passes + 1
        # project, bin, fwd (with the L1 loss), bwd, pbwd colour + geometry
        k = 1 + k_bin + 1 + 1 + 2
        k += 2 if self.zeta > 0 else 0
        k += 1 if self.keypoints is not None else 0
        k += 1 if self.optimise_params else 0
        return k


class TrackingStep:
    """Pose-only refinement of one or more views (Sec. 3.3 joint optimisation):
    L = w1 L_rpj + w2 L_c + w3 L_d with the filter gate G(p); the map is held
    fixed.  Each run() takes one Adam step on the twists xi (rho with lr_rho,
    phi with lr_phi) and folds them into the poses, E <- Exp(xi) E, on device."""

    def __init__(self, params, intr, size, viewmats, target_rgb, target_depth, keypoints=None, w_rpj=1.5,
                 w_c=0.5, w_d=1.0, gamma=0.99, lr_rho=5e-4, lr_phi=3e-4, pair_capacity=None, device="cuda",
                 tile=(16, 16)):
        dev = torch.device(device)
        self.params = params
        n = int(params["means"].shape[0])
        self.rast = Rasterizer(n, params["sh_degree"], intr, size, pair_capacity, dev, tile=tile)
        V = self.rast.V
        if V > GS_MAX_TRACK_VIEWS:
            raise ValueError(f"at most {GS_MAX_TRACK_VIEWS} views per tracking step")
        self.viewmats = torch.as_tensor(np.asarray(viewmats, np.float32).reshape(-1, 12), device=dev).contiguous()
        self.target_rgb, self.target_depth = target_rgb, target_depth
        self.keypoints = keypoints
        self.twist = torch.zeros(V * 6, device=dev)
        self.d_twist = torch.zeros(V * 6, device=dev)
        self.m = torch.zeros(V * 6, device=dev)
        self.v = torch.zeros(V * 6, device=dev)
        self.step_count = torch.zeros(2, dtype=torch.int32, device=dev)
        self.groups = []
        for k in range(V):
            self.groups += [(6 * k, 3, lr_rho), (6 * k + 3, 3, lr_phi)]
        P = self.rast.n_pix
        self.d_rgb = torch.zeros(P, 3, device=dev)
        self.d_depth = torch.zeros(P, device=dev)
        self.loss = torch.zeros(1, device=dev)
        self.w_rpj, self.w_c, self.w_d, self.gamma = float(w_rpj), float(w_c), float(w_d), float(gamma)

    def run(self, stream=None):
        from . import gs_pose_update, gs_render_bwd
        r = self.rast
        self.d_twist.zero_()
        self.loss.zero_()
        r.forward(self.params, self.viewmats, stream)
        gs_loss_l1(r.img["rgb"], r.img["depth"], r.img["alpha"], self.target_rgb, self.target_depth, self.w_c,
                   self.w_d, True, self.gamma, self.loss, self.d_rgb, self.d_depth, stream)
        gs_render_bwd(self.params, r.views, self.viewmats, r.proj, r.bins, r.img, self.d_rgb, self.d_depth, None,
                      r.grad2d, None, self.d_twist, r.work_counter, r.near_z, r.blur, stream)
        if self.keypoints is not None:
            kp = self.keypoints
            gs_reproj_loss_grad(kp["points"], kp["obs"], kp.get("view_ids"), r.views, self.viewmats, self.w_rpj,
                                self.loss, self.d_twist, r.near_z, stream)
        gs_adam_step(self.twist, self.d_twist, self.m, self.v, self.groups, self.step_count, stream=stream)
        gs_pose_update(self.viewmats, self.twist, stream)


GS_MAX_TRACK_VIEWS = 4
