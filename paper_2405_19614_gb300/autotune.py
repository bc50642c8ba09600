"""Autotuner for the compositing kernels (a5, a7): pixels per thread (1, 2, 4
or 8; a warp's band of a tile is 16 x 2 * that many rows).

Every variant computes the same result (the forward bit for bit, the backward
up to the order of floating-point additions); this times each one on the
caller's own workload with CUDA events and leaves the fastest selected in the
library.  Results are cached per GPU model and workload shape, in memory and
in a JSON file next to the library (not part of the sources).
"""
from __future__ import annotations

import json
import os

import torch

from . import (gs_get_render_variants, gs_render_bwd_splats, gs_render_fwd, gs_set_render_variants)

CACHE_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_cache.json")
_memory = {}


def _key(rast):
    name = torch.cuda.get_device_name()
    return f"{name}|n={rast.n}|deg={rast.sh_degree}|views={rast.size}"


def _load():
    try:
        with open(CACHE_PATH) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _time(fn, reps):
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune(rast, params, viewmats, d_rgb, d_depth, d_alpha=None, reps=3, use_cache=True):
    """Pick the fastest forward and backward variants for this rasterizer's
    workload.  Runs a forward first; leaves rast.grad2d zeroed.  Returns
    dict(fwd=, bwd=, fwd_ms=[...], bwd_ms=[...])."""
    key = _key(rast)
    if use_cache:
        hit = _memory.get(key) or _load().get(key)
        if hit:
            gs_set_render_variants(hit["fwd"], hit["bwd"])
            _memory[key] = hit
            return hit
    _, cur_bwd, n_fwd, n_bwd = gs_get_render_variants()
    rast.forward(params, viewmats)
    fwd_ms = []
    for fv in range(n_fwd):
        gs_set_render_variants(fv, cur_bwd)
        fwd_ms.append(_time(lambda: gs_render_fwd(rast.proj, rast.n, rast.bins, rast.views, rast.img,
                                                  rast.work_counter), reps))
    best_f = min(range(n_fwd), key=lambda i: fwd_ms[i])
    gs_set_render_variants(best_f, cur_bwd)
    gs_render_fwd(rast.proj, rast.n, rast.bins, rast.views, rast.img, rast.work_counter)
    bwd_ms = []
    for bv in range(n_bwd):
        gs_set_render_variants(best_f, bv)
        bwd_ms.append(_time(lambda: gs_render_bwd_splats(rast.proj, rast.n, rast.bins, rast.views, rast.img, d_rgb,
                                                         d_depth, d_alpha, rast.grad2d, rast.work_counter), reps))
    best_b = min(range(n_bwd), key=lambda i: bwd_ms[i])
    gs_set_render_variants(best_f, best_b)
    rast.grad2d.zero_()
    torch.cuda.synchronize()
    res = dict(fwd=best_f, bwd=best_b, fwd_ms=fwd_ms, bwd_ms=bwd_ms)
    _memory[key] = res
    if use_cache:
        data = _load()
        data[key] = res
        try:
            tmp = CACHE_PATH + f".tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(data, f, indent=1)
            os.replace(tmp, CACHE_PATH)
        except OSError:
            pass
    return res
