"""Autotuner of the tile shape and the compositing kernels (Sec. 3.4
"Differentiable Rasterization" bins Gaussians per screen tile and composites
each tile's list; the shapes are this library's choices).

Two levels, both timed with CUDA events on the caller's own workload:

* ``tune``: for a rasterizer (a fixed tile shape), the forward and backward
  compositing variants whose bands divide the tile: pixels per thread and
  band width ((1, 8) (2, 8) (2, 16) (4, 8) (4, 16) (8, 16)), each with its
  ways of staging a chunk of list entries in shared memory (lane loads of 32
  entries, asynchronous copies of 32, gathers by the tensor memory
  accelerator of 32 or 64).  Every variant computes the
  same result (the forward bit for bit, the backward up to the order of
  floating-point additions).
* ``tune_tiles``: the tile shape.  For each candidate the rasterizer is
  rebuilt, its variants tuned, and projection + binning + both compositing
  passes timed: the shape changes the pair count and sort as well as the
  walks.

Results of ``tune`` are cached per GPU model and workload shape, in memory and
in a JSON file next to the library (not part of the sources).
"""
from __future__ import annotations

import json
import os

import torch

from . import (Rasterizer, gs_bin_sort, gs_get_render_variants, gs_project, gs_render_bwd_splats, gs_render_fwd,
               gs_set_render_variants, variant_fits)

CACHE_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_cache.json")
TILE_CANDIDATES = ((8, 8), (16, 8), (16, 16), (32, 16), (32, 32), (64, 32))
_memory = {}


def _key(rast):
    name = torch.cuda.get_device_name()
    return f"{name}|n={rast.n}|deg={rast.sh_degree}|views={rast.size}|tile={rast.tile}"


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
    workload among those that fit its tile.  Runs a forward first; leaves
    rast.grad2d zeroed.  Returns dict(fwd=, bwd=, fwd_ms={variant: ms},
    bwd_ms={variant: ms})."""
    key = _key(rast)
    if use_cache:
        hit = _memory.get(key) or _load().get(key)
        if hit:
            gs_set_render_variants(hit["fwd"], hit["bwd"])
            _memory[key] = hit
            return hit
    _, cur_bwd, n_fwd, n_bwd = gs_get_render_variants()
    rast.forward(params, viewmats)
    fwd_ms = {}
    for fv in range(n_fwd):
        if not variant_fits(fv, rast.tile):
            continue
        gs_set_render_variants(fv, cur_bwd)
        fwd_ms[fv] = _time(lambda: gs_render_fwd(rast.proj, rast.n, rast.bins, rast.views, rast.img,
                                                 rast.work_counter), reps)
    best_f = min(fwd_ms, key=fwd_ms.get)
    gs_set_render_variants(best_f, cur_bwd)
    gs_render_fwd(rast.proj, rast.n, rast.bins, rast.views, rast.img, rast.work_counter)
    bwd_ms = {}
    for bv in range(n_bwd):
        if not variant_fits(bv, rast.tile):
            continue
        gs_set_render_variants(best_f, bv)
        bwd_ms[bv] = _time(lambda: gs_render_bwd_splats(rast.proj, rast.n, rast.bins, rast.views, rast.img, d_rgb,
                                                        d_depth, d_alpha, rast.grad2d, rast.work_counter), reps)
    best_b = min(bwd_ms, key=bwd_ms.get)
    gs_set_render_variants(best_f, best_b)
    rast.grad2d.zero_()
    torch.cuda.synchronize()
    res = dict(fwd=best_f, bwd=best_b, fwd_ms={str(k): v for k, v in fwd_ms.items()},
               bwd_ms={str(k): v for k, v in bwd_ms.items()})
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


def tune_tiles(rast, params, viewmats, d_rgb, d_depth, candidates=TILE_CANDIDATES, reps=3):
    """Pick the tile shape for rast's configuration: for each candidate a
    rasterizer of that shape is built, its variants tuned and projection +
    binning + forward + backward compositing timed.  Returns (rasterizer of
    the best shape, dict(tile=, fwd=, bwd=, ms={tile: total ms})) with the
    best shape's variants selected in the library."""
    results = {}
    best = None
    for tile in candidates:
        r = rast if tuple(tile) == tuple(rast.tile) else Rasterizer(
            rast.n, rast.sh_degree, rast.intr, rast.size, rast.pair_capacity, rast.device, rast.near_z, rast.blur,
            tile=tile)
        t = tune(r, params, viewmats, d_rgb, d_depth, reps=reps, use_cache=False)
        binning = _time(lambda: (gs_project(params, r.views, viewmats, r.proj, r.near_z, r.blur),
                                 gs_bin_sort(r.proj, r.n, r.views, r.bins, r.workspace)), reps)
        if r.status() != 0:  # this shape overflows the pair capacity
            continue
        total = binning + t["fwd_ms"][str(t["fwd"])] + t["bwd_ms"][str(t["bwd"])]
        results[f"{tile[0]}x{tile[1]}"] = dict(total_ms=total, binning_ms=binning, fwd=t["fwd"], bwd=t["bwd"],
                                               fwd_ms=t["fwd_ms"], bwd_ms=t["bwd_ms"])
        if best is None or total < best[0]:
            best = (total, r, t)
        elif r is not rast:
            del r
    total, r, t = best
    gs_set_render_variants(t["fwd"], t["bwd"])
    r.forward(params, viewmats)
    torch.cuda.synchronize()
    return r, dict(tile=list(r.tile), fwd=t["fwd"], bwd=t["bwd"], candidates=results)
