"""The allocation-free binning entry point, for callers that cannot allocate
device memory (for example in the middle of a CUDA graph capture, or in a
fixed-rate tracking loop that cannot take an allocation's synchronisation).

gs_bin_sort_noalloc must produce exactly what gs_bin_sort produces with a
caller-owned workspace (keys, values and ranges are integers: bit-exact), on two
calls in a row with different inputs (its static scratch keeps the previous
call's contents), must accept a call exactly at both of its limits
(2,097,152 records and 2,097,152 pairs of capacity) and must refuse a call one
past either."""
import numpy as np
import pytest
import torch

import paper_2405_19614_gb300 as gs
import scenes
from gpu_util import params_on_device, viewmats_on_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2405_19614_gb300.build import build
    build()


def _bins_like(rast):
    b = rast.bins
    return {k: torch.zeros_like(v) for k, v in b.items()}


MAX_RECORDS = 1 << 21
MAX_PAIRS = 1 << 21


def _compare(scene, cams, capacity=1 << 18):
    rast = gs.Rasterizer(scene["means"].shape[0], scene["sh_degree"], cams["intr"], cams["size"],
                         pair_capacity=capacity)
    p = params_on_device(scene)
    vm = viewmats_on_device(cams)
    gs.gs_project(p, rast.views, vm, rast.proj)
    gs.gs_bin_sort(rast.proj, rast.n, rast.views, rast.bins, rast.workspace)
    other = _bins_like(rast)
    gs.gs_bin_sort_noalloc(rast.proj, rast.n, rast.views, other)
    torch.cuda.synchronize()
    K = int(rast.bins["n_pairs"].item())
    assert K > 0 and int(other["n_pairs"].item()) == K
    assert int(other["status"].item()) == 0
    for k in ("keys", "vals"):
        np.testing.assert_array_equal(other[k][:K].cpu().numpy(), rast.bins[k][:K].cpu().numpy())
    np.testing.assert_array_equal(other["ranges"].cpu().numpy(), rast.bins["ranges"].cpu().numpy())


def test_noalloc_matches_workspace_path_twice_in_a_row():
    c = scenes.config(1)
    _compare(c["scene"], c["cams"])
    sc = scenes.cube_scene(5000, seed=321, sh_degree=3, log_scale=(-3.0, 0.5))
    vms = np.stack([scenes.look_at((0.2 * k, -0.1, -0.3), (0.0, 0.0, 3.0)) for k in range(2)])
    cams = scenes.cams_from([[80, 80, 60, 40], [70, 70, 50, 33]], [[120, 80], [97, 61]], vms)
    _compare(sc, cams)


def test_noalloc_exactly_at_both_limits():
    # every (view, Gaussian) record counts toward the limit, drawn or not:
    # all but 20,000 Gaussians sit behind the camera, so the pairs stay few
    sc = scenes.cube_scene(MAX_RECORDS, seed=77, sh_degree=0, log_scale=(-3.5, 0.3))
    sc["means"][20000:, 2] = -5.0
    _compare(sc, scenes.pinhole(320, 240, 300.0), capacity=MAX_PAIRS)


def test_noalloc_rejects_sizes_beyond_its_limits():
    c = scenes.config(1)
    cams = c["cams"]
    views = gs.make_views(cams["intr"], cams["size"])
    big = MAX_RECORDS + 1  # one record past the limit; nothing is enqueued
    proj = dict(rec=torch.zeros(16, device="cuda"), rect=torch.zeros(4, 2, dtype=torch.int32, device="cuda"),
                radii=torch.zeros(4, dtype=torch.int32, device="cuda"),
                tiles_touched=torch.zeros(4, dtype=torch.int32, device="cuda"),
                tile_mask=torch.zeros(4, dtype=torch.int64, device="cuda"))
    bins = dict(keys=torch.zeros(4, dtype=torch.int64, device="cuda"),
                vals=torch.zeros(4, dtype=torch.int32, device="cuda"),
                ranges=torch.zeros(12, 2, dtype=torch.int32, device="cuda"),
                n_pairs=torch.zeros(1, dtype=torch.int32, device="cuda"),
                status=torch.zeros(1, dtype=torch.int32, device="cuda"))
    with pytest.raises(gs.GsError, match="CAPACITY"):
        gs.gs_bin_sort_noalloc(proj, big, views, bins)
    bins["keys"] = torch.zeros(MAX_PAIRS + 1, dtype=torch.int64, device="cuda")
    with pytest.raises(gs.GsError, match="CAPACITY"):
        gs.gs_bin_sort_noalloc(proj, 4, views, bins)
