"""Densification, pruning and view point selection on the GPU against the
oracle (Sec. 3.4 densification and pruning, Sec. 3.3 view point selection):
indices and counts bit-exact, values within FP32 rounding."""
import numpy as np
import pytest
import torch

import paper_2405_19614_gb300 as gs
import scenes
from gpu_util import t
from oracle import map_update as MU

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2405_19614_gb300.build import build
    build()


def _alloc(cap, deg):
    K = (deg + 1) ** 2
    z = lambda *s: torch.zeros(*s, device="cuda")
    return dict(means=z(cap, 3), log_scales=z(cap, 3), quats=z(cap, 4), opacity_logit=z(cap), sh=z(cap, K, 3),
                sh_degree=deg)


@pytest.mark.parametrize("capacity_extra", [100000, 500])
def test_densify_matches_oracle(capacity_extra):
    rng = np.random.default_rng(3)
    vms = np.stack([scenes.look_at((0.2 * k, -0.1, 0.0), (0.0, 0.2, 3.0)) for k in range(2)])
    cams = scenes.cams_from([[60, 60, 32, 24], [80, 75, 40.5, 30]], [[64, 48], [81, 61]], vms)
    P = 64 * 48 + 81 * 61
    alpha = rng.uniform(0, 1, P).astype(np.float32)
    depth = rng.uniform(0.5, 5.0, P).astype(np.float32)
    depth[rng.uniform(0, 1, P) < 0.1] = 0.0
    rgb = rng.uniform(0, 1, (P, 3)).astype(np.float32)
    idx, ref = MU.densify(alpha, rgb, depth, cams, 0.5, -1.0, 3)
    n_old = 37
    cap = n_old + min(capacity_extra, len(idx))
    params = _alloc(cap, 3)
    n_added = torch.zeros(1, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(gs.gs_select_workspace_size(P), dtype=torch.uint8, device="cuda")
    views = gs.make_views(cams["intr"], cams["size"])
    gs.gs_densify(t(alpha), t(rgb), t(depth), views, t(cams["viewmats"].reshape(-1, 12)), 0.5, -1.0, params,
                  n_old, cap, n_added, ws, status)
    torch.cuda.synchronize()
    m = cap - n_old
    assert int(n_added) == m
    assert (int(status) != 0) == (m < len(idx))
    for k in ("means", "log_scales", "quats", "opacity_logit", "sh"):
        got = params[k][n_old:cap].cpu().numpy()
        np.testing.assert_allclose(got, ref[k][:m], rtol=2e-6, atol=2e-6, err_msg=k)
    assert float(params["means"][:n_old].abs().max()) == 0.0


def test_prune_and_compact_match_oracle():
    rng = np.random.default_rng(4)
    n = 200_001
    logit = rng.normal(-4, 3, n).astype(np.float32)
    ref_index, ref_kept = MU.prune_select(logit, 0.005)
    new_index = torch.empty(n, dtype=torch.int32, device="cuda")
    n_kept = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(gs.gs_select_workspace_size(n), dtype=torch.uint8, device="cuda")
    gs.gs_prune_select(t(logit), 0.005, new_index, n_kept, ws)
    torch.cuda.synchronize()
    assert int(n_kept) == ref_kept
    np.testing.assert_array_equal(new_index.cpu().numpy(), ref_index)
    src = [t(rng.standard_normal((n, w)).astype(np.float32)) for w in (3, 4, 1, 48)]
    dst = [torch.zeros(ref_kept, s.shape[1], device="cuda") for s in src]
    gs.gs_compact_rows(new_index, list(zip(src, dst)))
    torch.cuda.synchronize()
    keep = ref_index >= 0
    for s_, d_ in zip(src, dst):
        np.testing.assert_array_equal(d_.cpu().numpy(), s_.cpu().numpy()[keep])


def test_view_selection_matches_oracle():
    rng = np.random.default_rng(5)
    M = rng.integers(0, 200, 500).tolist()
    T = rng.integers(1, 250, 500).tolist()
    assert gs.gs_select_views(M, T, 0.75, 20) == MU.select_views(M, T, 0.75, 20)


def _spread10(v):
    v = v.astype(np.uint32) & np.uint32(0x3FF)
    out = np.zeros_like(v)
    for b in range(10):
        out |= ((v >> np.uint32(b)) & np.uint32(1)) << np.uint32(3 * b)
    return out


def _morton_ranks(means):
    """Ranks by the Morton code of the FP32-quantised means (1024 cells per
    axis of the bounding box), ties in index order: the definition, in numpy
    float32 arithmetic (each operation correctly rounded, as on the GPU)."""
    m = np.asarray(means, np.float32)
    lo, hi = m.min(0), m.max(0)
    q = np.zeros(m.shape, np.uint32)
    for a in range(3):
        ext = np.float32(hi[a] - lo[a])
        if ext > 0:
            t = (m[:, a] - lo[a]).astype(np.float32) * (np.float32(1024.0) / ext)
            q[:, a] = np.where(t >= np.float32(1023.0), 1023, np.floor(t)).astype(np.uint32)
    code = _spread10(q[:, 0]) | (_spread10(q[:, 1]) << np.uint32(1)) | (_spread10(q[:, 2]) << np.uint32(2))
    order = np.argsort(code, kind="stable")
    rank = np.empty(len(m), np.int32)
    rank[order] = np.arange(len(m), dtype=np.int32)
    return rank


@pytest.mark.parametrize("n", [1, 37, 5000, 100003])
def test_spatial_order_is_the_morton_rank(n):
    sc = scenes.cube_scene(n, seed=11, sh_degree=0)
    means = sc["means"].copy()
    if n > 40:
        means[5] = means[6]  # equal codes keep index order
        means[:7, 2] = means[0, 2]
    new_index = torch.empty(n, dtype=torch.int32, device="cuda")
    ws = torch.empty(gs.gs_spatial_order_workspace_size(n), dtype=torch.uint8, device="cuda")
    gs.gs_spatial_order(t(means), new_index, ws)
    got = new_index.cpu().numpy()
    assert sorted(got.tolist()) == list(range(n))
    np.testing.assert_array_equal(got, _morton_ranks(means))


def test_spatial_order_leaves_the_render_unchanged():
    """Reordering the Gaussians changes no image (list order within a tile is
    by depth; only exactly equal depths could swap)."""
    from gpu_util import make_rast, params_on_device, viewmats_on_device
    c = scenes.config(2, 0.02)
    sc, cams = c["scene"], c["cams"]
    n = sc["means"].shape[0]
    rast = make_rast(sc, cams)
    vm = viewmats_on_device(cams)
    rast.forward(params_on_device(sc), vm)
    ref = {k: rast.img[k].clone() for k in ("rgb", "depth", "alpha")}
    new_index = torch.empty(n, dtype=torch.int32, device="cuda")
    ws = torch.empty(gs.gs_spatial_order_workspace_size(n), dtype=torch.uint8, device="cuda")
    gs.gs_spatial_order(t(sc["means"]), new_index, ws)
    perm = new_index.cpu().numpy()
    assert not np.array_equal(perm, np.arange(n))
    sc2 = dict(sc)
    for k in ("means", "log_scales", "quats", "opacity_logit", "sh"):
        a = np.empty_like(sc[k])
        a[perm] = sc[k]
        sc2[k] = a
    rast.forward(params_on_device(sc2), vm)
    torch.cuda.synchronize()
    for k in ref:
        np.testing.assert_allclose(rast.img[k].cpu().numpy(), ref[k].cpu().numpy(), atol=1e-6, err_msg=k)
