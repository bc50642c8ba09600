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
