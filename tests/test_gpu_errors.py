"""The asynchronous error path of the C ABI: a bounded wait that runs out
sets its bit in the device status word, the kernel returns, and the context
stays usable (no fault, no hang).

The wait made to run out is the decoupled look-back of a onesweep radix pass:
gs_check_lookback_timeout starts the pass's tile counter past tile 0, so
nothing ever publishes tile 0 and tile 1's look-back gives up after a short
spin limit.  The same pass with tile 0 processed must sort correctly and
leave the status word at zero.

The second is the barrier wait of the SSIM gradient pass's staged copies:
gs_check_ssim_timeout makes the barrier expect 16 bytes more than the copy
delivers (the copy itself completes, nothing is left in flight), so every
block's wait gives up, sets the bit and returns without touching d_rgb."""
import numpy as np
import pytest
import torch

import paper_2405_19614_gb300 as gs
from gpu_util import make_rast, params_on_device, viewmats_on_device
from paper_2405_19614_gb300._lib import ERR_TIMEOUT, GS_OP_CHECK_LOOKBACK

import scenes

pytestmark = pytest.mark.gpu

N_KEYS = 8192


def _workspace():
    ws = gs.gs_workspace_size(GS_OP_CHECK_LOOKBACK)
    assert ws == int(gs.lib().gs_check_lookback_timeout_workspace_size()) and ws >= 16 * N_KEYS
    return torch.zeros(ws, dtype=torch.uint8, device="cuda")


def _check_sorted(ws):
    out = ws[:8 * N_KEYS].cpu().numpy().view(np.uint32)
    keys, vals = out[:N_KEYS], out[N_KEYS:]
    idx = np.arange(N_KEYS, dtype=np.uint64)
    src = ((idx * 2654435761) % (1 << 32)).astype(np.uint32)
    # stable sort by the low byte, by its definition
    order = np.argsort(src & 0xFF, kind="stable")
    np.testing.assert_array_equal(vals, order.astype(np.uint32))
    np.testing.assert_array_equal(keys, src[order])


def test_lookback_pass_sorts_and_leaves_status_clear():
    ws = _workspace()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    gs.gs_check_lookback_timeout(0, False, status, ws)
    assert gs.gs_get_device_status(status) == 0
    _check_sorted(ws)


def test_expired_lookback_wait_sets_timeout_and_returns():
    ws = _workspace()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    gs.gs_check_lookback_timeout(1000, True, status, ws)
    st = gs.gs_get_device_status(status)
    assert st == (1 << ERR_TIMEOUT), st
    # the context is still usable: the normal pass runs and sorts after it
    status2 = torch.zeros(1, dtype=torch.int32, device="cuda")
    gs.gs_check_lookback_timeout(0, False, status2, ws)
    torch.cuda.synchronize()
    assert gs.gs_get_device_status(status2) == 0
    _check_sorted(ws)


def test_timeout_reaches_the_binning_status_word():
    """The bit lands in a gs_bins_t status word like the binning's own errors,
    and a following render of the same rasterizer still runs."""
    c = scenes.config(1, scale=0.25)
    rast = make_rast(c["scene"], c["cams"])
    ws = _workspace()
    gs.gs_check_lookback_timeout(500, True, rast.bins["status"], ws)
    assert rast.status() == (1 << ERR_TIMEOUT)
    rast.bins["status"].zero_()
    rast.forward(params_on_device(c["scene"]), viewmats_on_device(c["cams"]))
    torch.cuda.synchronize()
    assert rast.status() == 0


def test_expired_ssim_copy_wait_sets_timeout_and_returns():
    from oracle import ssim as S
    rng = np.random.default_rng(3)
    size = np.array([[64, 48], [40, 20]])  # widths a multiple of 4: the staged pass runs
    P = int((size[:, 0] * size[:, 1]).sum())
    x = rng.uniform(0, 1, (P, 3)).astype(np.float32)
    y = np.clip(x + rng.normal(0, 0.15, x.shape), 0, 1).astype(np.float32)
    views = gs.make_views([[50, 50, 20, 20]] * len(size), size)
    ws = torch.empty(gs.gs_ssim_workspace_size(P), dtype=torch.uint8, device="cuda")
    xt, yt = torch.as_tensor(x, device="cuda"), torch.as_tensor(y, device="cuda")
    base = torch.as_tensor(rng.normal(0, 1e-5, (P, 3)).astype(np.float32), device="cuda")
    d_rgb = base.clone()
    loss = torch.zeros(1, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    gs.gs_check_ssim_timeout(xt, yt, views, loss, d_rgb, ws, status)
    st = gs.gs_get_device_status(status)
    assert st == (1 << ERR_TIMEOUT), st
    assert torch.equal(d_rgb, base)  # the blocks returned before their writes
    # the context is still usable: the normal pass runs after it and matches the oracle
    L, g = S.loss_ssim(x.astype(np.float64), y.astype(np.float64), size, weight=0.3)
    loss2 = torch.zeros(1, device="cuda")
    status2 = torch.zeros(1, dtype=torch.int32, device="cuda")
    gs.gs_loss_ssim(xt, yt, views, 0.3, loss2, d_rgb, ws, status2)
    torch.cuda.synchronize()
    assert gs.gs_get_device_status(status2) == 0
    got = (d_rgb - base).cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - g) <= 1e-3 * np.linalg.norm(g)
    assert abs(float(loss2) - L) <= 2e-6 * max(1.0, L)
