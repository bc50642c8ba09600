"""The asynchronous error path of the C ABI: a bounded wait that runs out
sets its bit in the device status word, the kernel returns, and the context
stays usable (no fault, no hang).

The wait made to run out is the decoupled look-back of a onesweep radix pass:
gs_check_lookback_timeout starts the pass's tile counter past tile 0, so
nothing ever publishes tile 0 and tile 1's look-back gives up after a short
spin limit.  The same pass with tile 0 processed must sort correctly and
leave the status word at zero."""
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
