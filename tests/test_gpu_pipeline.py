"""The mapping step as a whole (rows a1-a10 with the SSIM term and the
keypoint re-projection term on its second stream): replaying it as a CUDA
graph, or as the two captured parts the end-to-end loop uses, gives the same
parameters and losses as launching it eagerly, and the loss falls over a few
iterations."""
import os
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2405_19614_gb300.build import build
    build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def _state(step):
    return [t.clone() for t in (step.flat.buf, step.m, step.v, step.step_count)]


def _restore(step, state):
    for t, s in zip((step.flat.buf, step.m, step.v, step.step_count), state):
        t.copy_(s)


def _capture(step, **kw):
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step.run(**kw)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        step.run(**kw)
    return g


def test_graph_replay_and_parts_equal_eager_steps():
    import bench
    c, step, cap = bench.build_workload(4, 0.02, torch.device("cuda", 0))
    assert step.keypoints is not None and step.zeta > 0
    s0 = _state(step)
    iters = 4

    def run_eager():
        out = []
        for _ in range(iters):
            step.run()
            out.append(float(step.loss))
        return out, step.flat.buf.clone()

    loss_e, p_e = run_eager()
    assert step.rast.status() == 0
    assert loss_e[-1] < loss_e[0]  # Adam on the joint loss makes progress

    _restore(step, s0)
    g = _capture(step)
    _restore(step, s0)  # the capture's warm-up run stepped the parameters
    loss_g = []
    for _ in range(iters):
        g.replay()
        loss_g.append(float(step.loss))
    p_g = step.flat.buf.clone()

    _restore(step, s0)
    g1, g2 = _capture(step, part=1), _capture(step, part=2)
    _restore(step, s0)
    loss_p = []
    for _ in range(iters):
        g1.replay()
        g2.replay()
        loss_p.append(float(step.loss))
    p_p = step.flat.buf.clone()

    # the compositing backward adds with atomics, so runs agree to rounding
    for other, p in ((loss_g, p_g), (loss_p, p_p)):
        for a, b in zip(other, loss_e):
            assert abs(a - b) <= 1e-4 * abs(b)
        rel = float((p - p_e).norm() / p_e.norm())
        assert rel < 1e-4, rel
    assert int(step.step_count[0]) == int(s0[3][0]) + iters
