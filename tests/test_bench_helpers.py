"""Host-side pieces of bench.py that decide what the JSON line reports: the
DRAM-traffic figure is taken from the committed ncu counters only while the
profiled kernel's sources, variant and workload are the ones captured; the
per-stage work model is complete and positive; the oracle pool's plan keeps a
sample near its time budget."""
import os
import shutil

import pytest

import bench
from paper_2405_19614_gb300.build import build

WORKLOAD = "batched-1M-sh3-8x1200x680"


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()


def test_traffic_is_reported_for_the_profiled_sources_only(tmp_path, monkeypatch):
    import json
    import paper_2405_19614_gb300 as gs
    root = tmp_path / "repo"
    shutil.copytree(os.path.join(bench.ROOT, "paper_2405_19614_gb300", "csrc"),
                    root / "paper_2405_19614_gb300" / "csrc")
    (root / "profiles").mkdir()
    _, variant, _, _ = gs.gs_get_render_variants()
    rec = dict(workload=WORKLOAD, tile=[32, 16], variant=variant, bytes_per_launch=123456,
               sources_sha256=bench.traffic_sources_sha256("render_bwd", str(root)))
    (root / "profiles" / "traffic.json").write_text(json.dumps({"render_bwd": rec}))
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.kernel_traffic("render_bwd", WORKLOAD, None) == 123456  # record matches the sources

    class R:
        tile = (32, 16)
    assert bench.kernel_traffic("render_bwd", WORKLOAD, R()) == 123456
    R.tile = (16, 16)
    assert bench.kernel_traffic("render_bwd", WORKLOAD, R()) is None  # another tile shape
    assert bench.kernel_traffic("render_bwd", "another-workload", None) is None
    assert bench.kernel_traffic("ssim", WORKLOAD, None) is None  # no capture for that stage
    # the backward source differs by one byte: nothing is reported
    src = root / "paper_2405_19614_gb300" / "csrc" / "render_bwd.cu"
    src.write_text(src.read_text() + "\n")
    assert bench.kernel_traffic("render_bwd", WORKLOAD, None) is None


def test_stage_work_covers_every_timed_stage():
    w = dict(N=1000, V=2, P=5000, T=40, K=9000, V_vis=1500, E=70000, B=20000, C=60000, sh_floats=48)
    works = bench.stage_work(w)
    for stage in ("project", "bin_sort", "render_fwd", "ssim", "render_bwd", "project_bwd", "adam"):
        kind, amount = works[stage]
        assert kind in ("hbm", "alu") and amount > 0, stage
    # Adam moves 28 bytes a parameter; the projection backward reads and writes each parameter once
    param_b = 4 * (11 + 48)
    assert works["adam"][1] == 28 * (param_b // 4) * 1000
    assert works["project_bwd"][1] == 2 * param_b * 1000 + 96 * 1500


def test_oracle_pool_plan_fits_the_budget():
    class Pool(bench.OraclePool):
        def __init__(self):  # no worker processes: only the planning arithmetic
            self.H, self.fixed, self.per_row = 680, 0.8, 0.01

    p = Pool()
    rows, per_core = p.plan(12.0)
    assert rows == 680 and per_core == 2  # a whole view is 7.6 s; two of them near 12 s
    rows, per_core = p.plan(3.0)
    assert rows % 16 == 0 and per_core == 1 and abs(p.fixed + rows * p.per_row - 3.0) < 0.2


def test_survey_bytes_follow_the_stated_model():
    import bench
    w = dict(N=10, V=2, P=100, T=300, K=40, V_vis=15, sh_floats=48)
    sb = bench.survey_bytes(w)
    # 300 tiles: 9 bits + 32 depth bits = 41 bits, 6 passes of 8 bits
    assert sb["a3"] == 8 * 40 + 6 * 24 * 40
    assert sb["a1"] == 12 * 10 * 2 + 272 * 15
    assert sb["a8"] == 276 * 15 + 4 * 59 * 10
    assert sb["a10"] == 7 * 4 * 59 * 10
    assert sum(sb.values()) == (240 + 4080) + (60 + 480) + (320 + 5760) + 320 + (1760 + 2800) + 1600 + \
        (1760 + 4800 + 600) + (4140 + 2360) + 16520 + 14400
