"""The paper's hyper-parameter table (appendix A), stored in
tests/golden/hyperparameters.txt, against the defaults of the oracle and the
library and the loss settings of the workloads, with worked cases of the
selection rules at those values (Sec. 3.3 view point selection, Sec. 3.4
pruning).  CPU only: the view selection runs on the host side of the C ABI."""
import inspect
import math
import os

import numpy as np
import pytest

import paper_2405_19614_gb300 as gs
import scenes
from oracle import map_update as MU
from paper_2405_19614_gb300 import _lib
from paper_2405_19614_gb300.build import build
from paper_2405_19614_gb300.pipeline import MappingStep

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "hyperparameters.txt")


def _table():
    out = {}
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if line:
            name, value = line.split()
            out[name] = float(value)
    return out


H = _table()


def _defaults(fn):
    return {k: p.default for k, p in inspect.signature(fn).parameters.items() if p.default is not p.empty}


def test_table_is_complete():
    assert sorted(H) == sorted(["alpha", "beta", "gamma", "zeta", "tau", "w1", "w2", "w3", "w4", "w5"])


def test_library_and_oracle_defaults_are_the_papers():
    for fn in (MU.select_views, gs.gs_select_views):
        d = _defaults(fn)
        assert d["alpha"] == H["alpha"] and d["beta"] == H["beta"], fn
    d = _defaults(MappingStep.__init__)
    assert d["gamma"] == H["gamma"]
    assert d["w_rpj"] == H["w1"]


def test_workload_loss_settings_are_the_papers():
    # the tracking workload optimises the joint loss of the Fusion Bridge,
    # the batched mapping workloads the mapping loss
    t = scenes.config(3, scale=1e-4)
    assert (t["w_rpj"], t["w_c"], t["w_d"], t["gamma"]) == (H["w1"], H["w2"], H["w3"], H["gamma"])
    assert t["gate"]
    for idx in (4, 5):
        m = scenes.config(idx, scale=1e-5)
        assert (m["w_c"], m["w_d"], m["zeta"]) == (H["w5"], H["w4"], H["zeta"])


# Worked cases of R_i = 1 iff beta <= M < alpha T at alpha = 0.75, beta = 20
# (the first keyframe is always taken): the two ends of the interval and their
# neighbours.
VIEW_CASES = [
    # (M, T, R)
    (20, 100, 1),   # M = beta: the lower end is closed
    (19, 100, 0),   # below beta
    (74, 100, 1),   # just below alpha T = 75
    (75, 100, 0),   # M = alpha T: the upper end is open
    (20, 26, 0),    # alpha T = 19.5 < beta: empty interval
    (20, 27, 1),    # alpha T = 20.25
    (0, 0, 0),      # no matches at all
]


@pytest.fixture(scope="module")
def lib():
    build()
    return _lib.load()


def test_view_selection_worked_cases(lib):
    M = [0] + [m for m, _, _ in VIEW_CASES]
    T = [0] + [t for _, t, _ in VIEW_CASES]
    want = [1] + [r for _, _, r in VIEW_CASES]
    assert MU.select_views(M, T, H["alpha"], int(H["beta"])) == want
    assert gs.gs_select_views(M, T, H["alpha"], int(H["beta"])) == want


def test_pruning_at_the_papers_threshold():
    tau = H["tau"]
    op = np.array([1e-9, 0.001, 0.0049, 0.0051, 0.01, 0.5, 0.99], np.float64)
    logit = np.log(op / (1.0 - op)).astype(np.float32)
    new_index, n_kept = MU.prune_select(logit, tau)
    np.testing.assert_array_equal(new_index, [-1, -1, -1, 0, 1, 2, 3])
    assert n_kept == 4
    assert math.isclose(1.0 / (1.0 + math.exp(-math.log(tau / (1.0 - tau)))), tau)
