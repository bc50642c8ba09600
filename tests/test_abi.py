"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
entry point include/gs.h declares; host-side argument checks reject bad calls
before anything is enqueued (no compute call is made here)."""
import ctypes
import os
import re

import pytest

import paper_2405_19614_gb300 as gs
from paper_2405_19614_gb300 import _lib
from paper_2405_19614_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return _lib.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"binding lacks {name}"


def test_version_and_status_strings(lib):
    assert lib.gs_version().decode().startswith("gs-sm103a")
    assert lib.gs_status_string(3).decode() == "pair capacity exceeded"


def test_layout_and_sizes(lib):
    views = gs.make_views([[60, 60, 32, 24], [600, 600, 600, 340]], [[64, 48], [1200, 680]])
    nt, npix = ctypes.c_int64(), ctypes.c_int64()
    assert lib.gs_layout(views, 2, ctypes.byref(nt), ctypes.byref(npix)) == 0
    assert nt.value == 4 * 3 + 75 * 43 and npix.value == 64 * 48 + 1200 * 680
    assert lib.gs_grad2d_size(1000, 3) == 1000 * 3 * 48
    assert lib.gs_bin_sort_workspace_size(1000, 1 << 20, 12) >= 8 * (1 << 20) + 16 * 1000


def test_tile_shapes_in_the_layout(lib):
    nt, npix = ctypes.c_int64(), ctypes.c_int64()
    for (tw, th) in [(8, 8), (16, 8), (32, 16), (64, 32), (16, 16)]:
        views = gs.make_views([[600, 600, 600, 340]], [[1200, 680]], (tw, th))
        assert lib.gs_layout(views, 1, ctypes.byref(nt), ctypes.byref(npix)) == 0
        assert nt.value == -(-1200 // tw) * -(-680 // th)
    for bad in [(12, 16), (16, 4), (64, 64), (128, 8)]:
        views = gs.make_views([[600, 600, 600, 340]], [[1200, 680]], bad)
        assert lib.gs_layout(views, 1, ctypes.byref(nt), ctypes.byref(npix)) == 1, bad
    assert gs.variant_fits(3, (16, 16)) and not gs.variant_fits(3, (16, 8))  # (4, 8): 8 x 16 bands


def test_argument_errors_are_synchronous(lib):
    views = gs.make_views([[60, 60, 32, 24]], [[64, 48]])
    bad = gs.make_views([[60, 60, 32, 24]], [[0, 48]])
    opt = _lib.GsOptions(0.2, 0.3)
    params = _lib.GsParams(None, None, None, None, None, 10, 0)
    proj = _lib.GsProjected(None, None, None)
    assert lib.gs_project(None, views, None, 1, ctypes.byref(opt), ctypes.byref(proj), None) == 1
    assert lib.gs_project(ctypes.byref(params), bad, ctypes.c_void_p(16), 1, ctypes.byref(opt),
                          ctypes.byref(proj), None) == 1
    params.sh_degree = 4
    assert lib.gs_project(ctypes.byref(params), views, ctypes.c_void_p(16), 1, ctypes.byref(opt),
                          ctypes.byref(proj), None) == 1
    assert lib.gs_layout(views, 0, None, None) == 1
    assert lib.gs_layout(views, 65, None, None) == 1
    bins = _lib.GsBins(None, None, None, None, None, 0)
    assert lib.gs_bin_sort(ctypes.byref(proj), 10, views, 1, ctypes.byref(bins), None, 0, None) == 1
    grp = (_lib.GsAdamGroup * 1)(_lib.GsAdamGroup(0, 10, 1e-3))
    assert lib.gs_adam_step(None, None, None, None, grp, 1, 0.9, 0.999, 1e-15, None, None) == 1
    assert lib.gs_pose_update(None, None, 1, None) == 1
    assert lib.gs_loss_l1(None, None, None, None, None, -1, 1.0, 1.0, 0, 0.99, None, None, None, None) == 1
    assert lib.gs_reproj_loss_grad(None, None, None, -1, views, None, 1, 1.0, 0.2, None, None, None) == 1


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libgs.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(_lib.GsError):
        _lib.load()
