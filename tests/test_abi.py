"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/gsff.h declares (no GPU needed; no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    hdr = open(os.path.join(ROOT, "include", "gsff.h")).read()
    return sorted(set(re.findall(r"^\s*(?:const char\*|gs_status|size_t|int32_t|void)\s+(gs_\w+)\s*\(", hdr, re.M)))


@pytest.fixture(scope="module")
def built():
    from paper_2504_19409_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    names = _declared()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    import paper_2504_19409_gb300 as g
    assert set(g.EXPORTS) == set(names)


def test_host_only_entry_points(built):
    import paper_2504_19409_gb300 as g
    L = g.lib()
    assert L.gs_version() == 1
    assert L.gs_status_string(g.GS_ERR_CAPACITY) == b"instance capacity exceeded"
    # workspace sizing is pure host arithmetic
    a = g.bin_sort_workspace_bytes(1000, 5000, 48)
    b = g.bin_sort_workspace_bytes(1000, 50000, 48)
    assert a >= 5000 * 16 and b > a and a % 256 == 0
    assert g.render_bwd_workspace_bytes(1000) >= 1000 * 24


def test_invalid_arguments_rejected_synchronously(built):
    """Bad arguments come back as GS_ERR_INVALID_ARG before anything is
    launched (null camera, negative sizes, missing outputs)."""
    import paper_2504_19409_gb300 as g
    L = g.lib()
    assert L.gs_project(None, 10, *([None] * 11)) == g.GS_ERR_INVALID_ARG
    cam = g.GsCamera()
    cam.width, cam.height, cam.fx, cam.fy = 64, 48, 50.0, 50.0
    assert L.gs_project(ctypes.byref(cam), -1, *([None] * 11)) == g.GS_ERR_INVALID_ARG
    assert L.gs_project(ctypes.byref(cam), 5, *([None] * 11)) == g.GS_ERR_INVALID_ARG
    assert L.gs_bin_sort(ctypes.byref(cam), 5, None, None, None, 0, None, 0, None, None, None, None, None,
                         None) == g.GS_ERR_INVALID_ARG
    assert L.gs_l1_loss_grad(-1, None, None, 1.0, None, None, None) == g.GS_ERR_INVALID_ARG
    assert L.gs_tile_order(-1, None, None, None) == g.GS_ERR_INVALID_ARG
    assert L.gs_tile_order(4, None, None, None) == g.GS_ERR_INVALID_ARG
    assert L.gs_tile_order(0, None, None, None) == g.GS_OK
    assert L.gs_zero(None, 16, None) == g.GS_ERR_INVALID_ARG
    assert L.gs_zero(None, 0, None) == g.GS_OK


def test_product_path_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_2504_19409_gb300 as g
    monkeypatch.setattr(g, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(g, "_lib", None)
    with pytest.raises(g.GsffError):
        g.lib()


def test_checked_build_exports_the_same_symbols():
    """The bounds-checked variant (GS_CHECKED) is the same C ABI."""
    from paper_2504_19409_gb300 import build
    lib = ctypes.CDLL(build.build(checked=True))
    for n in _declared():
        assert hasattr(lib, n), n


def test_status_word_plumbing(built):
    """Device status words decode bit by bit into the error kinds, including
    the bounds-checked build's GS_ERR_BOUNDS (no GPU needed)."""
    import paper_2504_19409_gb300 as g
    assert g.GS_ERR_BOUNDS == 6
    assert g.status_names(1 << g.GS_ERR_BOUNDS) == ["index out of range (bounds-checked build)"]
    both = (1 << g.GS_ERR_TIMEOUT) | (1 << g.GS_ERR_BOUNDS)
    assert g.status_names(both) == ["bounded wait timed out", "index out of range (bounds-checked build)"]
    assert g.status_names(0) == []
    L = g.lib()
    # the scan rejects a missing output synchronously (nothing is launched)
    assert L.gs_count_nonfinite(16, ctypes.c_void_p(256), None, None) == g.GS_ERR_INVALID_ARG
    assert L.gs_count_nonfinite(-1, None, ctypes.c_void_p(256), None) == g.GS_ERR_INVALID_ARG
