"""gs_bin_sort_static: the tile x depth sort for callers that cannot allocate
device memory (a tracking thread with a frame deadline, or a host that owns
every allocation). It keeps its scratch space in a fixed array inside the
library, so its results must equal gs_bin_sort's (which uses a caller
workspace) bit for bit, call after call, although the array keeps whatever
the previous call left in it.

This file is collected last so that a run that stops at the first failure
has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _projected(gs, sg, cam, sc):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return gs.project(cam, t(sc.means), t(sc.scales), t(sc.quats), t(sc.opacity))


def _static_sort(gs, cam, proj, capacity, with_keys=True):
    T = cam.tiles_x * cam.tiles_y
    out = dict(keys=torch.full((capacity,), -1, dtype=torch.int64, device="cuda"),
               gids=torch.full((capacity,), -1, dtype=torch.int32, device="cuda"),
               tile_ranges=torch.full((T, 2), -1, dtype=torch.int32, device="cuda"),
               n_instances=torch.zeros(1, dtype=torch.int64, device="cuda"),
               status=torch.zeros(1, dtype=torch.int32, device="cuda"))
    c = gs.camera_struct(cam)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = gs.lib().gs_bin_sort_static(ctypes.byref(c), proj["depth"].shape[0], _ptr(proj["depth"]),
                                       _ptr(proj["rect"]), _ptr(proj["tiles_touched"]), capacity,
                                       _ptr(out["keys"]) if with_keys else None,
                                       _ptr(out["gids"]), _ptr(out["tile_ranges"]), _ptr(out["n_instances"]),
                                       _ptr(out["status"]), stream)
    assert code == gs.GS_OK, gs.lib().gs_status_string(code)
    if not with_keys:
        out["keys"] = None
    return out


def _same(gs, a, b):
    torch.cuda.synchronize()
    I = int(a["n_instances"].item())
    assert I == int(b["n_instances"].item()) and I > 0
    assert int(a["status"].item()) == 0 and int(b["status"].item()) == 0
    assert torch.equal(a["tile_ranges"], b["tile_ranges"])
    assert torch.equal(a["gids"][:I], b["gids"][:I])
    if a["keys"] is not None:
        assert torch.equal(a["keys"][:I], b["keys"][:I])


def test_static_scratch_sort_equals_workspace_sort_twice(gs, sg):
    """Two calls in a row on different frames: each equals gs_bin_sort."""
    sc, _ = sg.room_case(seed=3, P=120_000, N=0)
    for k in (11, 12):
        cam = sg.room_trajectory(k, width=640, height=360, f=320.0).as_f32()
        proj = _projected(gs, sg, cam, sc)
        I = int(proj["n_instances"].item())
        cap = I + 1000
        ref = gs.bin_sort(cam, proj, cap)
        got = _static_sort(gs, cam, proj, cap)
        _same(gs, got, ref)


def test_static_scratch_sort_large_then_small(gs, sg):
    """A large sort, then a small one in the same array (which keeps the large
    sort's words past the small one's end): both equal gs_bin_sort, whatever
    ran before this test."""
    sc, _ = sg.room_case(seed=3, P=120_000, N=0)
    cam = sg.room_trajectory(13, width=640, height=360, f=320.0).as_f32()
    proj = _projected(gs, sg, cam, sc)
    I = int(proj["n_instances"].item())
    _same(gs, _static_sort(gs, cam, proj, I + 1000), gs.bin_sort(cam, proj, I + 1000))
    sc, cam = sg.small_case(seed=4, P=2000, N=0)
    cam = cam.as_f32()
    proj = _projected(gs, sg, cam, sc)
    I = int(proj["n_instances"].item())
    _same(gs, _static_sort(gs, cam, proj, I), gs.bin_sort(cam, proj, I))


def test_static_scratch_sort_without_keys(gs, sg):
    """keys = NULL (the 64-bit keys are optional, as for gs_bin_sort): the
    lists and ranges still equal gs_bin_sort's."""
    sc, cam = sg.small_case(seed=5, P=2000, N=0)
    cam = cam.as_f32()
    proj = _projected(gs, sg, cam, sc)
    I = int(proj["n_instances"].item())
    _same(gs, _static_sort(gs, cam, proj, I + 7, with_keys=False), gs.bin_sort(cam, proj, I + 7))


def test_static_scratch_rejects_sizes_beyond_the_array(gs, sg):
    sc, cam = sg.small_case(seed=4, P=500, N=0)
    cam = cam.as_f32()
    proj = _projected(gs, sg, cam, sc)
    limit = 32 << 20
    cap = 1
    while gs.bin_sort_workspace_bytes(500, cap, cam.tiles_x * cam.tiles_y) <= limit:
        cap *= 2
    big = torch.zeros(1, dtype=torch.int64, device="cuda")
    c = gs.camera_struct(cam)
    code = gs.lib().gs_bin_sort_static(ctypes.byref(c), 500, _ptr(proj["depth"]), _ptr(proj["rect"]),
                                       _ptr(proj["tiles_touched"]), cap, _ptr(big), _ptr(big), _ptr(big), None, None,
                                       None)
    assert code == gs.GS_ERR_INVALID_ARG
