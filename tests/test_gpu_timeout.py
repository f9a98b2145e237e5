"""Failure handling of the sort's bounded waits, tested without a GPU fault.

Each radix pass of gs_bin_sort waits for earlier chunks' digit counts (the
decoupled look-back) with a bound. gs_set_lookback_wait_ns(0) makes every
chunk after the first give up before its look-back, which is the timeout path
taken deterministically: the pass flags GS_ERR_TIMEOUT in the status word and
scatters with an incomplete offset, so its output has unwritten slots. The
workspace here starts as 0xFF bytes, so those slots hold ids far past P: the
sort's later kernels must treat them as absent, and the tile ranges must stay
empty so that no render call reads a list entry. Only gs_bin_sort runs under
the forced bound; the bound is restored before anything else runs.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _scene(gs, sg, P):
    sc, cam = sg.small_case(seed=7, P=P, N=0)
    cam = cam.as_f32()
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    proj = gs.project(cam, t(sc.means), t(sc.scales), t(sc.quats), t(sc.opacity))
    return sc, cam, proj


def _outputs(cap, T):
    return dict(keys=torch.full((cap,), -1, dtype=torch.int64, device="cuda"),
                gids=torch.full((cap,), -1, dtype=torch.int32, device="cuda"),
                tile_ranges=torch.full((T, 2), -1, dtype=torch.int32, device="cuda"),
                n_instances=torch.zeros(1, dtype=torch.int64, device="cuda"))


def test_forced_lookback_timeout_is_flagged_and_leaves_no_list(gs, sg, ora):
    # 6000 Gaussians: three chunks in each depth pass and several in each tile
    # pass, so both kinds of pass take the timeout path
    sc, cam, proj = _scene(gs, sg, 6000)
    I = int(proj["n_instances"].item())
    assert I > 4 * 2048
    T = cam.tiles_x * cam.tiles_y
    ws = torch.full((gs.bin_sort_workspace_bytes(sc.P, I, T),), 255, dtype=torch.uint8, device="cuda")
    out = _outputs(I, T)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    try:
        gs.set_lookback_wait_ns(0)
        gs.bin_sort(cam, proj, I, workspace=ws, out=out, status=status, tile_order=False)
    finally:
        gs.set_lookback_wait_ns(10 ** 9)
    torch.cuda.synchronize()
    st = int(status.item())
    assert st & (1 << gs.GS_ERR_TIMEOUT), st
    assert not st & (1 << gs.GS_ERR_CUDA)
    assert torch.count_nonzero(out["tile_ranges"]).item() == 0
    assert 0 <= int(out["n_instances"].item()) <= 2 ** 31

    # the default bound: the same call, same (dirty) workspace, gives the exact lists
    status.zero_()
    out = _outputs(I, T)
    gs.bin_sort(cam, proj, I, workspace=ws, out=out, status=status, tile_order=False)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    pr = ora.project_b32(cam, sc.means, sc.scales, sc.quats, sc.opacity)
    ranges, gids = ora.bin_lists(cam, pr["rect"], pr["depth"])
    assert int(out["n_instances"].item()) == len(gids) == I
    assert np.array_equal(out["tile_ranges"].cpu().numpy(), ranges)
    assert np.array_equal(out["gids"][:I].cpu().numpy().astype(np.int64), gids.astype(np.int64))
