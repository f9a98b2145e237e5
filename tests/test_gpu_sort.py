"""gs_bin_sort's per-tile sort against the FP64 oracle's lists (Sec. 3.1: the
instances of a tile in front-to-back order; the oracle sorts the (tile, depth
bits, id) triples with std::sort, pinned by brute force).

The sort places every instance into its tile's range and then sorts each
tile's (depth bits, id) pairs on their own: lists of up to 2048 keys in one
piece, longer ones as 2048-key runs merged pairwise. The "pile" scenes here put
every Gaussian over all tiles of a 48x32 image (6 tiles), so each list holds
all P Gaussians, and draw the depths from 7 values, so most keys tie on depth
and are ordered by id alone. The list lengths straddle every size class of the
sort: 1, 256 / 257 (one key per thread), 2048 / 2049 (the last single piece
and the first merged list), 4097 (three runs: an odd run copied through a
merge round) and 9000 (five runs, three merge rounds).
"""
import numpy as np
import pytest
import torch

from paper_2504_19409_gb300 import scenegen as sg_mod

pytestmark = pytest.mark.gpu


def pile_scene(P, seed=11):
    cam = sg_mod.identity_camera(48, 32, 50.0)
    rng = np.random.default_rng(seed)
    z = rng.choice(np.array([1.5, 2.0, 2.5, 3.0, 3.5, 4.0, 4.5]), P)
    xy = rng.uniform(-0.05, 0.05, (P, 2)) * z[:, None]
    means = np.column_stack([xy, z]).astype(np.float32)
    scales = np.full((P, 3), 1.5, np.float32)  # >= 3 sigma of 16 px at z = 4.5: the whole image
    quats = np.tile(np.array([1, 0, 0, 0], np.float32), (P, 1))
    sc = sg_mod.Scene(means, scales, quats, np.full(P, 0.5, np.float32), np.full((P, 3), 0.5, np.float32),
                      np.zeros((P, 0), np.float32))
    return sc, cam.as_f32()


def _project(gs, cam, sc):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return gs.project(cam, t(sc.means), t(sc.scales), t(sc.quats), t(sc.opacity))


def _oracle_lists(ora, cam, sc):
    pr = ora.project_b32(cam, sc.means, sc.scales, sc.quats, sc.opacity)
    return pr, *ora.bin_lists(cam, pr["rect"], pr["depth"])


@pytest.mark.parametrize("P", [1, 256, 257, 2048, 2049, 4097, 9000])
def test_pile_lists_match_oracle(gs, ora, P):
    sc, cam = pile_scene(P)
    T = cam.tiles_x * cam.tiles_y
    proj = _project(gs, cam, sc)
    I = int(proj["n_instances"].item())
    assert I == P * T  # every Gaussian over every tile
    srt = gs.bin_sort(cam, proj, I, tile_order=False)
    torch.cuda.synchronize()
    assert int(srt["status"].item()) == 0
    pr, ranges, gids = _oracle_lists(ora, cam, sc)
    assert np.array_equal(srt["tile_ranges"].cpu().numpy(), ranges)
    assert np.array_equal(srt["gids"].cpu().numpy()[:I].view(np.uint32), gids.astype(np.uint32))
    # the 64-bit keys: (tile << 32) | depth bits of the listed Gaussian
    keys = srt["keys"].cpu().numpy()[:I].view(np.uint64)
    tile_of = np.repeat(np.arange(T, dtype=np.uint64), np.diff(ranges, axis=1).ravel())
    want = (tile_of << np.uint64(32)) | pr["depth"].view(np.uint32)[gids].astype(np.uint64)
    assert np.array_equal(keys, want)
    # the scene is what it claims: many ties on depth
    if P >= 256:
        assert len(np.unique(pr["depth"].view(np.uint32))) <= 7


def test_capacity_truncation_keeps_valid_sorted_ranges(gs, ora):
    """18,000 instances (3,000 per tile) into a capacity of 10,000: tiles 0-2
    complete and equal to the oracle's, tile 3 cut to 1,000 entries (some of
    its instances, sorted, each once), tiles 4 and 5 empty, the flag set."""
    P = 3000
    sc, cam = pile_scene(P, seed=12)
    proj = _project(gs, cam, sc)
    I = int(proj["n_instances"].item())
    assert I == 6 * P
    cap = 10_000
    srt = gs.bin_sort(cam, proj, cap, tile_order=False)
    torch.cuda.synchronize()
    assert int(srt["status"].item()) & (1 << gs.GS_ERR_CAPACITY)
    assert int(srt["n_instances"].item()) == I
    rg = srt["tile_ranges"].cpu().numpy()
    _, ranges, gids = _oracle_lists(ora, cam, sc)
    assert np.array_equal(rg[:3], ranges[:3])
    assert rg[3].tolist() == [3 * P, cap] and rg[4:].tolist() == [[0, 0], [0, 0]]
    got = srt["gids"].cpu().numpy().view(np.uint32)
    assert np.array_equal(got[:3 * P], gids[:3 * P].astype(np.uint32))
    part = got[3 * P:cap].astype(np.int64)
    assert len(np.unique(part)) == len(part) and part.max() < P
    depth_bits = proj["depth"].cpu().numpy().view(np.uint32).astype(np.uint64)
    k = (depth_bits[part] << np.uint64(32)) | part.astype(np.uint64)
    assert np.all(k[1:] > k[:-1])


def test_sort_is_repeatable_on_a_dirty_workspace(gs, ora, sg):
    """The slots inside a tile are taken in whatever order the atomics give;
    the sorted lists must not depend on it, nor on what the workspace held:
    three sorts of the 2,000-Gaussian case, the workspace filled with 0xFF
    bytes before the first, give the oracle's lists each time."""
    sc, cam = sg.small_case(seed=4, P=2000, N=0)
    cam = cam.as_f32()
    proj = _project(gs, cam, sc)
    I = int(proj["n_instances"].item())
    T = cam.tiles_x * cam.tiles_y
    ws = torch.full((gs.bin_sort_workspace_bytes(sc.P, I, T),), 255, dtype=torch.uint8, device="cuda")
    _, ranges, gids = _oracle_lists(ora, cam, sc)
    for _ in range(3):
        srt = gs.bin_sort(cam, proj, I, workspace=ws, tile_order=False)
        torch.cuda.synchronize()
        assert int(srt["status"].item()) == 0
        assert np.array_equal(srt["tile_ranges"].cpu().numpy(), ranges)
        assert np.array_equal(srt["gids"].cpu().numpy()[:I].view(np.uint32), gids.astype(np.uint32))


def test_many_tiles_and_an_empty_frame(gs, ora):
    """2,000 Gaussians on a 2560 x 1440 image (14,400 tiles: the one-block range
    scan takes 15 tiles per thread, in two rounds of loads), then the same
    Gaussians all behind the camera (no instance: every range (0, 0), I = 0)."""
    sc, _ = sg_mod.small_case(seed=13, P=2000, N=0)
    cam = sg_mod.identity_camera(2560, 1440, 1000.0).as_f32()
    assert cam.tiles_x * cam.tiles_y == 14400
    proj = _project(gs, cam, sc)
    I = int(proj["n_instances"].item())
    assert I > 10_000
    srt = gs.bin_sort(cam, proj, I, tile_order=False)
    torch.cuda.synchronize()
    assert int(srt["status"].item()) == 0
    _, ranges, gids = _oracle_lists(ora, cam, sc)
    assert np.array_equal(srt["tile_ranges"].cpu().numpy(), ranges)
    assert np.array_equal(srt["gids"].cpu().numpy()[:I].view(np.uint32), gids.astype(np.uint32))
    behind = sg_mod.Scene(sc.means * np.array([1, 1, -1], np.float32), sc.scales, sc.quats, sc.opacity, sc.colors,
                          sc.feats)
    proj = _project(gs, cam, behind)
    assert int(proj["n_instances"].item()) == 0
    srt = gs.bin_sort(cam, proj, 16, tile_order=False)
    torch.cuda.synchronize()
    assert int(srt["status"].item()) == 0
    assert int(srt["n_instances"].item()) == 0
    assert not srt["tile_ranges"].any()
