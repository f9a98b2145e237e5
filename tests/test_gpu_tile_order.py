"""gs_tile_order: the compositing kernels' launch order (tiles by descending
list length, in buckets of 8 instances). The order is a scheduling aid: the
forward's outputs are bit-identical with and without it."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

BUCKET = 8
NBUCKETS = 1024


def _bucket(lengths):
    return np.minimum(lengths // BUCKET, NBUCKETS - 1)


def _frame(gs, sg):
    sc, _ = sg.room_case()
    cam = sg.room_trajectory(3).as_f32()
    dev = "cuda"
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
    proj = gs.project(cam, t(sc.means), t(sc.scales), t(sc.quats), t(sc.opacity))
    srt = gs.bin_sort(cam, proj, max(int(proj["n_instances"].item()), 1))
    return sc, cam, proj, srt, t


def test_order_is_a_permutation_by_descending_length(gs, sg):
    sc, cam, proj, srt, _ = _frame(gs, sg)
    order = srt["tile_order"].cpu().numpy()
    r = srt["tile_ranges"].cpu().numpy()
    T = r.shape[0]
    assert np.array_equal(np.sort(order), np.arange(T))
    b = _bucket((r[:, 1] - r[:, 0])[order])
    assert np.all(np.diff(b) <= 0)           # buckets of non-increasing length
    assert b[0] > b[-1]                       # the frame has long and empty tiles


def test_forward_outputs_do_not_depend_on_the_order(gs, sg):
    sc, cam, proj, srt, t = _frame(gs, sg)
    cols, feats = t(sc.colors), t(sc.feats)
    a = gs.render_fwd(cam, proj, srt, cols, feats, status=srt["status"])
    plain = {k: v for k, v in srt.items() if k != "tile_order"}
    b = gs.render_fwd(cam, proj, plain, cols, feats, status=srt["status"])
    for k in ("rgb", "depth", "alpha", "feat", "T_final", "last_idx", "n_contrib"):
        assert torch.equal(a[k], b[k]), k


@pytest.mark.parametrize("T", [1, 5, 1000, 5000])
def test_small_and_ragged_tile_counts(gs, T):
    rng = np.random.default_rng(T)
    lengths = rng.integers(0, 20000, size=T).astype(np.int32)
    lengths[rng.random(T) < 0.3] = 0
    starts = np.concatenate([[0], np.cumsum(lengths)[:-1]]).astype(np.int32)
    ranges = torch.from_numpy(np.stack([starts, starts + lengths], 1)).cuda()
    order = torch.full((T,), -1, dtype=torch.int32, device="cuda")
    lib = gs.lib()
    import ctypes
    assert lib.gs_tile_order(T, ctypes.c_void_p(ranges.data_ptr()), ctypes.c_void_p(order.data_ptr()), None) == 0
    torch.cuda.synchronize()
    o = order.cpu().numpy()
    assert np.array_equal(np.sort(o), np.arange(T))
    assert np.all(np.diff(_bucket(lengths[o])) <= 0)


def test_adjoint_with_and_without_stored_masks(gs, sg):
    """The forward's per-instance skip masks (inst_masks) change only which
    pixel blocks skip a Gaussian: the adjoint that reads them equals the one
    that tests each Gaussian again, to the summation order of its atomics
    (1e-5 normwise: the room frame's sums cancel)."""
    sc, cam, proj, srt, t = _frame(gs, sg)
    means, scales, quats, cols, feats = (t(x) for x in (sc.means, sc.scales, sc.quats, sc.colors, sc.feats))
    fw = gs.render_fwd(cam, proj, srt, cols, feats, status=srt["status"])
    rng = np.random.default_rng(8)
    g_rgb = torch.from_numpy(rng.normal(size=(3, cam.height, cam.width)).astype(np.float32)).cuda()
    g_feat = torch.from_numpy(rng.normal(size=(sc.N, cam.height, cam.width)).astype(np.float32)).cuda()
    a = gs.render_bwd(cam, means, scales, quats, cols, feats, proj, srt, fw, g_rgb, None, None, g_feat)
    plain = {k: v for k, v in srt.items() if k != "inst_masks"}
    b = gs.render_bwd(cam, means, scales, quats, cols, feats, proj, plain, fw, g_rgb, None, None, g_feat)
    torch.cuda.synchronize()
    # every instance the adjoint reads (a tile's positions below its largest
    # last index, all loaded by the forward) holds a 4-bit mask
    masks = srt["inst_masks"].cpu().numpy()
    r = srt["tile_ranges"].cpu().numpy()
    last = fw["last_idx"].cpu().numpy()
    H, W = last.shape
    tx = (W + 15) // 16
    pad = np.zeros(((H + 15) // 16 * 16, tx * 16), np.int32)
    pad[:H, :W] = last
    maxlast = pad.reshape(pad.shape[0] // 16, 16, tx, 16).max(axis=(1, 3)).ravel()
    read = np.concatenate([np.arange(r[t, 0], r[t, 0] + maxlast[t]) for t in range(r.shape[0]) if maxlast[t] > 0])
    assert read.size > 100_000 and masks[read].max() <= 15
    for k in ("means", "scales", "quats", "opacity", "colors", "feats", "pose"):
        x, y = a[k].double(), b[k].double()
        assert float((x - y).norm() / y.norm()) <= 1e-5, k


def test_masks_from_the_chunked_forward_serve_a_pose_only_adjoint(gs, sg):
    """N = 32 features composite on the one-pixel kernel in 32-channel chunks;
    its first chunk stores the same 8x8-block masks, which a features-off
    (pose-only, as in tracking) adjoint of the same frame then reads."""
    sc, cam = sg.small_case(seed=6, N=32)
    cam = cam.as_f32()
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    means, scales, quats, opac, cols, feats = (t(x) for x in (sc.means, sc.scales, sc.quats, sc.opacity, sc.colors,
                                                              sc.feats))
    proj = gs.project(cam, means, scales, quats, opac)
    srt = gs.bin_sort(cam, proj, max(int(proj["n_instances"].item()), 1))
    fw = gs.render_fwd(cam, proj, srt, cols, feats, status=srt["status"])
    rng = np.random.default_rng(9)
    g_rgb = torch.from_numpy(rng.normal(size=(3, cam.height, cam.width)).astype(np.float32)).cuda()
    g_depth = torch.from_numpy(rng.normal(size=(cam.height, cam.width)).astype(np.float32)).cuda()
    a = gs.render_bwd(cam, means, scales, quats, cols, None, proj, srt, fw, g_rgb, g_depth, None, None,
                      flags=gs.GS_FEAT_OFF)
    plain = {k: v for k, v in srt.items() if k != "inst_masks"}
    b = gs.render_bwd(cam, means, scales, quats, cols, None, proj, plain, fw, g_rgb, g_depth, None, None,
                      flags=gs.GS_FEAT_OFF)
    torch.cuda.synchronize()
    for k in ("means", "scales", "quats", "opacity", "colors", "pose"):
        x, y = a[k].double(), b[k].double()
        assert float(y.norm()) > 0, k
        assert float((x - y).norm() / y.norm()) <= 1e-5, k
