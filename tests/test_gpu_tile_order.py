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
