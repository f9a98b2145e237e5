"""Full-size parity of the forms the benchmark times, against the FP64 oracle
on a band of tile rows.

* The wide-feature form (500,000 Gaussians in the box room, 1200 x 680,
  N = 512 unit-norm bf16 features, the tensor-core forward and adjoint),
  as bench.py launches it (Rasterizer, HWC, GS_FEAT_TENSOR_CORE).
* The SLAM-frame step's adjoint (300,000 Gaussians, N = 16): the L1 loss as
  sign words (gs_l1_signs) and the adjoint that rebuilds its cotangents from
  them (gs_render_bwd_l1), every gradient class and the pose.

The GPU renders the whole frame. The oracle composites only the tiles of a
band of tile rows (its other tile ranges are emptied, and the Gaussians the
band lists are renumbered), since its FP64 512-channel sums over a whole frame
take minutes. For the adjoints the cotangents are zero outside the band (for
the L1 loss, targets equal to the render there, so every sign is 0), so the
whole-frame GPU gradients and the band's oracle gradients are the same sums.

Tensor-core bounds (u = 2^-8, the unit roundoff of bf16, which has 8
significant bits; GAMMA = 1e-5, the fp32 bar of the plain path):
* forward, per pixel and channel: the weights w = alpha T are rounded to bf16
  (|fl(w) - w| <= u w); bf16 x bf16 products are exact in fp32; what remains
  is fp32 arithmetic (the weights' alpha and T, the accumulation), held to
  GAMMA relative to sum_i w_i |f_i| as the plain fp32 path is:
      |F_tc - F| <= (u + GAMMA (1 + u)) sum_i w_i |f_i| + 1e-7;
* adjoint, per Gaussian and channel: both factors of each product are
  rounded (w and dL/dF), |fl(w) fl(g) - w g| <= (2u + u^2) |w g|:
      |df_tc - df| <= (2u + u^2 + GAMMA (1 + u)^2) sum_p w_p |g_p| + 1e-7.
sum_i w_i |f_i| and sum_p w_p |g_p| are the oracle's renders of |f| and |g|.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

U = 2.0 ** -8
GAMMA = 1e-5
MARGIN = 1e-5
BAND = (20, 22)  # tile rows [20, 22): pixel rows 320..351 of the 680


def _t(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def _bf16_exact(f):
    return torch.from_numpy(np.ascontiguousarray(f)).to(torch.bfloat16).float().numpy().astype(np.float64)


def _band(cam, ranges, gids, band=BAND):
    """Oracle lists restricted to the band's tiles, the Gaussians renumbered to
    those the band lists (returned as `used`, ascending)."""
    tx = cam.tiles_x
    keep = np.zeros(len(ranges), bool)
    keep[band[0] * tx:band[1] * tx] = True
    r = np.where(keep[:, None], ranges, 0).astype(np.int32)
    used = np.unique(np.concatenate([gids[a:b] for a, b in r[keep]]))
    remap = np.zeros(int(gids.max()) + 1, np.int32)
    remap[used] = np.arange(len(used), dtype=np.int32)
    return r, remap[gids], used


def _rows(band=BAND):
    return slice(16 * band[0], 16 * band[1])


@pytest.fixture(scope="module")
def wide(gs, ora, sg):
    sc = sg.room_scene(6, 500_000, 512, feat_kind="unit")
    cam = sg.room_trajectory(3, 100, 1200, 680, 600.0).as_f32()
    means, scales, quats, opac, cols = (_t(x) for x in (sc.means, sc.scales, sc.quats, sc.opacity, sc.colors))
    feats = _t(sc.feats, torch.bfloat16)
    ras = gs.Rasterizer(sc.P, cam.width, cam.height, N=512, layout=gs.GS_LAYOUT_HWC,
                        flags=gs.GS_FEAT_ON | gs.GS_FEAT_TENSOR_CORE)
    ras.ensure_capacity(cam, means, scales, quats, opac)
    fw = ras.forward(cam, means, scales, quats, opac, cols, feats)
    torch.cuda.synchronize()
    ras.check_status()
    I = int(ras.sort["n_instances"].item())
    pr = ora.project_b32(cam, sc.means, sc.scales, sc.quats, sc.opacity)
    ranges, gids = ora.bin_lists(cam, pr["rect"], pr["depth"])
    assert I == len(gids) and np.array_equal(ras.sort["tile_ranges"].cpu().numpy(), ranges)
    assert np.array_equal(ras.sort["gids"][:I].cpu().numpy(), gids)
    rb, gb, used = _band(cam, ranges, gids)
    rec = dict(uv=pr["uv"][used], conic=pr["conic"][used], opacity=sc.opacity[used], colors=sc.colors[used],
               depth=pr["depth"][used])
    f_exact = _bf16_exact(sc.feats[used])
    rows = _rows()
    out = dict(sc=sc, cam=cam, ras=ras, tensors=(means, scales, quats, opac, cols, feats), rb=rb, gb=gb, used=used,
               rec=rec, f_exact=f_exact, F_tc=fw["feat"][rows].cpu().numpy(),
               last_idx=fw["last_idx"][rows].cpu().numpy(), n_contrib=fw["n_contrib"][rows].cpu().numpy())
    yield out
    del out
    torch.cuda.empty_cache()


def _oracle_fwd(ora, w, feats):
    r = w["rec"]
    fo = ora.render_fwd(w["cam"], w["rb"], w["gb"], r["uv"], r["conic"], r["opacity"], r["colors"], r["depth"], feats)
    rows = _rows()
    # copies, so that the whole-frame arrays (3.3 GB of features) are freed
    return {k: np.ascontiguousarray(v[..., rows, :]) for k, v in fo.items()}


def test_wide_tensor_core_forward_band_vs_oracle(ora, wide):
    fo = _oracle_fwd(ora, wide, wide["f_exact"])
    ok = fo["margin"] > MARGIN
    assert (~ok).sum() <= max(3, int(1e-3 * ok.size))
    assert np.array_equal(wide["n_contrib"][ok], fo["n_contrib"][ok])
    assert np.array_equal(wide["last_idx"][ok], fo["last_idx"][ok])
    assert fo["n_contrib"].mean() > 5
    S = _oracle_fwd(ora, wide, np.abs(wide["f_exact"]))["feat"]
    F_tc = np.transpose(wide["F_tc"], (2, 0, 1)).astype(np.float64)
    err = np.abs(F_tc - fo["feat"])[:, ok]
    bound = (U + GAMMA * (1 + U)) * S[:, ok] + 1e-7
    ratio = err / bound
    assert (ratio <= 1.0).all(), float(ratio.max())
    assert ratio.max() > 0.05  # the bound is not vacuous


def test_wide_tensor_core_adjoint_band_vs_oracle(gs, ora, wide):
    cam, ras = wide["cam"], wide["ras"]
    means, scales, quats, opac, cols, feats = wide["tensors"]
    H, W, N = cam.height, cam.width, 512
    rows = _rows()
    rng = np.random.default_rng(42)
    g_band = (rng.standard_normal((rows.stop - rows.start, W, N)) / N).astype(np.float32)
    g_f = torch.zeros(H, W, N, device="cuda")
    g_f[rows] = _t(g_band)
    gr = ras.backward(cam, means, scales, quats, cols, feats, g_feat=g_f)
    torch.cuda.synchronize()
    ras.check_status()
    d_tc = gr["feats"].cpu().numpy()
    del g_f
    used = wide["used"]
    others = np.ones(d_tc.shape[0], bool)
    others[used] = False
    assert not d_tc[others].any()  # nothing reaches Gaussians the band does not list
    r = wide["rec"]
    g_chw = np.zeros((N, H, W))
    g_chw[:, rows, :] = np.transpose(g_band, (2, 0, 1))
    ref = ora.render_bwd(cam, wide["rb"], wide["gb"], r["uv"], r["conic"], r["opacity"], r["colors"], r["depth"],
                         wide["f_exact"], None, None, None, g_chw)["d_feats"]
    np.abs(g_chw, out=g_chw)
    S = ora.render_bwd(cam, wide["rb"], wide["gb"], r["uv"], r["conic"], r["opacity"], r["colors"], r["depth"],
                       wide["f_exact"], None, None, None, g_chw)["d_feats"]
    del g_chw
    err = np.abs(d_tc[used] - ref)
    bound = (2 * U + U * U + GAMMA * (1 + U) ** 2) * S + 1e-7
    ratio = err / bound
    assert (ratio <= 1.0).all(), float(ratio.max())
    assert ratio.max() > 0.02


def test_l1_sign_adjoint_slam_frame_band_vs_oracle(gs, ora, sg):
    """The benchmark step's adjoint (k_render_bwd_mma with the L1 sign operand)
    on a whole SLAM frame: gradients of every class and the pose within 1e-4
    normwise (cosine >= 0.99999) of the oracle given the same cotangents."""
    sc, _ = sg.room_case()
    cam = sg.room_trajectory(9).as_f32()
    H, W, N = cam.height, cam.width, sc.N
    means, scales, quats, opac, cols, feats = (_t(x) for x in (sc.means, sc.scales, sc.quats, sc.opacity, sc.colors,
                                                               sc.feats))
    ras = gs.Rasterizer(sc.P, W, H, N=N)
    ras.ensure_capacity(cam, means, scales, quats, opac)
    fw = ras.forward(cam, means, scales, quats, opac, cols, feats)
    rows = _rows()
    rng = np.random.default_rng(9)
    targets = {k: fw[k].clone() for k in ("rgb", "depth", "feat")}
    for k in targets:  # perturb the band rows only: elsewhere every sign is 0
        band = targets[k][..., rows, :]
        band += _t(rng.normal(scale=0.05, size=tuple(band.shape)).astype(np.float32))
    HW = H * W
    weights = {"rgb": 1.0 / (3 * HW), "depth": 1.0 / HW, "feat": 1.0 / (N * HW)}
    loss = torch.zeros(1, device="cuda")
    ras.l1_loss(cam, targets, weights, loss)
    gr = ras.backward_l1(cam, means, scales, quats, cols, feats, weights)
    torch.cuda.synchronize()
    ras.check_status()
    got = {k: v.double().cpu().numpy() for k, v in gr.items()}
    # the oracle's cotangents: w sign(pred - target) from the same binary32 differences
    cot = {}
    for k in ("rgb", "depth", "feat"):
        d = fw[k].cpu().numpy() - targets[k].cpu().numpy()
        cot[k] = np.sign(d).astype(np.float64) * float(np.float32(weights[k]))
        outside = np.ones(d.shape[-2], bool)
        outside[rows] = False
        assert not cot[k][..., outside, :].any()
    pr = ora.project_b32(cam, sc.means, sc.scales, sc.quats, sc.opacity)
    ranges, gids = ora.bin_lists(cam, pr["rect"], pr["depth"])
    tx = cam.tiles_x
    keep = np.zeros(len(ranges), bool)
    keep[BAND[0] * tx:BAND[1] * tx] = True
    rb = np.where(keep[:, None], ranges, 0).astype(np.int32)
    ob = ora.render_bwd(cam, rb, gids, pr["uv"], pr["conic"], sc.opacity, sc.colors, pr["depth"], sc.feats,
                        cot["rgb"], cot["depth"], None, cot["feat"])
    pb = ora.project_bwd_f64(cam, sc.means, sc.scales, sc.quats, sc.opacity, ob["d_uv"], ob["d_conic"],
                             ob["d_depth"])
    want = dict(means=pb["d_means"], scales=pb["d_scales"], quats=pb["d_quats"], opacity=ob["d_opacity"],
                colors=ob["d_colors"], feats=ob["d_feats"], pose=pb["d_pose"])
    for k, b in want.items():
        a, b = got[k].ravel(), b.ravel()
        nb = np.linalg.norm(b)
        assert nb > 0, k
        rel = np.linalg.norm(a - b) / nb
        c = float(a @ b / (np.linalg.norm(a) * nb))
        assert rel <= 1e-4 and c >= 0.99999, (k, rel, c)
