"""Tensor-core (tcgen05) form of the feature channels vs the FP64 oracle.

Error bounds, with u = 2^-8 the unit roundoff of bf16 (8 significant bits,
so |fl(x) - x| <= u |x| under round-to-nearest) and GAMMA = 1e-5 the fp32 bar
of the plain path (relative error of the fp32 weights alpha T and of the fp32
accumulation, taken relative to the sum of absolute terms):
* forward, per pixel and channel: the weights w = alpha T are rounded to
  bf16, the features are bf16 by construction (the oracle uses their exact
  values), bf16 x bf16 products are exact in fp32, so
      |F_tc - F| <= (u + GAMMA (1 + u)) sum_i w_i |f_i| + 1e-7;
* adjoint, per Gaussian and channel: w and dL/dF are both rounded, and
  |fl(w) fl(g) - w g| <= (2u + u^2) |w g|, so
      |df_tc - df| <= (2u + u^2 + GAMMA (1 + u)^2) sum_p w_p |g_p| + 1e-7.
The sums of absolute terms are the oracle's renders of |f| and |g|. RGB,
depth, alpha and the saved state come from the SIMT kernel and must equal
the plain path's bit for bit.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

U = 2.0 ** -8
GAMMA = 1e-5


def _t(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def _bf16_exact(f):
    return torch.from_numpy(np.ascontiguousarray(f)).to(torch.bfloat16).float().numpy().astype(np.float64)


def _render(gs, cam, sc, flags):
    means, scales, quats, opac, cols = (_t(x) for x in (sc.means, sc.scales, sc.quats, sc.opacity, sc.colors))
    feats = _t(sc.feats, torch.bfloat16)
    proj = gs.project(cam, means, scales, quats, opac)
    srt = gs.bin_sort(cam, proj, max(int(proj["n_instances"].item()), 1))
    vis = torch.zeros(sc.P, dtype=torch.uint8, device="cuda")
    fw = gs.render_fwd(cam, proj, srt, cols, feats, flags=flags, layout=gs.GS_LAYOUT_HWC, status=srt["status"],
                       visible=vis)
    torch.cuda.synchronize()
    assert int(srt["status"].item()) == 0
    out = {k: v.cpu().numpy() for k, v in fw.items()}
    out["visible"] = vis.cpu().numpy()
    return out


@pytest.mark.parametrize("N,shape,P,seed", [(512, (96, 64), 1500, 21), (128, (100, 37), 900, 22),
                                             (256, (64, 48), 700, 23), (448, (50, 70), 600, 24),
                                             (512, (400, 300), 6000, 25)])
def test_tc_features_within_bound(gs, ora, sg, N, shape, P, seed):
    cam = sg.identity_camera(shape[0], shape[1], 0.8 * shape[0]).as_f32()
    sc = sg.frustum_scene(seed, P, cam, N)
    g = sc.feats
    sc.feats = (g / np.linalg.norm(g, axis=1, keepdims=True)).astype(np.float32)
    f_exact = _bf16_exact(sc.feats)
    tc = _render(gs, cam, sc, gs.GS_FEAT_ON | gs.GS_FEAT_TENSOR_CORE)
    plain = _render(gs, cam, sc, gs.GS_FEAT_ON)
    for k in ("rgb", "depth", "alpha", "T_final", "last_idx", "n_contrib", "visible"):
        assert np.array_equal(tc[k], plain[k]), k
    pr = ora.project_b32(cam, sc.means, sc.scales, sc.quats, sc.opacity)
    ranges, gids = ora.bin_lists(cam, pr["rect"], pr["depth"])
    fo = ora.render_fwd(cam, ranges, gids, pr["uv"], pr["conic"], sc.opacity, sc.colors, pr["depth"], f_exact)
    fa = ora.render_fwd(cam, ranges, gids, pr["uv"], pr["conic"], sc.opacity, sc.colors, pr["depth"],
                        np.abs(f_exact))
    ok = fo["margin"] > 1e-5
    F_tc = np.transpose(tc["feat"], (2, 0, 1))
    bound = (U + GAMMA * (1 + U)) * fa["feat"] + 1e-7
    err = np.abs(F_tc - fo["feat"])
    assert (err[:, ok] <= bound[:, ok]).all(), float((err[:, ok] / bound[:, ok]).max())
    # the bound is not vacuous: the error is a visible fraction of it
    assert (err[:, ok] / bound[:, ok]).max() > 0.05
    # the plain fp32 path is far tighter
    F_pl = np.transpose(plain["feat"], (2, 0, 1))
    assert np.abs(F_pl - fo["feat"])[:, ok].max() <= 1e-5 * max(1.0, np.abs(fo["feat"]).max())


def test_tc_empty_tiles_write_zeros(gs, sg):
    cam = sg.identity_camera(64, 48, 50.0).as_f32()
    sc = sg.frustum_scene(5, 3, cam, 64)
    tc = _render(gs, cam, sc, gs.GS_FEAT_ON | gs.GS_FEAT_TENSOR_CORE)
    plain = _render(gs, cam, sc, gs.GS_FEAT_ON)
    empty = plain["n_contrib"] == 0
    assert empty.sum() > 100
    assert (tc["feat"][empty] == 0).all()


def test_tc_rejects_unsupported_shapes(gs, sg):
    cam = sg.identity_camera(64, 48, 50.0).as_f32()
    sc = sg.frustum_scene(5, 50, cam, 48)
    with pytest.raises(gs.GsffError):
        _render(gs, cam, sc, gs.GS_FEAT_ON | gs.GS_FEAT_TENSOR_CORE)


@pytest.mark.parametrize("N,shape,P,seed", [(256, (96, 64), 1200, 31), (512, (100, 37), 900, 33),
                                             (128, (64, 48), 700, 34), (384, (72, 40), 800, 35),
                                             (512, (400, 300), 6000, 36), (384, (410, 300), 6000, 37)])
def test_tc_feature_gradient_within_bound(gs, ora, sg, N, shape, P, seed):
    """Decoupled feature gradient on tcgen05 within the adjoint bound of the
    module docstring; the geometry gradients equal the fp32 path's
    (tolerance 1e-5). Every channel-block count (N / 128 = 1..4) and a
    ragged image are covered. The 400 x 300 and 410 x 300 cases have 950 and
    988 half tiles, more than one per CTA, so every half tile after a CTA's
    first takes its cotangents through the staging ring (one bulk copy per
    8-pixel row chunk): the last tile row is 12 pixels tall, so its lower
    half tiles have 4 rows of chunks with no pixel in the image (nothing
    copied, zeros converted), and at 410 pixels the last tile column is 10
    wide, so its second chunk of each row copies 2 pixels and zeros 6."""
    cam = sg.identity_camera(shape[0], shape[1], 0.73 * shape[0]).as_f32()
    sc = sg.frustum_scene(seed, P, cam, N)
    sc.feats = (sc.feats / np.linalg.norm(sc.feats, axis=1, keepdims=True)).astype(np.float32)
    f_exact = _bf16_exact(sc.feats)
    cot = sg.random_linear_functional(seed + 1, cam.height, cam.width, N)
    g_rgb, g_d, g_a, g_f = (_t(x) for x in cot)
    g_f_hwc = g_f.permute(1, 2, 0).contiguous()
    means, scales, quats, opac, cols = (_t(x) for x in (sc.means, sc.scales, sc.quats, sc.opacity, sc.colors))
    feats = _t(sc.feats, torch.bfloat16)
    out = {}
    for name, flags in (("tc", gs.GS_FEAT_ON | gs.GS_FEAT_TENSOR_CORE), ("plain", gs.GS_FEAT_ON)):
        proj = gs.project(cam, means, scales, quats, opac)
        srt = gs.bin_sort(cam, proj, max(int(proj["n_instances"].item()), 1))
        fw = gs.render_fwd(cam, proj, srt, cols, feats, flags=flags, layout=gs.GS_LAYOUT_HWC, status=srt["status"])
        gr = gs.render_bwd(cam, means, scales, quats, cols, feats, proj, srt, fw, g_rgb, g_d, g_a, g_f_hwc,
                           flags=flags, layout=gs.GS_LAYOUT_HWC, status=srt["status"])
        torch.cuda.synchronize()
        assert int(srt["status"].item()) == 0
        out[name] = {k: v.cpu().numpy() for k, v in gr.items()}
    pr = ora.project_b32(cam, sc.means, sc.scales, sc.quats, sc.opacity)
    ranges, gids = ora.bin_lists(cam, pr["rect"], pr["depth"])
    c64 = tuple(x.astype(np.float64) for x in cot)
    rb = ora.render_bwd(cam, ranges, gids, pr["uv"], pr["conic"], sc.opacity, sc.colors, pr["depth"], f_exact, *c64)
    ra = ora.render_bwd(cam, ranges, gids, pr["uv"], pr["conic"], sc.opacity, sc.colors, pr["depth"], f_exact,
                        None, None, None, np.abs(c64[3]))
    err = np.abs(out["tc"]["feats"] - rb["d_feats"])
    bound = (2 * U + U * U + GAMMA * (1 + U) ** 2) * ra["d_feats"] + 1e-7
    assert (err <= bound).all(), float((err / bound).max())
    assert (err / bound).max() > 0.02
    for k in ("means", "scales", "quats", "opacity", "colors", "pose"):
        a, b = out["tc"][k].ravel(), out["plain"][k].ravel()
        assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b), k
