"""gs_render_fwd_l1 / gs_render_bwd_l1: an L1 image loss evaluated in the
compositing epilogue, its cotangent signs kept as bits, and the adjoint that
rebuilds the cotangents from them -- against the oracle and against the
two-step path (gs_l1_loss_grad, then gs_render_bwd).

The cotangent signs are decisions on the same binary32 images on both sides,
so the oracle is given exactly the cotangents w sign(pred - target) of the
GPU's forward images; gradients then meet the adjoint's bars (normwise 1e-4,
cosine 0.99999). Against the two-step path, which forms the same cotangents
as floats, the gradients agree to 1e-5 normwise: the fused adjoint multiplies
exact +-1 signs on the tensor cores and applies w after the sum, the two-step
one multiplies w split into bf16 hi + lo (about 2^-16 per term). The loss
agrees to 1e-5 (relative; fp32 sums in another order).
"""
import numpy as np
import pytest
import torch

from tests.test_gpu_parity import GRAD_COS, GRAD_TOL, check_grads, oracle_frame

pytestmark = pytest.mark.gpu

CLASSES = ("means", "scales", "quats", "opacity", "colors", "feats", "pose")


def _t(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def _setup(gs, cam, sc, layout, bg):
    means, scales, quats, opac, cols = (_t(x) for x in (sc.means, sc.scales, sc.quats, sc.opacity, sc.colors))
    feats = _t(sc.feats) if sc.N > 0 else None
    proj = gs.project(cam, means, scales, quats, opac)
    srt = gs.bin_sort(cam, proj, max(int(proj["n_instances"].item()), 1))
    fw = gs.render_fwd(cam, proj, srt, cols, feats, layout=layout, bg=bg, status=srt["status"])
    return (means, scales, quats, cols, feats), proj, srt, fw


def _fused(gs, cam, args, proj, srt, targets, weights, layout, bg):
    """Forward with the L1 loss, then its adjoint; returns (gradients, loss, forward outputs)."""
    means, scales, quats, cols, feats = args
    loss = torch.zeros(1, device="cuda")
    fw = gs.render_fwd(cam, proj, srt, cols, feats, layout=layout, bg=bg, status=srt["status"], l1_targets=targets,
                       l1_weights=weights, l1_loss=loss)
    g = gs.render_bwd_l1(cam, means, scales, quats, cols, feats, proj, srt, fw, weights, layout=layout, bg=bg)
    return g, loss, fw


def _targets(fw, rng, drop=()):
    """Targets near the rendered images, with exact ties on a few pixels."""
    out = {}
    for k in ("rgb", "depth", "feat"):
        if k in drop or k not in fw:
            continue
        x = fw[k]
        t = x + torch.from_numpy(rng.normal(scale=0.05, size=tuple(x.shape)).astype(np.float32)).to(x.device)
        t.view(-1)[::11] = x.view(-1)[::11]
        out[k] = t.contiguous()
    return out


def _two_step(gs, cam, args, proj, srt, fw, targets, weights, layout, bg):
    loss = torch.zeros(1, device="cuda")
    g = {}
    for k, t in targets.items():
        g[k] = gs.l1_loss_grad(fw[k], t, weights[k], loss=loss)
    means, scales, quats, cols, feats = args
    gr = gs.render_bwd(cam, means, scales, quats, cols, feats, proj, srt, fw, g.get("rgb"), g.get("depth"), None,
                       g.get("feat"), layout=layout, bg=bg)
    return gr, loss


def _normwise(a, b):
    a, b = a.double().cpu().numpy().ravel(), b.double().cpu().numpy().ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("case", ["chw_bg", "hwc", "features_off", "rgb_only", "n5_chw", "n8_hwc"])
def test_fused_l1_matches_two_step_and_oracle(gs, ora, sg, case):
    """N = 16, 0, 5 (scalar feature-gradient path, rows not 16-byte aligned)
    and 8 (HWC; vector path for the first two channel groups)."""
    N = {"features_off": 0, "n5_chw": 5, "n8_hwc": 8}.get(case, 16)
    sc, cam = sg.small_case(seed=4, N=N)
    cam = cam.as_f32()
    layout = gs.GS_LAYOUT_HWC if case in ("hwc", "n8_hwc") else gs.GS_LAYOUT_CHW
    bg = (0.1, 0.3, 0.2) if case == "chw_bg" else None
    args, proj, srt, fw = _setup(gs, cam, sc, layout, bg)
    rng = np.random.default_rng(40 + len(case))
    targets = _targets(fw, rng, drop=("depth", "feat") if case == "rgb_only" else ())
    HW = cam.width * cam.height
    weights = {"rgb": 0.9 / (3 * HW), "depth": 0.1 / HW, "feat": 1.0 / (max(N, 1) * HW)}
    got, loss, fw2 = _fused(gs, cam, args, proj, srt, targets, weights, layout, bg)
    ref, ref_loss = _two_step(gs, cam, args, proj, srt, fw, targets, weights, layout, bg)
    torch.cuda.synchronize()
    for k in ("rgb", "depth", "alpha", "T_final", "last_idx", "n_contrib") + (("feat",) if N else ()):
        assert torch.equal(fw2[k], fw[k]), k
    # the sign words: exactly the signs of pred - target, bit c for channel c
    words = fw2["l1_signs"].cpu().numpy().view(np.uint32).reshape(cam.height, cam.width, 2)
    chans = []
    if "feat" in targets:
        f = (fw["feat"] - targets["feat"]).cpu().numpy()
        f = f if layout == gs.GS_LAYOUT_CHW else np.transpose(f, (2, 0, 1))
        chans += [(c, f[c]) for c in range(N)]
    if "rgb" in targets:
        d = (fw["rgb"] - targets["rgb"]).cpu().numpy()
        chans += [(16 + c, d[c]) for c in range(3)]
    if "depth" in targets:
        chans.append((19, (fw["depth"] - targets["depth"]).cpu().numpy()))
    want_nz = np.zeros((cam.height, cam.width), np.uint32)
    want_ng = np.zeros((cam.height, cam.width), np.uint32)
    for bit, d in chans:
        want_nz |= (d != 0).astype(np.uint32) << np.uint32(bit)
        want_ng |= (d < 0).astype(np.uint32) << np.uint32(bit)
    assert np.array_equal(words[..., 0], want_nz) and np.array_equal(words[..., 1], want_ng)
    assert (want_nz != 0).mean() > 0.5 and (want_nz != (want_nz | want_ng)).sum() == 0
    assert abs(loss.item() - ref_loss.item()) <= 1e-5 * ref_loss.item()
    for k in CLASSES:
        if k == "feats" and N == 0:
            continue
        assert _normwise(got[k], ref[k]) <= 1e-5, k
    # the oracle, given the same cotangents
    cot = []
    for k in ("rgb", "depth", "feat"):
        if k not in targets:
            cot.append(None)
            continue
        d = fw[k].cpu().numpy() - targets[k].cpu().numpy()
        c = (np.sign(d) * np.float32(weights[k])).astype(np.float64)
        if k == "feat" and layout == gs.GS_LAYOUT_HWC:
            c = np.transpose(c, (2, 0, 1))
        cot.append(c)
    o = oracle_frame(ora, cam, sc, bg=bg or (0.0, 0.0, 0.0), grads=(cot[0], cot[1], None, cot[2]))
    gg = {k: v.cpu().numpy() for k, v in got.items()}
    # (no feature term: the feature gradient is zero on both sides)
    check_grads(gg, o["grads"], [k for k in CLASSES if not (k == "feats" and "feat" not in targets)], GRAD_TOL,
                GRAD_COS)
    if "feat" not in targets and N > 0:
        assert not gg["feats"].any()


def test_fused_l1_room_frame(gs, sg):
    """The benchmark's launch shape: 300,000 Gaussians at 1200x680, N = 16."""
    sc, _ = sg.room_case()
    cam = sg.room_trajectory(11).as_f32()
    args, proj, srt, fw = _setup(gs, cam, sc, gs.GS_LAYOUT_CHW, None)
    targets = _targets(fw, np.random.default_rng(5))
    HW = cam.width * cam.height
    weights = {"rgb": 1.0 / (3 * HW), "depth": 1.0 / HW, "feat": 1.0 / (16 * HW)}
    got, loss, _ = _fused(gs, cam, args, proj, srt, targets, weights, gs.GS_LAYOUT_CHW, None)
    ref, ref_loss = _two_step(gs, cam, args, proj, srt, fw, targets, weights, gs.GS_LAYOUT_CHW, None)
    torch.cuda.synchronize()
    assert int(srt["status"].item()) == 0
    assert abs(loss.item() - ref_loss.item()) <= 1e-5 * ref_loss.item()
    for k in CLASSES:
        assert _normwise(got[k], ref[k]) <= 1e-5, k


def test_fused_l1_rejects_unsupported(gs, sg):
    """More than 16 feature channels (the chunked SIMT form):
    GS_ERR_UNSUPPORTED from both calls, nothing launched."""
    sc, cam = sg.small_case(seed=5, N=32)
    cam = cam.as_f32()
    args, proj, srt, fw = _setup(gs, cam, sc, gs.GS_LAYOUT_CHW, None)
    means, scales, quats, cols, feats = args
    targets = {"rgb": fw["rgb"].clone()}
    with pytest.raises(gs.GsffError):
        gs.render_fwd(cam, proj, srt, cols, feats, l1_targets=targets, l1_weights={"rgb": 1.0})
    fw["l1_signs"] = torch.zeros(cam.height * cam.width, 2, dtype=torch.int32, device="cuda")
    with pytest.raises(gs.GsffError):
        gs.render_bwd_l1(cam, means, scales, quats, cols, feats, proj, srt, fw, {"rgb": 1.0})


@pytest.mark.parametrize("case", ["chw_bg", "hwc", "features_off", "rgb_only", "n5_chw", "n8_hwc", "room",
                                  "ragged_chw", "ragged_hwc"])
def test_separate_l1_pass_equals_fused_epilogue(gs, sg, case):
    """gs_l1_signs over a plain forward's images writes the fused forward's
    sign words bit for bit (the same binary32 differences) and the same loss
    to 1e-5 (fp32 sums in another order); the adjoint from its words then
    equals the fused pair's to 1e-5 normwise: the same arithmetic, but the
    per-tile float atomics add in a run-dependent order, and the room frame's
    quaternion gradients are sums with cancellation."""
    N = {"features_off": 0, "n5_chw": 5, "n8_hwc": 8}.get(case, 16)
    if case == "room":
        sc, _ = sg.room_case()
        cam = sg.room_trajectory(11).as_f32()
    elif case.startswith("ragged"):
        # 101 x 37 pixels: an odd pixel count, so the pass takes its scalar path
        cam = sg.identity_camera(101, 37, 45.0).as_f32()
        sc = sg.frustum_scene(78, 900, cam, N)
    else:
        sc, cam = sg.small_case(seed=4, N=N)
        cam = cam.as_f32()
    layout = gs.GS_LAYOUT_HWC if case in ("hwc", "n8_hwc", "ragged_hwc") else gs.GS_LAYOUT_CHW
    bg = (0.1, 0.3, 0.2) if case == "chw_bg" else None
    args, proj, srt, fw = _setup(gs, cam, sc, layout, bg)
    targets = _targets(fw, np.random.default_rng(70 + len(case)), drop=("depth", "feat") if case == "rgb_only" else ())
    HW = cam.width * cam.height
    weights = {"rgb": 0.9 / (3 * HW), "depth": 0.1 / HW, "feat": 1.0 / (max(N, 1) * HW)}
    got, loss, fw2 = _fused(gs, cam, args, proj, srt, targets, weights, layout, bg)
    loss_sep = torch.zeros(1, device="cuda")
    gs.l1_signs(cam, fw, targets, weights, loss_sep, layout=layout)
    means, scales, quats, cols, feats = args
    sep = gs.render_bwd_l1(cam, means, scales, quats, cols, feats, proj, srt, fw, weights, layout=layout, bg=bg)
    torch.cuda.synchronize()
    assert torch.equal(fw["l1_signs"], fw2["l1_signs"])
    assert abs(loss_sep.item() - loss.item()) <= 1e-5 * loss.item()
    for k in CLASSES:
        if k == "feats" and N == 0:
            continue
        assert _normwise(sep[k], got[k]) <= 1e-5, k
