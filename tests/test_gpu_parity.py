"""CUDA path vs the FP64 oracle, through the C ABI.

Bars (stated here and derived in the design notes):
* discrete outputs -- tile rectangles, touched counts, depth keys, per-tile
  sorted lists, contributor counts and last indices -- bit-exact; contributor
  counts are compared at every pixel whose oracle decision margins all exceed
  1e-5 (relative; the GPU's fp32 alpha and T carry at most a few 1e-6 of
  relative error after ~50 blends). Pixels inside that band must number
  <= max(3, 1e-3 HW): with ~100-200 alpha/T decisions per pixel about 2.5e-4
  of the pixels of these scenes sit within 1e-5 of a threshold;
* fp32 images: |gpu - ora| <= 1e-5 max(|ora|, s), s = 1 for RGB / alpha,
  max depth for depth, RMS of the features for features;
* gradients: normwise relative error <= 1e-4 per parameter class and cosine
  >= 0.99999.
The oracle composites in double from the projection's binary32 replay, so
both sides start from identical per-Gaussian records.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

MARGIN = 1e-5
MAX_AMBIGUOUS = 1e-3
IMG_TOL = 1e-5
GRAD_TOL = 1e-4
GRAD_COS = 0.99999


def _t(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def gpu_frame(gs, cam, sc, N=None, layout=0, bg=None, feat_bf16=False, grads=None, coupled=False, capacity=None,
              visible=False):
    """Run project -> bin_sort -> fwd (-> bwd) on the GPU; returns numpy dicts."""
    means, scales, quats, opac, cols = (_t(x) for x in (sc.means, sc.scales, sc.quats, sc.opacity, sc.colors))
    feats = None
    if sc.N > 0 and N != 0:
        feats = _t(sc.feats, torch.bfloat16 if feat_bf16 else torch.float32)
    proj = gs.project(cam, means, scales, quats, opac)
    I = int(proj["n_instances"].item())
    srt = gs.bin_sort(cam, proj, capacity or max(I, 1))
    vis = torch.zeros(sc.P, dtype=torch.uint8, device="cuda") if visible else None
    fw = gs.render_fwd(cam, proj, srt, cols, feats, layout=layout, bg=bg, status=srt["status"], visible=vis)
    out = dict(I=I, proj={k: v.cpu().numpy() for k, v in proj.items()},
               sort={k: v.cpu().numpy() for k, v in srt.items()}, fwd={k: v.cpu().numpy() for k, v in fw.items()})
    if visible:
        out["visible"] = vis.cpu().numpy()
    if grads is not None:
        g_rgb, g_d, g_a, g_f = (None if x is None else _t(x) for x in grads)
        if g_f is not None and layout == 1:
            g_f = g_f.permute(1, 2, 0).contiguous()
        gr = gs.render_bwd(cam, means, scales, quats, cols, feats, proj, srt, fw, g_rgb, g_d, g_a, g_f, layout=layout,
                           bg=bg, coupled=coupled, status=srt["status"])
        out["grads"] = {k: v.cpu().numpy() for k, v in gr.items()}
    torch.cuda.synchronize()
    out["status"] = int(srt["status"].item())
    return out


def oracle_frame(ora, cam, sc, bg=(0.0, 0.0, 0.0), grads=None, coupled=False, feats=None):
    feats = sc.feats if feats is None else feats
    pr = ora.project_b32(cam, sc.means, sc.scales, sc.quats, sc.opacity)
    ranges, gids = ora.bin_lists(cam, pr["rect"], pr["depth"])
    fw = ora.render_fwd(cam, ranges, gids, pr["uv"], pr["conic"], sc.opacity, sc.colors, pr["depth"],
                        feats if feats.shape[1] > 0 else None, bg)
    out = dict(proj=pr, ranges=ranges, gids=gids, fwd=fw)
    if grads is not None:
        g_rgb, g_d, g_a, g_f = grads
        rb = ora.render_bwd(cam, ranges, gids, pr["uv"], pr["conic"], sc.opacity, sc.colors, pr["depth"],
                            feats if feats.shape[1] > 0 else None, g_rgb, g_d, g_a, g_f, coupled, bg)
        pb = ora.project_bwd_f64(cam, sc.means, sc.scales, sc.quats, sc.opacity, rb["d_uv"], rb["d_conic"],
                                 rb["d_depth"])
        out["grads"] = dict(means=pb["d_means"], scales=pb["d_scales"], quats=pb["d_quats"], opacity=rb["d_opacity"],
                            colors=rb["d_colors"], feats=rb["d_feats"], pose=pb["d_pose"])
    return out


def check_projection(gp, op):
    assert np.array_equal(gp["tiles_touched"], op["touched"])
    assert np.array_equal(gp["rect"], op["rect"])
    assert np.array_equal(gp["uv"].view(np.uint32), op["uv"].view(np.uint32))
    assert np.array_equal(gp["conic_opacity"][:, :3].view(np.uint32), op["conic"].view(np.uint32))
    assert np.array_equal(gp["depth"].view(np.uint32), op["depth"].view(np.uint32))


def check_lists(cam, g, o):
    I = g["I"]
    assert I == len(o["gids"])
    assert np.array_equal(g["sort"]["tile_ranges"], o["ranges"])
    assert np.array_equal(g["sort"]["gids"][:I], o["gids"])
    keys = g["sort"]["keys"][:I].view(np.uint64)
    assert np.all(np.diff(keys.astype(np.float64)) >= 0) or np.all(keys[1:] >= keys[:-1])


def check_images(g, o, N, layout=0, tol=IMG_TOL, feats=None):
    fo, fg = o["fwd"], g["fwd"]
    HW = fo["T_final"].size
    ok = fo["margin"] > MARGIN
    assert (~ok).sum() <= max(3, int(MAX_AMBIGUOUS * HW)), (~ok).sum()
    assert np.array_equal(fg["n_contrib"][ok], fo["n_contrib"][ok])
    assert np.array_equal(fg["last_idx"][ok], fo["last_idx"][ok])

    def close(a, b, s):
        err = np.abs(a - b) / np.maximum(np.abs(b), s)
        return err.max() if err.size else 0.0

    assert close(fg["rgb"][:, ok], fo["rgb"][:, ok], 1.0) <= tol
    assert close(fg["alpha"][ok], fo["alpha"][ok], 1.0) <= tol
    assert close(fg["T_final"][ok], fo["T_final"][ok], 1.0) <= tol
    assert close(fg["depth"][ok], fo["depth"][ok], max(fo["depth"].max(), 1e-6)) <= tol
    if N > 0:
        gf = fg["feat"] if layout == 0 else np.transpose(fg["feat"], (2, 0, 1))
        s = float(np.sqrt((np.asarray(feats, np.float64) ** 2).mean())) if feats is not None else 1.0
        assert close(gf[:, ok], fo["feat"][:, ok], s) <= tol


def check_grads(gg, og, classes, tol=GRAD_TOL, cos=GRAD_COS):
    for k in classes:
        a, b = gg[k].astype(np.float64).ravel(), og[k].ravel()
        nb = np.linalg.norm(b)
        assert nb > 0, k
        rel = np.linalg.norm(a - b) / nb
        c = float(a @ b / (np.linalg.norm(a) * nb))
        assert rel <= tol and c >= cos, (k, rel, c)


# ---- small case: 2,000 Gaussians at 128x96, N=16 --------------------------------

def test_small_case_projection_sort_and_forward(gs, ora, sg):
    sc, cam = sg.small_case()
    cam = cam.as_f32()
    g = gpu_frame(gs, cam, sc)
    o = oracle_frame(ora, cam, sc)
    assert g["status"] == 0
    check_projection(g["proj"], o["proj"])
    check_lists(cam, g, o)
    check_images(g, o, sc.N, feats=sc.feats)


def test_small_case_gradients(gs, ora, sg):
    sc, cam = sg.small_case()
    cam = cam.as_f32()
    cot = tuple(x.astype(np.float32) for x in sg.random_linear_functional(9, cam.height, cam.width, sc.N))
    bg = (0.1, 0.3, 0.2)
    g = gpu_frame(gs, cam, sc, grads=cot, bg=bg)
    o = oracle_frame(ora, cam, sc, bg=bg, grads=tuple(x.astype(np.float64) for x in cot))
    check_images(g, o, sc.N, feats=sc.feats)
    check_grads(g["grads"], o["grads"], ("means", "scales", "quats", "opacity", "colors", "feats", "pose"))


def test_l1_loss_against_second_render(gs, ora, sg):
    """The small workload's loss: mean L1 of RGB, depth and features against
    the render of a second seeded scene; gradients flow to every class."""
    sc, cam = sg.small_case(seed=1)
    tgt, _ = sg.small_case(seed=2)
    cam = cam.as_f32()
    t = oracle_frame(ora, cam, tgt)["fwd"]
    g0 = gpu_frame(gs, cam, sc)["fwd"]
    n = cam.width * cam.height
    pred = [g0["rgb"], g0["depth"], g0["feat"]]
    targ = [t["rgb"], t["depth"], t["feat"]]
    cots = []
    for p_, t_ in zip(pred, targ):
        t32 = t_.astype(np.float32)
        scale = np.float32(1.0 / p_.size)
        loss = torch.zeros(1, device="cuda")
        gr = gs.l1_loss_grad(_t(p_), _t(t32), float(scale), loss=loss)
        want = (np.sign(p_ - t32) * scale).astype(np.float32)
        assert np.array_equal(gr.cpu().numpy(), want)
        ref = float(np.abs(p_.astype(np.float64) - t32).sum()) * float(scale)
        assert abs(loss.item() - ref) <= 1e-4 * max(ref, 1e-6)
        cots.append(gr.cpu().numpy())
    cot = (cots[0], cots[1], None, cots[2])
    g = gpu_frame(gs, cam, sc, grads=cot)
    o = oracle_frame(ora, cam, sc, grads=tuple(None if x is None else x.astype(np.float64) for x in cot))
    check_grads(g["grads"], o["grads"], ("means", "scales", "quats", "opacity", "colors", "feats", "pose"))


@pytest.mark.parametrize("offset,n", [(0, 1003), (1, 1003), (0, 4096), (3, 5)])
def test_l1_loss_vector_and_scalar_paths(gs, offset, n):
    """gs_l1_loss_grad on 16-byte-aligned arrays (float4 body + scalar tail)
    and on arrays shifted by `offset` floats (scalar path): the same signs,
    exactly, and the same loss."""
    rng = np.random.default_rng(7 + offset + n)
    p_ = rng.normal(size=n + offset).astype(np.float32)
    t_ = rng.normal(size=n + offset).astype(np.float32)
    t_[offset::7] = p_[offset::7]  # exact ties give a zero gradient
    P, T = _t(p_), _t(t_)
    G = torch.full((n + offset,), 5.0, device="cuda")
    loss = torch.zeros(1, device="cuda")
    scale = 0.25
    gs.l1_loss_grad(P[offset:], T[offset:], scale, grad=G[offset:], loss=loss)
    torch.cuda.synchronize()
    want = (np.sign(p_[offset:] - t_[offset:]) * np.float32(scale)).astype(np.float32)
    got = G.cpu().numpy()
    assert np.array_equal(got[offset:], want)
    assert (got[:offset] == 5.0).all()
    ref = float(np.abs(p_[offset:].astype(np.float64) - t_[offset:]).sum()) * scale
    assert abs(loss.item() - ref) <= 1e-5 * max(ref, 1e-6)


# ---- differentiation case: 500 Gaussians at 64x48, N=64 (two 32-channel chunks) --

@pytest.mark.parametrize("coupled", [False, True])
def test_fd_case_gradients_chunked_features(gs, ora, sg, coupled):
    sc, cam = sg.fd_case()
    cam = cam.as_f32()
    cot = tuple(x.astype(np.float32) for x in sg.random_linear_functional(105, cam.height, cam.width, sc.N))
    g = gpu_frame(gs, cam, sc, grads=cot, coupled=coupled)
    o = oracle_frame(ora, cam, sc, grads=tuple(x.astype(np.float64) for x in cot), coupled=coupled)
    check_projection(g["proj"], o["proj"])
    check_lists(cam, g, o)
    check_images(g, o, sc.N, feats=sc.feats)
    check_grads(g["grads"], o["grads"], ("means", "scales", "quats", "opacity", "colors", "feats", "pose"))


def test_hwc_layout_and_bf16_features(gs, ora, sg):
    sc, cam = sg.fd_case(seed=8, N=48)
    cam = cam.as_f32()
    f_bf = torch.from_numpy(sc.feats).to(torch.bfloat16).float().numpy().astype(np.float64)
    cot = tuple(x.astype(np.float32) for x in sg.random_linear_functional(108, cam.height, cam.width, sc.N))
    g = gpu_frame(gs, cam, sc, layout=1, feat_bf16=True, grads=cot)
    o = oracle_frame(ora, cam, sc, feats=f_bf, grads=tuple(x.astype(np.float64) for x in cot))
    check_images(g, o, sc.N, layout=1, feats=sc.feats)
    check_grads(g["grads"], o["grads"], ("means", "opacity", "feats", "pose"))


@pytest.mark.parametrize("N,layout,bf16", [(5, 0, False), (12, 1, True)])
def test_partial_feature_counts(gs, ora, sg, N, layout, bf16):
    """Fewer than 16 channels on the N <= 16 kernels: 5 (rows not 16-byte
    aligned, scalar feature-gradient adds) and 12 in HWC layout from bf16
    features."""
    sc, cam = sg.small_case(seed=6, N=N)
    cam = cam.as_f32()
    feats = torch.from_numpy(sc.feats).to(torch.bfloat16).float().numpy().astype(np.float64) if bf16 else None
    cot = tuple(x.astype(np.float32) for x in sg.random_linear_functional(60 + N, cam.height, cam.width, N))
    g = gpu_frame(gs, cam, sc, layout=layout, feat_bf16=bf16, grads=cot)
    o = oracle_frame(ora, cam, sc, feats=feats, grads=tuple(x.astype(np.float64) for x in cot))
    check_images(g, o, N, layout=layout, feats=sc.feats)
    check_grads(g["grads"], o["grads"], ("means", "scales", "quats", "opacity", "colors", "feats", "pose"))


# ---- edge cases -----------------------------------------------------------------------

def test_ragged_image_and_features_off(gs, ora, sg):
    """Width and height not multiples of 16 (ragged last tile row/column),
    features off (Eq. 3 'otherwise')."""
    cam = sg.identity_camera(100, 37, 45.0).as_f32()
    sc = sg.frustum_scene(77, 900, cam, 0)
    cot = tuple(x.astype(np.float32) for x in sg.random_linear_functional(77, cam.height, cam.width, 0))
    g = gpu_frame(gs, cam, sc, grads=cot[:3] + (None,))
    o = oracle_frame(ora, cam, sc, grads=tuple(x.astype(np.float64) for x in cot[:3]) + (None,))
    check_projection(g["proj"], o["proj"])
    check_lists(cam, g, o)
    check_images(g, o, 0)
    assert "feat" not in g["fwd"]
    check_grads(g["grads"], o["grads"], ("means", "scales", "quats", "opacity", "colors", "pose"))


def test_empty_and_fully_culled_scenes(gs, ora, sg):
    cam = sg.identity_camera(64, 48, 50.0).as_f32()
    sc = sg.frustum_scene(3, 50, cam, 4)
    sc.means[:, 2] = -1.0          # all behind the camera
    sc.means[0, 0] = np.nan        # and one non-finite
    g = gpu_frame(gs, cam, sc, capacity=16)
    assert g["I"] == 0 and g["status"] == 0
    assert (g["fwd"]["n_contrib"] == 0).all() and (g["fwd"]["alpha"] == 0).all()
    assert np.array_equal(g["sort"]["tile_ranges"], np.zeros_like(g["sort"]["tile_ranges"]))
    empty = sg.frustum_scene(3, 0, cam, 4)
    g0 = gpu_frame(gs, cam, empty, capacity=16)
    assert g0["I"] == 0 and (g0["fwd"]["T_final"] == 1).all()


def test_capacity_overflow_is_flagged(gs, sg):
    sc, cam = sg.small_case(P=500)
    g = gpu_frame(gs, cam.as_f32(), sc, capacity=64)
    assert g["I"] > 64
    assert g["status"] & (1 << gs.GS_ERR_CAPACITY)


def test_non_finite_parameters_are_culled(gs, ora, sg):
    sc, cam = sg.small_case(P=300)
    cam = cam.as_f32()
    sc.scales[5, 1] = np.inf
    sc.quats[7] = 0.0
    sc.opacity[9] = np.nan
    g = gpu_frame(gs, cam, sc)
    o = oracle_frame(ora, cam, sc)
    assert g["proj"]["tiles_touched"][[5, 7, 9]].sum() == 0
    check_projection(g["proj"], o["proj"])
    check_images(g, o, sc.N, feats=sc.feats)


def test_autograd_function_matches_direct_calls(gs, ora, sg):
    sc, cam = sg.small_case(P=800)
    cam = cam.as_f32()
    params = [_t(x).requires_grad_(True) for x in (sc.means, sc.scales, sc.quats, sc.opacity, sc.colors, sc.feats)]
    pose = torch.zeros(6, device="cuda", requires_grad=True)
    rgb, depth, alpha, feat, _, _ = gs.render(*params, pose, cam, bg=(0.2, 0.2, 0.2))
    cot = [torch.from_numpy(x).cuda() for x in sg.random_linear_functional(31, cam.height, cam.width, sc.N)]
    L = (rgb * cot[0]).sum() + (depth * cot[1]).sum() + (alpha * cot[2]).sum() + (feat * cot[3]).sum()
    L.backward()
    o = oracle_frame(ora, cam, sc, bg=(0.2, 0.2, 0.2), grads=tuple(c.cpu().numpy().astype(np.float64) for c in cot))
    got = dict(means=params[0].grad, scales=params[1].grad, quats=params[2].grad, opacity=params[3].grad,
               colors=params[4].grad, feats=params[5].grad, pose=pose.grad)
    check_grads({k: v.cpu().numpy() for k, v in got.items()}, o["grads"], tuple(got))


def test_chunked_512_channel_simt_matches_oracle(gs, ora, sg):
    """The plain fp32 compositing of 512 channels (sixteen 32-channel chunks),
    the reference point for the tensor-core form."""
    cam = sg.identity_camera(96, 64, 60.0).as_f32()
    sc = sg.frustum_scene(12, 1500, cam, 512)
    cot = tuple(x.astype(np.float32) for x in sg.random_linear_functional(12, cam.height, cam.width, 512))
    g = gpu_frame(gs, cam, sc, layout=1, grads=cot)
    o = oracle_frame(ora, cam, sc, grads=tuple(x.astype(np.float64) for x in cot))
    check_images(g, o, 512, layout=1, feats=sc.feats)
    check_grads(g["grads"], o["grads"], ("feats", "means", "pose"))


# ---- SLAM-frame scale (300,000 Gaussians, 1200x680), the benchmark's launch shape ----

@pytest.fixture(scope="module")
def room_frame(gs, ora, sg):
    sc, _ = sg.room_case()
    cam = sg.room_trajectory(7).as_f32()
    cot = tuple(x.astype(np.float32) for x in sg.random_linear_functional(70, cam.height, cam.width, sc.N))
    g = gpu_frame(gs, cam, sc, grads=cot, visible=True)
    o = oracle_frame(ora, cam, sc, grads=tuple(x.astype(np.float64) for x in cot))
    return sc, cam, g, o


def test_room_scale_discrete_outputs_bit_exact(room_frame):
    sc, cam, g, o = room_frame
    assert g["status"] == 0 and g["I"] > 100_000
    check_projection(g["proj"], o["proj"])
    check_lists(cam, g, o)


def test_room_scale_images(room_frame):
    sc, cam, g, o = room_frame
    check_images(g, o, sc.N, feats=sc.feats)
    assert o["fwd"]["n_contrib"].mean() > 3


def test_room_scale_gradients(room_frame):
    sc, cam, g, o = room_frame
    check_grads(g["grads"], o["grads"], ("means", "scales", "quats", "opacity", "colors", "feats", "pose"))


# ---- keyframe visibility (Sec. 3.2, Eq. 5) and co-visibility IoU ----------------

VIS_BAND = 1e-5  # relative distance of the oracle's max T from 0.5 below which a decision is not compared


def check_visibility(ora, cam, sc, g, o, min_each=100):
    maxT = ora.visibility(cam, o["ranges"], o["gids"], o["proj"]["uv"], o["proj"]["conic"], sc.opacity)
    want = maxT > 0.5
    sure = np.abs(maxT - 0.5) > VIS_BAND * 0.5
    assert (~sure).sum() <= max(2, int(1e-4 * sc.P))
    assert np.array_equal(g["visible"][sure] != 0, want[sure]), int(((g["visible"] != 0) != want)[sure].sum())
    assert set(np.unique(g["visible"])) <= {0, 1}
    assert want.sum() >= min_each and ((maxT > 0) & ~want).sum() >= min_each


def test_small_case_visibility(gs, ora, sg):
    """gs_render_fwd's visibility output (blended with T > 0.5 in front)
    against the oracle's per-Gaussian max T: equal wherever the oracle's
    decision is more than 1e-5 (relative) from the threshold."""
    sc, cam = sg.small_case(seed=21)
    cam = cam.as_f32()
    g = gpu_frame(gs, cam, sc, visible=True)
    o = oracle_frame(ora, cam, sc)
    check_visibility(ora, cam, sc, g, o)


def test_room_scale_visibility(ora, room_frame):
    sc, cam, g, o = room_frame
    check_visibility(ora, cam, sc, g, o, min_each=1000)


def test_visibility_iou_counts(gs, sg):
    """gs_visibility_iou against the definition (|a and b|, |a or b|) on the
    visibility of two neighbouring SLAM-trajectory frames, plus the edge
    cases: identical vectors, an empty vector, and P = 0."""
    sc, _ = sg.room_case()
    means, scales, quats, opac, cols = (_t(x) for x in (sc.means, sc.scales, sc.quats, sc.opacity, sc.colors))
    ras = gs.Rasterizer(sc.P, 1200, 680, N=0)
    vis = []
    for k in (7, 12):
        cam = sg.room_trajectory(k).as_f32()
        ras.ensure_capacity(cam, means, scales, quats, opac)
        v = torch.zeros(sc.P, dtype=torch.uint8, device="cuda")
        ras.forward(cam, means, scales, quats, opac, cols, visible=v)
        vis.append(v)
    a, b = (v.cpu().numpy() != 0 for v in vis)
    c = gs.visibility_iou(vis[0], vis[1]).cpu().numpy()
    assert c[0] == int((a & b).sum()) and c[1] == int((a | b).sum())
    assert 0.2 < c[0] / c[1] < 1.0
    c = gs.visibility_iou(vis[0], vis[0]).cpu().numpy()
    assert c[0] == c[1] == int(a.sum())
    z = torch.zeros_like(vis[0])
    c = gs.visibility_iou(z, vis[1]).cpu().numpy()
    assert c[0] == 0 and c[1] == int(b.sum())
    e = torch.zeros(0, dtype=torch.uint8, device="cuda")
    c = gs.visibility_iou(e, e).cpu().numpy()
    assert c[0] == 0 and c[1] == 0
