"""Camera tracking (Sec. 3.2, Eq. 6) on the GPU against the oracle, and
what the loop achieves.

Bars: the edge mask and the loss cotangents are decisions and signs taken on
the same binary32 inputs, so they are compared exactly (the cotangent scale
is lambda / (3 H W) rounded to binary32 once); the loss sum within 1e-5;
the pose update (fp32 against FP64, a handful of flops on O(1) values)
within 2e-6; the device pose reproduces the host pose bit for bit.
"""
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _t(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


@pytest.fixture(scope="module")
def room(gs, sg):
    sc, _ = sg.room_case(N=0)
    scene = tuple(_t(x) for x in (sc.means, sc.scales, sc.quats, sc.opacity, sc.colors))
    return sc, scene


def _render(gs, cam, scene, P):
    ras = gs.Rasterizer(P, cam.width, cam.height, N=0)
    ras.ensure_capacity(cam, *scene[:4])
    fw = ras.forward(cam, *scene)
    torch.cuda.synchronize()
    ras.check_status()
    return {k: v.clone() for k, v in fw.items()}


def test_device_pose_equals_host_pose(gs, sg, room):
    """The same R, t given through gs_camera.pose_dev: projection and
    images bit-identical, pose gradient equal up to the order of float
    atomics; the pose-only adjoint gives the full adjoint's pose gradient."""
    sc, scene = room
    cam = sg.room_trajectory(21).as_f32()
    pose = _t(np.concatenate([cam.R.reshape(9), cam.t]).astype(np.float32))
    camd = gs.with_device_pose(cam, pose)
    a = gs.project(cam, *scene[:4])
    b = gs.project(camd, *scene[:4])
    for k in ("uv", "conic_opacity", "depth", "rect", "tiles_touched"):
        assert torch.equal(a[k], b[k]), k
    fa, fb = _render(gs, cam, scene, sc.P), _render(gs, camd, scene, sc.P)
    for k in ("rgb", "depth", "alpha", "last_idx"):
        assert torch.equal(fa[k], fb[k]), k
    g_rgb = torch.randn(3, cam.height, cam.width, device="cuda")
    poses = []
    for c in (cam, camd):
        ras = gs.Rasterizer(sc.P, cam.width, cam.height, N=0)
        ras.ensure_capacity(cam, *scene[:4])
        ras.forward(c, *scene)
        full = ras.backward(c, scene[0], scene[1], scene[2], scene[4], g_rgb=g_rgb)["pose"].clone()
        only = ras.render_pose_grad(c, scene[0], scene[1], scene[2], scene[4], g_rgb, None,
                                    dict(pose=torch.zeros(6, device="cuda")))["pose"]
        torch.cuda.synchronize()
        # the pose tangent sums large terms of both signs over the Gaussians, in
        # atomic order: compare normwise (1e-5), as the other gradient checks do
        assert float(torch.linalg.norm(full - only)) <= 1e-5 * float(torch.linalg.norm(full))
        poses.append(full)
    assert float(torch.linalg.norm(poses[0] - poses[1])) <= 1e-5 * float(torch.linalg.norm(poses[0]))


@pytest.mark.parametrize("tau", [0.005, 0.02, 0.08])
def test_edge_mask_bit_exact(gs, ora, sg, room, tau):
    sc, scene = room
    cam = sg.room_trajectory(33).as_f32()
    rgb = _render(gs, cam, scene, sc.P)["rgb"]
    m = gs.edge_mask(rgb, tau)
    torch.cuda.synchronize()
    want = ora.edge_mask(rgb.cpu().numpy(), tau)
    assert np.array_equal(m.cpu().numpy(), want)
    assert want.sum() > 100 and not want.all()


def test_tracking_loss_grad_matches_oracle(gs, ora, sg, room):
    sc, scene = room
    true = sg.room_trajectory(40)
    est = sg.perturb_pose(true, [0.01, -0.005, 0.008], [0.01, -0.02, 0.005]).as_f32()
    obs = _render(gs, true.as_f32(), scene, sc.P)
    cur = _render(gs, est, scene, sc.P)
    gt_depth = obs["depth"].clone()
    gt_depth[:40] = 0.0  # a band of depth holes
    m_e = gs.edge_mask(obs["rgb"], 0.02)
    lam = float(np.float32(0.9))
    loss = torch.zeros(1, device="cuda")
    g_rgb, g_depth = gs.tracking_loss_grad(cur["rgb"], cur["depth"], obs["rgb"], gt_depth, cur["alpha"], m_e,
                                           lambda_t=lam, alpha_min=0.5, loss=loss)
    torch.cuda.synchronize()
    n = lambda x: x.cpu().numpy()
    L, wr, wd = ora.tracking_grad(n(cur["rgb"]), n(cur["depth"]), n(obs["rgb"]), n(gt_depth), n(cur["alpha"]), 0.5,
                                  n(m_e), lam)
    assert np.array_equal(n(g_rgb), wr.astype(np.float32))
    assert np.array_equal(n(g_depth), wd.astype(np.float32))
    assert abs(loss.item() - L) <= 1e-5 * L
    assert (n(g_rgb) != 0).mean() > 0.01 and (n(g_depth) != 0).mean() > 0.1


def test_pose_update_matches_oracle(gs, ora, sg):
    rng = np.random.default_rng(9)
    cam = sg.room_trajectory(5)
    pose64 = np.concatenate([cam.R.reshape(9), cam.t])
    pose = _t(pose64.astype(np.float32))
    p_ref = pose.cpu().numpy().astype(np.float64)
    m, v = torch.zeros(6, device="cuda"), torch.zeros(6, device="cuda")
    m_ref, v_ref = np.zeros(6), np.zeros(6)
    conv = torch.zeros(1, dtype=torch.int32, device="cuda")
    for step in range(1, 7):
        g = (rng.normal(size=6) * [1, 1, 1, 3, 3, 3]).astype(np.float32)
        if step == 6:
            g *= 0.0  # zero gradient: the moments still move the pose
        gs.pose_update(pose, _t(g), m, v, step, lr_trans=2e-3, lr_rot=5e-3, converged=conv)
        want_conv = ora.pose_update(p_ref, g.astype(np.float64), m_ref, v_ref, step, 2e-3, 5e-3)
        torch.cuda.synchronize()
        assert np.abs(pose.cpu().numpy() - p_ref).max() < 2e-6, step
        assert int(conv.item()) == want_conv
    R = pose.cpu().numpy()[:9].reshape(3, 3).astype(np.float64)
    assert np.abs(R @ R.T - np.eye(3)).max() < 1e-5


def _pose_error(pose, true):
    P = pose.cpu().numpy().astype(np.float64)
    R, t = P[:9].reshape(3, 3), P[9:]
    dR = R @ true.R.T
    ang = math.degrees(math.acos(max(-1.0, min(1.0, (np.trace(dR) - 1) / 2))))
    # camera centres: c = -R^T t
    dc = np.linalg.norm(-R.T @ t - (-true.R.T @ true.t))
    return dc, ang


@pytest.mark.parametrize("k", [10, 55])
def test_tracking_recovers_a_perturbed_pose(gs, sg, room, k):
    """The SLAM-frame scene, observed (RGB + depth) at the true pose; the
    tracker starts 1 cm and 1 degree away (a seeded direction) and must end
    within 2 mm and 0.1 degree, with the loss falling."""
    from paper_2504_19409_gb300.tracking import Tracker
    sc, scene = room
    true = sg.room_trajectory(k)
    obs = _render(gs, true.as_f32(), scene, sc.P)
    rng = np.random.default_rng(k)
    d_rho, d_th = rng.normal(size=3), rng.normal(size=3)
    init = sg.perturb_pose(true, 0.01 * d_rho / np.linalg.norm(d_rho),
                           math.radians(1.0) * d_th / np.linalg.norm(d_th)).as_f32()
    tr = Tracker(sc.P, true.width, true.height)
    losses = []
    pose = tr.track(init, scene, obs["rgb"], obs["depth"], max_iters=300, losses=losses)
    torch.cuda.synchronize()
    tr.ras.check_status()
    e0 = _pose_error(_t(np.concatenate([init.R.reshape(9), init.t]).astype(np.float32)), true)
    e1 = _pose_error(pose, true)
    print(f"frame {k}: {tr.iterations} iterations, start {e0[0] * 1e3:.2f} mm {e0[1]:.3f} deg -> "
          f"{e1[0] * 1e3:.3f} mm {e1[1]:.4f} deg")
    assert e0[0] > 0.009 and e0[1] > 0.9
    assert e1[0] < 0.002 and e1[1] < 0.1
    assert losses[-1].item() < 0.2 * losses[0].item()
