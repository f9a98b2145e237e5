"""Pins of the oracle's tracking pieces (Sec. 3.2, Eq. 6): the SE(3) update,
the Adam step on the pose tangent, the edge mask and the tracking loss.

* Exp(delta) against scipy.linalg.expm of the 4x4 twist matrix (an
  independent library routine), on large and tiny angles (the series branch),
  plus the closed forms of a pure rotation about z and a pure translation;
* Adam through properties of the algorithm, not its formula: the first step
  is -lr sign(g), a constant gradient repeats that step, and scaling every
  gradient by c > 0 changes nothing;
* the edge mask on a step image (Sobel 1/8-normalised gives exactly 0.5 on
  the two columns beside the step) and against scipy.ndimage.sobel with
  replicated borders;
* the loss on a 2x2 image worked by hand.
"""
import math

import numpy as np
import pytest

scipy_linalg = pytest.importorskip("scipy.linalg")
scipy_ndimage = pytest.importorskip("scipy.ndimage")

LR_T, LR_R = 1e-2, 3e-2


def _pose(R, t):
    return np.concatenate([np.asarray(R, np.float64).reshape(9), np.asarray(t, np.float64)])


def _rot(axis, ang):
    axis = np.asarray(axis, np.float64) / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return scipy_linalg.expm(ang * K)


def _one_step(ora, pose, g):
    p = pose.copy()
    m, v = np.zeros(6), np.zeros(6)
    conv = ora.pose_update(p, np.asarray(g, np.float64), m, v, 1, LR_T, LR_R)
    return p, conv


def _twist(delta):
    rho, w = delta[:3], delta[3:]
    T = np.zeros((4, 4))
    T[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
    T[:3, 3] = rho
    return T


def test_first_adam_step_is_signed_learning_rate(ora):
    """First step: m_hat = g, v_hat = g^2, so delta = -lr g / (|g| + eps),
    i.e. -lr sign(g) for |g| >> eps, and 0 where g = 0."""
    pose0 = _pose(np.eye(3), [0.1, -0.2, 1.5])
    p, _ = _one_step(ora, pose0, [-3.0, 0, 0, 0, 0, 0])
    assert np.allclose(p[:9], np.eye(3).ravel(), atol=1e-15)
    assert abs(p[9] - (0.1 + LR_T)) < 1e-9 and abs(p[10] + 0.2) < 1e-15 and abs(p[11] - 1.5) < 1e-15


def test_pure_rotation_about_z_closed_form(ora):
    """g = (0,0,0,0,0,-1): delta = (0, 0, 0, 0, 0, lr_r): R <- Rz(lr_r) R,
    t <- Rz(lr_r) t (no translation part when rho = 0)."""
    R0 = _rot([0.3, -0.5, 0.8], 0.7)
    t0 = np.array([0.4, 0.1, -0.3])
    p, _ = _one_step(ora, _pose(R0, t0), [0, 0, 0, 0, 0, -2.0])
    a = LR_R / (1 + 1e-8 / 2.0)
    Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
    assert np.allclose(p[:9].reshape(3, 3), Rz @ R0, atol=1e-14)
    assert np.allclose(p[9:], Rz @ t0, atol=1e-14)


@pytest.mark.parametrize("scale", [1.0, 1e-5])
def test_exp_update_matches_matrix_exponential(ora, scale):
    """T <- expm(twist(delta)) T for a general delta, at ordinary and at tiny
    step sizes (the tiny one takes the series branch)."""
    rng = np.random.default_rng(3)
    R0 = _rot(rng.normal(size=3), 1.1)
    t0 = rng.normal(size=3)
    g = rng.normal(size=6)
    p = _pose(R0, t0)
    m, v = np.zeros(6), np.zeros(6)
    ora.pose_update(p, g, m, v, 1, LR_T * scale, LR_R * scale)
    lr = np.array([LR_T] * 3 + [LR_R] * 3) * scale
    delta = -lr * g / (np.abs(g) + 1e-8)
    T0 = np.eye(4)
    T0[:3, :3], T0[:3, 3] = R0, t0
    T1 = scipy_linalg.expm(_twist(delta)) @ T0
    assert np.allclose(p[:9].reshape(3, 3), T1[:3, :3], atol=1e-13)
    assert np.allclose(p[9:], T1[:3, 3], atol=1e-13)


def test_constant_gradient_repeats_the_step_and_scale_invariance(ora):
    """A constant gradient keeps m_hat = g and v_hat = g^2 at every step,
    so every step equals the first; scaling all gradients by c > 0 leaves the
    steps unchanged (up to eps)."""
    g = np.array([0.5, -2.0, 0.0, 1.0, -0.25, 3.0])
    runs = []
    for c in (1.0, 37.0):
        p = _pose(np.eye(3), np.zeros(3))
        m, v = np.zeros(6), np.zeros(6)
        traj = []
        for step in range(1, 4):
            ora.pose_update(p, c * g, m, v, step, LR_T, LR_R)
            traj.append(p.copy())
        runs.append(np.array(traj))
    p1, p2, p3 = runs[0]
    # translation-only parts compose additively only when theta = 0; compare
    # the rotations instead: R3 = Rd^3 with Rd the first step's rotation
    Rd = p1[:9].reshape(3, 3)
    assert np.allclose(p3[:9].reshape(3, 3), Rd @ Rd @ Rd, atol=1e-13)
    assert np.allclose(runs[0], runs[1], atol=1e-9)


def test_convergence_flag(ora):
    pose0 = _pose(np.eye(3), np.zeros(3))
    p, m, v = pose0.copy(), np.zeros(6), np.zeros(6)
    assert ora.pose_update(p, np.ones(6), m, v, 1, 1e-6, 1e-6, tol_t=1e-4, tol_r=1e-4) == 1
    p, m, v = pose0.copy(), np.zeros(6), np.zeros(6)
    assert ora.pose_update(p, np.ones(6), m, v, 1, 1e-3, 1e-6, tol_t=1e-4, tol_r=1e-4) == 0


def test_edge_mask_step_image(ora):
    """A vertical step 0 -> 1 between columns 7 and 8: the 1/8-normalised
    Sobel gx is exactly 0.5 on columns 7 and 8 and 0 elsewhere, gy = 0; the
    mask holds those two columns for tau < 0.5 and nothing at tau = 0.5
    (strict test)."""
    H, W = 10, 16
    L = np.zeros((H, W), np.float32)
    L[:, 8:] = 1.0
    rgb = np.stack([L, L, L])
    m = ora.edge_mask(rgb, 0.49)
    want = np.zeros((H, W), np.uint8)
    want[:, 7:9] = 1
    assert np.array_equal(m, want)
    assert not ora.edge_mask(rgb, 0.5).any()


def test_edge_mask_against_scipy_sobel(ora):
    """Decisions equal scipy.ndimage.sobel's (mode 'nearest' = replicated
    border) magnitude test wherever the magnitude is not within 1e-5 of the
    threshold."""
    rng = np.random.default_rng(5)
    rgb = rng.uniform(size=(3, 40, 56)).astype(np.float32)
    rgb[:, 10:30, 20:40] += 0.7
    L = rgb.astype(np.float64).sum(0) / 3.0
    gx = scipy_ndimage.sobel(L, axis=1, mode="nearest") / 8.0
    gy = scipy_ndimage.sobel(L, axis=0, mode="nearest") / 8.0
    tau = 0.15
    mag2 = gx * gx + gy * gy
    m = ora.edge_mask(rgb, tau)
    sure = np.abs(mag2 - tau * tau) > 1e-5
    assert np.array_equal(m[sure] != 0, (mag2 > tau * tau)[sure])
    assert 50 < m.sum() < m.size - 50


def test_tracking_loss_two_by_two(ora):
    """Hand-worked Eq. 6 on a 2x2 image, lambda = 0.75, HW = 4:
    colour weight 0.75/12 = 1/16 on pixels with m_v m_e, depth weight
    0.25/4 = 1/16 on pixels with m_v and observed depth > 0."""
    rgb = np.zeros((3, 2, 2))
    gt = np.zeros((3, 2, 2))
    rgb[:, 0, 0] = [0.5, 0.2, 0.2]       # pixel a: visible, edge
    rgb[:, 0, 1] = [0.9, 0.9, 0.9]       # pixel b: visible, not edge
    rgb[:, 1, 0] = [0.3, 0.3, 0.3]       # pixel c: not visible
    depth = np.array([[2.0, 1.0], [4.0, 3.0]])
    gt_depth = np.array([[1.5, 1.0], [0.0, 0.0]])   # d: observed hole
    alpha = np.array([[0.9, 0.8], [0.2, 0.6]])
    me = np.array([[1, 0], [1, 1]], np.uint8)
    loss, g_rgb, g_depth = ora.tracking_grad(rgb, depth, gt, gt_depth, alpha, 0.5, me, 0.75)
    # colour: pixel a (|0.5|+|0.2|+|0.2| = 0.9) and d (0); depth: a (0.5), b (0)
    assert abs(loss - (0.9 / 16 + 0.5 / 16)) < 1e-15
    assert np.allclose(g_rgb[:, 0, 0], [1 / 16] * 3) and not g_rgb[:, 0, 1].any() and not g_rgb[:, 1].any()
    assert g_depth[0, 0] == 1 / 16 and g_depth[0, 1] == 0 and not g_depth[1].any()
