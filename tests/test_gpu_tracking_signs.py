"""gs_tracking_loss_signs: Eq. 6's cotangents as sign words. The words are
exactly the signs of gs_tracking_loss_grad's float cotangents (the same
binary32 differences and masks), the loss is the same to 1e-5, and the pose
gradient through gs_render_bwd_l1 equals the one of gs_render_bwd on the
float cotangents to 1e-5 normwise (the L1 adjoint multiplies the exact signs
and applies the weight after the sum)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_tracking_sign_words_match_float_cotangents(gs, sg):
    sc, _ = sg.room_case()
    cam_true = sg.room_trajectory(5).as_f32()
    cam = sg.room_trajectory(6).as_f32()  # a nearby pose: the residual is not zero
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    means, scales, quats, opac, cols = (t(x) for x in (sc.means, sc.scales, sc.quats, sc.opacity, sc.colors))
    ras = gs.Rasterizer(sc.means.shape[0], cam.width, cam.height, N=0, flags=gs.GS_FEAT_OFF)
    ras.ensure_capacity(cam_true, means, scales, quats, opac)
    gt = ras.forward(cam_true, means, scales, quats, opac, cols)
    gt_rgb, gt_depth = gt["rgb"].clone(), gt["depth"].clone()
    m_e = gs.edge_mask(gt_rgb, 0.02)
    ras.ensure_capacity(cam, means, scales, quats, opac)
    fw = ras.forward(cam, means, scales, quats, opac, cols)
    alpha_ref = fw["alpha"].clone()
    loss_f, loss_s = torch.zeros(1, device="cuda"), torch.zeros(1, device="cuda")
    g_rgb, g_depth = gs.tracking_loss_grad(fw["rgb"], fw["depth"], gt_rgb, gt_depth, alpha_ref, m_e, loss=loss_f)
    signs, weights = gs.tracking_loss_signs(fw["rgb"], fw["depth"], gt_rgb, gt_depth, alpha_ref, m_e, loss=loss_s)
    torch.cuda.synchronize()
    words = signs.cpu().numpy().view(np.uint32)
    gr, gd = g_rgb.cpu().numpy(), g_depth.cpu().numpy().ravel()
    want_nz = np.zeros(words.shape[0], np.uint32)
    want_ng = np.zeros(words.shape[0], np.uint32)
    for bit, g in [(16 + c, gr[c].ravel()) for c in range(3)] + [(19, gd)]:
        want_nz |= (g != 0).astype(np.uint32) << np.uint32(bit)
        want_ng |= (g < 0).astype(np.uint32) << np.uint32(bit)
    assert np.array_equal(words[:, 0], want_nz) and np.array_equal(words[:, 1], want_ng)
    assert (want_nz != 0).mean() > 0.05
    # the weights are the float cotangents' magnitudes
    assert np.all(np.abs(gr[gr != 0]) == np.float32(weights["rgb"]))
    assert np.all(np.abs(gd[gd != 0]) == np.float32(weights["depth"]))
    assert abs(loss_s.item() - loss_f.item()) <= 1e-5 * loss_f.item()
    a = dict(pose=torch.zeros(6, device="cuda"))
    ras.render_pose_grad(cam, means, scales, quats, cols, g_rgb, g_depth, a)
    fw["l1_signs"] = signs
    b = dict(pose=torch.zeros(6, device="cuda"))
    ras.render_pose_grad_l1(cam, means, scales, quats, cols, weights, b)
    torch.cuda.synchronize()
    x, y = b["pose"].double(), a["pose"].double()
    assert float(y.norm()) > 0
    assert float((x - y).norm() / y.norm()) <= 1e-5
