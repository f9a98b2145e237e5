"""Camera tracking of Sec. 3.2 on the library's kernels.

With the Gaussians frozen, the frame is rendered at the current pose
estimate; the first render's opacity gives the visibility mask m_v and the
observed image's gradient the edge mask m_e (gs_edge_mask); each iteration
renders (gs_project, gs_bin_sort, gs_tile_order, gs_render_fwd), forms the
cotangents of Eq. 6 as sign words with their two weights
(gs_tracking_loss_signs), back-propagates to the pose tangent only
(gs_render_bwd_l1 with the Gaussian gradients switched off) and updates the
pose on the device (gs_pose_update: Adam, then T <- Exp(delta) T). The pose
lives in a device array that the camera struct points to, so an iteration has
no host round trip; the convergence flag is read every `check_every`
iterations.
"""
from __future__ import annotations

import numpy as np
import torch

from . import GS_FEAT_OFF, Rasterizer, edge_mask, pose_update, tracking_loss_signs, with_device_pose


def pose_array(R, t) -> np.ndarray:
    return np.concatenate([np.asarray(R, np.float64).reshape(9), np.asarray(t, np.float64).reshape(3)]).astype(
        np.float32)


class Tracker:
    """Owns the buffers of one (P, image) shape; `track` refines one frame."""

    def __init__(self, P, width, height, capacity=None, device="cuda", lambda_t=0.9, alpha_min=0.5, tau_edge=0.02,
                 lr_trans=1e-3, lr_rot=3e-3, tol_trans=1e-4, tol_rot=1e-4):
        self.device = torch.device(device)
        self.ras = Rasterizer(P, width, height, N=0, capacity=capacity, device=device, flags=GS_FEAT_OFF)
        self.W, self.H = width, height
        self.opts = dict(lambda_t=lambda_t, alpha_min=alpha_min, tau_edge=tau_edge, lr_trans=lr_trans,
                         lr_rot=lr_rot, tol_trans=tol_trans, tol_rot=tol_rot)
        z = lambda *s, **k: torch.zeros(*s, device=self.device, **k)
        self.pose = z(12)
        self.m, self.v = z(6), z(6)
        self.converged = z(1, dtype=torch.int32)
        self.grads = dict(pose=z(6))
        self.signs = z(height * width, 2, dtype=torch.int32)
        self.alpha_ref = z(height, width)
        self.m_e = z(height, width, dtype=torch.uint8)
        self.loss = z(1)
        self.iterations = 0

    def track(self, cam0, scene, gt_rgb, gt_depth, max_iters=100, check_every=10, losses=None):
        """Refines cam0's pose against the observed (gt_rgb [3,H,W], gt_depth [H,W]); returns the pose
        (12 floats, device) after convergence or max_iters."""
        means, scales, quats, opac, cols = scene
        o = self.opts
        self.pose.copy_(torch.from_numpy(pose_array(cam0.R, cam0.t)))
        self.m.zero_()
        self.v.zero_()
        self.converged.zero_()
        cam = with_device_pose(cam0, self.pose)
        self.ras.ensure_capacity(cam0, means, scales, quats, opac)
        edge_mask(gt_rgb, o["tau_edge"], out=self.m_e)
        it = 0
        for it in range(1, max_iters + 1):
            fw = self.ras.forward(cam, means, scales, quats, opac, cols)
            if it == 1:
                self.alpha_ref.copy_(fw["alpha"])
            self.loss.zero_()
            signs, weights = tracking_loss_signs(fw["rgb"], fw["depth"], gt_rgb, gt_depth, self.alpha_ref, self.m_e,
                                                 lambda_t=o["lambda_t"], alpha_min=o["alpha_min"],
                                                 signs=self.signs, loss=self.loss)
            fw["l1_signs"] = signs
            if losses is not None:
                losses.append(self.loss.clone())
            self.grads["pose"].zero_()
            self.ras.render_pose_grad_l1(cam, means, scales, quats, cols, weights, self.grads)
            pose_update(self.pose, self.grads["pose"], self.m, self.v, it, lr_trans=o["lr_trans"],
                        lr_rot=o["lr_rot"], tol_trans=o["tol_trans"], tol_rot=o["tol_rot"],
                        converged=self.converged)
            if it % check_every == 0 and int(self.converged.item()):
                break
        self.iterations = it
        return self.pose
