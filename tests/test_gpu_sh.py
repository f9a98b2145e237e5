"""Spherical-harmonic colour (Sec. 3.1) on the GPU against the oracle.

Bars: colours within 2e-6 (fp32 evaluation of O(1) sums); the adjoint
normwise within 1e-5 per output class (d_sh, d_means, d_pose), the classes
accumulated in fp32 over thousands of Gaussians; degrees 0 to 3, a ragged
count, some clamped channels, the pose given on the host and on the device.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", torch.float32)


@pytest.mark.parametrize("degree", [0, 1, 2, 3])
@pytest.mark.parametrize("device_pose", [False, True])
def test_sh_colors_and_adjoint_match_oracle(gs, ora, sg, degree, device_pose):
    rng = np.random.default_rng(40 + degree)
    P, K = 5003, (degree + 1) ** 2
    cam = sg.room_trajectory(17)
    sc = sg.room_scene(3, P, 0)
    means = sc.means.astype(np.float32)
    sh = (rng.normal(size=(P, K, 3)) * 0.4).astype(np.float32)
    sh[:, 0] += 1.2
    sh[::97, 0, 1] = -3.0  # some clamped channels
    camf = cam.as_f32()
    c = camf
    if device_pose:
        c = gs.with_device_pose(camf, _t(np.concatenate([camf.R.reshape(9), camf.t])))
    col = gs.sh_colors(c, _t(means), _t(sh))
    G = rng.normal(size=(P, 3)).astype(np.float32)
    d_sh = torch.zeros(P, K, 3, device="cuda")
    d_means = torch.zeros(P, 3, device="cuda")
    d_pose = torch.zeros(6, device="cuda")
    gs.sh_colors_bwd(c, _t(means), _t(sh), _t(G), d_sh=d_sh, d_means=d_means, d_pose=d_pose)
    torch.cuda.synchronize()
    want = ora.sh_colors(camf, means, sh)
    assert np.abs(col.cpu().numpy() - want).max() < 2e-6
    assert (want == 0).any()
    w_sh, w_means, w_pose = ora.sh_colors_bwd(camf, means, sh, G)
    rel = lambda a, b: np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
    assert rel(d_sh.cpu().numpy(), w_sh) < 1e-5
    if degree > 0:
        assert rel(d_means.cpu().numpy(), w_means) < 1e-5
        assert rel(d_pose.cpu().numpy(), w_pose) < 1e-5 and not d_pose[3:].any()
    else:
        assert not d_means.any() and not d_pose.any()
