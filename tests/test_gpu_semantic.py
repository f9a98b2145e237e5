"""Semantic supervision and read-out (Sec. 3.3) on the GPU against the oracle.

Bars: the Eq. 9 gradient within 2e-6 / HW per entry and the loss within 1e-5
(fp32 softmax against FP64); the argmax of Eq. 10 and the Eq. 12 labels are
decisions taken on the same binary32 values (the logits replayed with the
kernel's fused multiply-add order), so they are compared exactly; the Eq. 12
probabilities within 1e-5.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _t(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


@pytest.fixture(scope="module")
def rendered(gs, sg):
    """A rendered 16-channel feature map of the small case (CHW) as logits."""
    sc, cam = sg.small_case(seed=8)
    cam = cam.as_f32()
    ras = gs.Rasterizer(sc.P, cam.width, cam.height, N=16)
    args = tuple(_t(x) for x in (sc.means, sc.scales, sc.quats, sc.opacity, sc.colors, sc.feats))
    ras.ensure_capacity(cam, *args[:4])
    fw = ras.forward(cam, *args)
    torch.cuda.synchronize()
    return fw["feat"].clone() * 4.0  # sharper logits


@pytest.mark.parametrize("hwc", [False, True])
def test_semantic_ce_matches_oracle(gs, ora, rendered, hwc):
    F = rendered
    N, H, W = F.shape
    rng = np.random.default_rng(11)
    labels = rng.integers(-1, N, size=(H, W)).astype(np.int32)
    layout = gs.GS_LAYOUT_HWC if hwc else gs.GS_LAYOUT_CHW
    Fl = F.permute(1, 2, 0).contiguous() if hwc else F
    loss = torch.zeros(1, device="cuda")
    g = gs.semantic_ce_grad(Fl, _t(labels, torch.int32), layout=layout, loss=loss)
    torch.cuda.synchronize()
    want_loss, want = ora.semantic_ce(Fl.cpu().numpy(), labels, hwc=hwc)
    assert abs(loss.item() - want_loss) <= 1e-5 * want_loss
    assert np.abs(g.cpu().numpy() - want).max() <= 2e-6 / (H * W)
    ign = labels < 0
    gg = g.cpu().numpy()
    assert not (gg[ign] if hwc else gg[:, ign]).any()


def test_argmax_labels_exact(gs, ora, rendered):
    F = rendered
    got = gs.argmax_labels(F)
    got_hwc = gs.argmax_labels(F.permute(1, 2, 0).contiguous(), layout=gs.GS_LAYOUT_HWC)
    torch.cuda.synchronize()
    want = ora.argmax_labels(F.cpu().numpy())
    assert np.array_equal(got.cpu().numpy(), want) and np.array_equal(got_hwc.cpu().numpy(), want)
    assert len(np.unique(want)) > 4


@pytest.mark.parametrize("L", [5, 16, 33, 64])
def test_label_probs_matches_oracle(gs, ora, L):
    rng = np.random.default_rng(20 + L)
    M, npix = 512, 3001
    f = rng.normal(size=(npix, M)).astype(np.float32)
    q = (rng.normal(size=(L, M)) / np.sqrt(M) * 3).astype(np.float32)
    probs, labels = gs.label_probs(_t(f), _t(q))
    torch.cuda.synchronize()
    z = ora.label_logits_b32(f, q)
    assert np.array_equal(labels.cpu().numpy(), np.argmax(z, axis=1))
    want = ora.label_probs(f, q)
    assert np.abs(probs.cpu().numpy() - want).max() < 1e-5
    assert np.abs(probs.cpu().numpy().sum(1) - 1).max() < 1e-5
    _, lab_only = gs.label_probs(_t(f), _t(q), probs=False)
    assert torch.equal(lab_only, labels)
