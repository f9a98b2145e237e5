"""Failure detection on the GPU without a fault: a bounded device wait that runs out.

The tensor-core feature kernels (forward and adjoint) are warp-specialised:
every role waits on mbarriers with a bound of 1 s of %globaltimer, after which
it ORs GS_ERR_TIMEOUT into the status word and raises its CTA's abort word, on
which every other role's waits return; each role then waits for what it has
issued and the CTA frees its tensor memory. The test hook
gs_test_hold_tc_producer keeps the producer warps idle (a flag that nothing
sets: no stage is ever filled, no product is issued), so the waits run out and
the launch returns with the flag set. The launches after it, on the same
context, must give the result of a normal run again (tensor memory was freed,
nothing was left in flight).
"""
import time

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _t(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def test_tc_forward_wait_runs_out_and_the_context_survives(gs, sg):
    cam = sg.identity_camera(96, 64, 76.8).as_f32()
    sc = sg.frustum_scene(21, 1500, cam, 128)
    means, scales, quats, opac, cols = (_t(x) for x in (sc.means, sc.scales, sc.quats, sc.opacity, sc.colors))
    feats = _t(sc.feats, torch.bfloat16)
    proj = gs.project(cam, means, scales, quats, opac)
    srt = gs.bin_sort(cam, proj, max(int(proj["n_instances"].item()), 1))
    flags = gs.GS_FEAT_ON | gs.GS_FEAT_TENSOR_CORE

    def render():
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        out = gs.render_fwd(cam, proj, srt, cols, feats, flags=flags, layout=gs.GS_LAYOUT_HWC, status=status)
        torch.cuda.synchronize()
        return out, int(status.item())

    ref, s0 = render()
    assert s0 == 0
    ref = {k: v.clone() for k, v in ref.items()}

    gs.hold_tc_producer(True)
    try:
        t0 = time.perf_counter()
        held, s1 = render()
        dt = time.perf_counter() - t0
    finally:
        gs.hold_tc_producer(False)
    assert s1 == 1 << gs.GS_ERR_TIMEOUT, gs.status_names(s1)
    assert gs.status_names(s1) == ["bounded wait timed out"]
    # the waits ran to their bound (1 s) and then returned
    assert 0.9 < dt < 60.0, dt
    # the SIMT forward launched before the tensor-core kernel wrote its outputs as usual
    for k in ("rgb", "depth", "alpha", "T_final", "last_idx", "n_contrib"):
        assert torch.equal(held[k], ref[k]), k

    for _ in range(2):
        again, s2 = render()
        assert s2 == 0
        assert torch.equal(again["feat"], ref["feat"])


def test_tc_adjoint_wait_runs_out_and_the_context_survives(gs, sg):
    """The same for the tensor-core feature adjoint, on a 400 x 300 image (950
    half tiles, several per CTA: the copier warp, the staging ring and the copy
    of A into tensor memory are live when the waits run out). The launch
    returns in about 1 s with exactly the timeout flag; the geometry gradients
    of the SIMT adjoint launched before it are as usual; the next adjoints on
    the same context give the feature gradient again (to the rounding of its
    float atomics, whose order varies from run to run)."""
    cam = sg.identity_camera(400, 300, 0.73 * 400).as_f32()
    N = 512
    sc = sg.frustum_scene(36, 6000, cam, N)
    sc.feats = (sc.feats / np.linalg.norm(sc.feats, axis=1, keepdims=True)).astype(np.float32)
    g_rgb, g_d, g_a, g_f = (_t(x) for x in sg.random_linear_functional(37, cam.height, cam.width, N))
    g_f_hwc = g_f.permute(1, 2, 0).contiguous()
    means, scales, quats, opac, cols = (_t(x) for x in (sc.means, sc.scales, sc.quats, sc.opacity, sc.colors))
    feats = _t(sc.feats, torch.bfloat16)
    flags = gs.GS_FEAT_ON | gs.GS_FEAT_TENSOR_CORE
    proj = gs.project(cam, means, scales, quats, opac)
    srt = gs.bin_sort(cam, proj, max(int(proj["n_instances"].item()), 1))
    fw = gs.render_fwd(cam, proj, srt, cols, feats, flags=flags, layout=gs.GS_LAYOUT_HWC, status=srt["status"])
    torch.cuda.synchronize()
    assert int(srt["status"].item()) == 0

    def adjoint():
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        gr = gs.render_bwd(cam, means, scales, quats, cols, feats, proj, srt, fw, g_rgb, g_d, g_a, g_f_hwc,
                           flags=flags, layout=gs.GS_LAYOUT_HWC, status=status)
        torch.cuda.synchronize()
        return {k: v.clone() for k, v in gr.items()}, int(status.item())

    ref, s0 = adjoint()
    assert s0 == 0
    assert ref["feats"].abs().max() > 0

    gs.hold_tc_producer(True)
    try:
        t0 = time.perf_counter()
        held, s1 = adjoint()
        dt = time.perf_counter() - t0
    finally:
        gs.hold_tc_producer(False)
    assert s1 == 1 << gs.GS_ERR_TIMEOUT, gs.status_names(s1)
    assert 0.9 < dt < 60.0, dt
    # float atomics sum in a varying order: compare max-norm-wise, against the
    # largest magnitude of each gradient (a corrupted result is off by O(1))
    def close(a, b):
        return float((a - b).abs().max()) <= 1e-4 * float(b.abs().max()) + 1e-7

    for k in ref:
        if k != "feats":
            assert close(held[k], ref[k]), k

    for _ in range(2):
        again, s2 = adjoint()
        assert s2 == 0
        assert close(again["feats"], ref["feats"])
