"""Per-pair saved state (the transmittance in front of every blended pair)
against the saved T_final / last index that the default adjoint recovers the
transmittance from by division (T_i = T_{i+1} / (1 - alpha_i)).

* gs_render_fwd_pairs: the offsets are the exclusive scan of the forward's
  contributor counts; each pixel's stored transmittances start at 1, do not
  increase, and its last one times (1 - alpha_last), alpha_last in
  [1/255, 0.99], is the forward's T_final;
* gs_render_bwd_pairs with either form of T against the FP64 oracle's
  adjoint (which keeps each pixel's blended list and divides nothing), on the
  500-Gaussian case with N = 64 (coupled) and on a near-opaque case (every
  opacity 0.999 and the scales tripled, so alpha sits at the 0.99 clamp near
  the centres, where a division by 1 - alpha = 0.01 is most sensitive, and
  about 90 % of the pixels end below T = 1e-3): normwise error per gradient
  class <= 1e-4, cosine >= 0.99999.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", torch.float32)


def _frame(gs, cam, sc):
    means, scales, quats, opac, cols, feats = (_t(x) for x in (sc.means, sc.scales, sc.quats, sc.opacity, sc.colors,
                                                               sc.feats))
    proj = gs.project(cam, means, scales, quats, opac)
    srt = gs.bin_sort(cam, proj, max(int(proj["n_instances"].item()), 1))
    fw = gs.render_fwd(cam, proj, srt, cols, feats, status=srt["status"])
    return (means, scales, quats, opac, cols, feats), proj, srt, fw


def test_pair_state_structure(gs, sg):
    sc, cam = sg.small_case(seed=8, P=2000, N=16)
    cam = cam.as_f32()
    _, proj, srt, fw = _frame(gs, cam, sc)
    pairs = gs.render_fwd_pairs(cam, proj, srt, fw, status=srt["status"])
    torch.cuda.synchronize()
    assert int(srt["status"].item()) == 0
    nc = fw["n_contrib"].cpu().numpy().ravel().astype(np.int64)
    off = pairs["pair_off"].cpu().numpy()
    assert np.array_equal(off, np.concatenate([[0], np.cumsum(nc)]))
    T = pairs["pair_T"][:int(off[-1])].cpu().numpy()
    Tf = fw["T_final"].cpu().numpy().ravel()
    starts, ends = off[:-1], off[1:]
    has = nc > 0
    assert has.sum() > 1000
    assert np.all(T[starts[has]] == 1.0)
    d = np.diff(T)
    inner = np.ones(len(T) - 1, bool)
    inner[ends[has][:-1] - 1] = False  # steps across pixel boundaries
    assert np.all(d[inner] <= 0)
    ratio = Tf[has] / T[ends[has] - 1]  # (1 - alpha_last)
    assert np.all(ratio >= 0.01 * (1 - 1e-6)) and np.all(ratio <= (1 - 1 / 255) * (1 + 1e-6))
    # the capacity bound: one pair short flags GS_ERR_CAPACITY and writes only what fits
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    small = gs.render_fwd_pairs(cam, proj, srt, fw, capacity=int(off[-1]) - 1, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) & (1 << gs.GS_ERR_CAPACITY)
    assert int(small["n_pairs"].item()) == off[-1]


def _grads_vs_oracle(gs, ora, cam, sc, coupled):
    tens, proj, srt, fw = _frame(gs, cam, sc)
    means, scales, quats, opac, cols, feats = tens
    from paper_2504_19409_gb300 import scenegen as sg
    cot = tuple(x.astype(np.float32) for x in sg.random_linear_functional(17, cam.height, cam.width, sc.N))
    g_rgb, g_d, g_a, g_f = (_t(x) for x in cot)
    pairs = gs.render_fwd_pairs(cam, proj, srt, fw, status=srt["status"])
    out = {}
    for name, pr in (("division", None), ("stored", pairs)):
        gr = gs.render_bwd_pairs(cam, means, scales, quats, cols, feats, proj, srt, fw, pairs=pr, g_rgb=g_rgb,
                                 g_depth=g_d, g_alpha=g_a, g_feat=g_f, coupled=coupled, status=srt["status"])
        out[name] = {k: v.double().cpu().numpy() for k, v in gr.items()}
    torch.cuda.synchronize()
    assert int(srt["status"].item()) == 0
    pr = ora.project_b32(cam, sc.means, sc.scales, sc.quats, sc.opacity)
    ranges, gids = ora.bin_lists(cam, pr["rect"], pr["depth"])
    c64 = tuple(x.astype(np.float64) for x in cot)
    rb = ora.render_bwd(cam, ranges, gids, pr["uv"], pr["conic"], sc.opacity, sc.colors, pr["depth"], sc.feats, *c64,
                        coupled)
    pb = ora.project_bwd_f64(cam, sc.means, sc.scales, sc.quats, sc.opacity, rb["d_uv"], rb["d_conic"], rb["d_depth"])
    want = dict(means=pb["d_means"], scales=pb["d_scales"], quats=pb["d_quats"], opacity=rb["d_opacity"],
                colors=rb["d_colors"], feats=rb["d_feats"], pose=pb["d_pose"])
    errs = {}
    for name, got in out.items():
        for k, b in want.items():
            a, b = got[k].ravel(), b.ravel()
            nb = np.linalg.norm(b)
            assert nb > 0, k
            errs[(name, k)] = (np.linalg.norm(a - b) / nb, float(a @ b / (np.linalg.norm(a) * nb)))
    return errs, fw


@pytest.mark.parametrize("coupled", [False, True])
def test_both_transmittance_forms_match_oracle(gs, ora, sg, coupled):
    sc, cam = sg.fd_case()
    errs, _ = _grads_vs_oracle(gs, ora, cam.as_f32(), sc, coupled)
    for (name, k), (rel, cos) in errs.items():
        assert rel <= 1e-4 and cos >= 0.99999, (name, k, rel, cos)


def test_near_opaque_case(gs, ora, sg):
    sc, cam = sg.fd_case(seed=9)
    sc.opacity[:] = np.float32(0.999)
    sc.scales[:] = (3 * sc.scales).astype(np.float32)
    errs, fw = _grads_vs_oracle(gs, ora, cam.as_f32(), sc, coupled=True)
    # the case is what it claims: many pixels saturate within a few layers
    nc = fw["n_contrib"].cpu().numpy()
    Tf = fw["T_final"].cpu().numpy()
    assert (Tf[nc > 0] < 1e-3).mean() > 0.8
    for (name, k), (rel, cos) in errs.items():
        assert rel <= 1e-4 and cos >= 0.99999, (name, k, rel, cos)
