"""The bounds-checked build and the non-finite scans (the sanitiser
substitutes: compute-sanitizer is not used here).

* gs_count_nonfinite counts NaN and infinite values exactly, over spans with
  odd lengths and starts off a 16-byte boundary;
* Rasterizer.check_finite passes on a clean frame and names a buffer that
  holds a NaN;
* libgsff_checked.so (GSFF_CHECKED=1, run in a child process) renders and
  differentiates the small case bit for bit like libgsff.so with a clean
  status word, and flags GS_ERR_BOUNDS for a Gaussian id past P planted in a
  sorted list (every array is padded past P, so the id stays inside the
  caller's allocations even unchecked).
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("offset,n", [(0, 1000), (1, 4099), (3, 5), (2, 1)])
def test_count_nonfinite_exact(gs, offset, n):
    buf = torch.randn(offset + n + 64, device="cuda")
    x = buf[offset:offset + n]
    want = 0
    for i, v in ((0, float("nan")), (n - 1, float("inf")), (n // 2, float("-inf")), (n // 3, float("nan"))):
        if x[i].isfinite():
            x[i] = v
            want += 1
    buf[offset + n:] = float("nan")  # past the span: not counted
    buf[:offset] = float("nan")
    got = gs.count_nonfinite([x]).item()
    assert got == want


def test_rasterizer_check_finite(gs, sg):
    sc, cam = sg.small_case(seed=2, P=2000, N=16)
    cam = cam.as_f32()
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    m, s, q, o, c, f = (t(x) for x in (sc.means, sc.scales, sc.quats, sc.opacity, sc.colors, sc.feats))
    ras = gs.Rasterizer(sc.P, cam.width, cam.height, N=16)
    ras.ensure_capacity(cam, m, s, q, o)
    fw = ras.forward(cam, m, s, q, o, c, f)
    ras.backward(cam, m, s, q, c, f, g_rgb=torch.ones_like(fw["rgb"]))
    ras.check_finite()
    ras.grads["means"][7, 1] = float("nan")
    with pytest.raises(gs.GsffError, match="gradients"):
        ras.check_finite()


_CHILD = r"""
import ctypes, json, sys
import numpy as np, torch
sys.path.insert(0, @ROOT@)
import paper_2504_19409_gb300 as g
from paper_2504_19409_gb300 import scenegen as sg
assert g.LIB_PATH.endswith(@LIBNAME@), g.LIB_PATH
sc, cam = sg.small_case(seed=2, P=2000, N=16)
cam = cam.as_f32()
t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
m, s, q, o, c, f = (t(x) for x in (sc.means, sc.scales, sc.quats, sc.opacity, sc.colors, sc.feats))
ras = g.Rasterizer(sc.P, cam.width, cam.height, N=16)
ras.ensure_capacity(cam, m, s, q, o)
fw = ras.forward(cam, m, s, q, o, c, f)
cot = [t(x.astype(np.float32)) for x in sg.random_linear_functional(3, cam.height, cam.width, 16)]
gr = ras.backward(cam, m, s, q, c, f, *cot)
torch.cuda.synchronize()
res = {"status": int(ras.status.item())}
np.savez(@OUT@, **{"fwd_" + k: v.cpu().numpy() for k, v in fw.items()}, **{"grad_" + k: v.cpu().numpy() for k, v in gr.items()})
if @PLANT@:
    # the same render with one planted id past P; every array holds P + 64 rows
    P = sc.P
    pad = lambda x, n: torch.cat([x, torch.zeros((64,) + tuple(x.shape[1:]), device="cuda", dtype=x.dtype)]).contiguous()
    uv, co, dp = (pad(ras.proj[k], 64) for k in ("uv", "conic_opacity", "depth"))
    cl, fe = pad(c, 64), pad(f, 64)
    gids = ras.sort["gids"].clone()
    rg = ras.sort["tile_ranges"].cpu().numpy()
    t0 = int(np.argmax(rg[:, 1] - rg[:, 0]))
    gids[int(rg[t0, 0]) + 3] = P + 7
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = {k: torch.empty_like(v) for k, v in fw.items()}
    bgc = (ctypes.c_float * 3)(0.0, 0.0, 0.0)
    cs = g.camera_struct(cam)
    P_ = g._ptr
    code = g.lib().gs_render_fwd(ctypes.byref(cs), P, P_(ras.sort["tile_ranges"]), None, P_(gids), None, P_(uv), P_(co),
                                 P_(dp), P_(cl), P_(fe), 16, g.GS_F32, g.GS_LAYOUT_CHW, g.GS_FEAT_ON,
                                 ctypes.cast(bgc, ctypes.c_void_p), P_(out["rgb"]), P_(out["depth"]), P_(out["alpha"]),
                                 P_(out["feat"]), P_(out["T_final"]), P_(out["last_idx"]), P_(out["n_contrib"]), None,
                                 P_(st), g._stream())
    torch.cuda.synchronize()
    res["plant_code"] = code
    res["plant_status"] = int(st.item())
print(json.dumps(res))
"""


def _child(tmp_path, checked, plant=False):
    env = dict(os.environ)
    if checked:
        env["GSFF_CHECKED"] = "1"
    else:
        env.pop("GSFF_CHECKED", None)
    out = str(tmp_path / ("checked.npz" if checked else "plain.npz"))
    code = (_CHILD.replace("@ROOT@", repr(ROOT))
            .replace("@LIBNAME@", repr("libgsff_checked.so" if checked else "libgsff.so"))
            .replace("@OUT@", repr(out)).replace("@PLANT@", repr(plant)))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1]), np.load(out)


def test_checked_build_equals_normal_build_and_flags_a_bad_id(gs, tmp_path):
    from paper_2504_19409_gb300 import build
    build.build(checked=True)
    res_n, a = _child(tmp_path, checked=False)
    res_c, b = _child(tmp_path, checked=True, plant=True)
    assert res_n["status"] == 0 and res_c["status"] == 0
    for k in a.files:
        if k.startswith("fwd_"):
            assert np.array_equal(a[k], b[k]), k
        else:
            # float atomics: the summation order may differ between runs
            assert np.allclose(a[k], b[k], rtol=1e-5, atol=1e-7 * np.abs(a[k]).max()), k
    assert res_c["plant_code"] == gs.GS_OK
    assert res_c["plant_status"] & (1 << gs.GS_ERR_BOUNDS), res_c
