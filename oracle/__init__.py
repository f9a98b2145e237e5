"""FP64 CPU oracle of the feature-field Gaussian rasterizer.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline / reference leg are the only callers. The product path never
imports this package. The C++ source (gsff_oracle.cpp) restates the paper's
Eq. 1-4 (Sec. 3.1-3.2) and the 3DGS compositing rules in double precision and
shares no code with the CUDA library.

Pins (tests/test_oracle_*.py): single-Gaussian closed form, two-Gaussian
closed form, sum of weights plus final transmittance equals one, feature
channels that copy colour and depth, linearity in the features, rigid
re-expression of the pose, brute-force ordering of tiny scenes, and FP64
central finite differences of every gradient including the pose tangent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gsff_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (-ffp-contract=off keeps binary32 replays exact)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]
    tmp = _LIB + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", _SRC, "-o", tmp], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [_SRC, "-o", tmp], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.ora_bin.restype = ctypes.c_int64
        _lib.ora_num_threads.restype = ctypes.c_int
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def cam_array(cam) -> np.ndarray:
    return _f64([cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, *np.asarray(cam.R).ravel(),
                 *np.asarray(cam.t).ravel(), cam.near])


def num_threads() -> int:
    return lib().ora_num_threads()


def set_threads(n: int) -> None:
    lib().ora_set_threads(int(n))


def project_f64(cam, means, scales, quats, opacity):
    P = means.shape[0]
    out = dict(uv=np.zeros((P, 2)), conic=np.zeros((P, 3)), depth=np.zeros(P), cov=np.zeros((P, 3)),
               radius=np.zeros(P), rect=np.zeros((P, 4), np.int32), touched=np.zeros(P, np.int32))
    m, s, q, o = _f64(means), _f64(scales), _f64(quats), _f64(opacity)
    lib().ora_project_f64(_p(cam_array(cam)), ctypes.c_int(P), _p(m), _p(s), _p(q), _p(o),
                          _p(out["uv"]), _p(out["conic"]), _p(out["depth"]), _p(out["cov"]),
                          _p(out["radius"]), _p(out["rect"]), _p(out["touched"]))
    return out


def project_b32(cam, means, scales, quats, opacity):
    """binary32 replay of the GPU's projection order of operations."""
    P = means.shape[0]
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    out = dict(uv=np.zeros((P, 2), np.float32), conic=np.zeros((P, 3), np.float32),
               depth=np.zeros(P, np.float32), rect=np.zeros((P, 4), np.int32),
               touched=np.zeros(P, np.int32))
    m, s, q, o = f(means), f(scales), f(quats), f(opacity)
    lib().ora_project_b32(_p(cam_array(cam)), ctypes.c_int(P), _p(m), _p(s), _p(q), _p(o),
                          _p(out["uv"]), _p(out["conic"]), _p(out["depth"]), _p(out["rect"]),
                          _p(out["touched"]))
    return out


def bin_lists(cam, rect, depth):
    """(ranges [T,2] int32, gids [I] int32) sorted by (tile, depth, id)."""
    T = cam.tiles_x * cam.tiles_y
    rect = np.ascontiguousarray(rect, dtype=np.int32)
    nI = int(((rect[:, 2] - rect[:, 0]) * (rect[:, 3] - rect[:, 1])).sum())
    ranges = np.zeros((T, 2), np.int32)
    gids = np.zeros(max(nI, 1), np.int32)
    n = lib().ora_bin(ctypes.c_int(rect.shape[0]), _p(rect), _p(_f64(depth)), ctypes.c_int(cam.tiles_x),
                      ctypes.c_int(cam.tiles_y), _p(ranges), _p(gids))
    assert n == nI
    return ranges, gids[:nI]


def render_fwd(cam, ranges, gids, uv, conic, opacity, colors, depth, feats, bg=(0.0, 0.0, 0.0)):
    H, W = cam.height, cam.width
    N = 0 if feats is None else feats.shape[1]
    out = dict(rgb=np.zeros((3, H, W)), depth=np.zeros((H, W)), alpha=np.zeros((H, W)),
               feat=np.zeros((N, H, W)), T_final=np.zeros((H, W)),
               last_idx=np.zeros((H, W), np.int32), n_contrib=np.zeros((H, W), np.int32),
               margin=np.zeros((H, W)))
    fe = _f64(feats) if N > 0 else np.zeros((1,))
    lib().ora_render_fwd(_p(cam_array(cam)), ctypes.c_int(cam.tiles_x), _p(np.ascontiguousarray(ranges, np.int32)),
                         _p(np.ascontiguousarray(gids, np.int32)), _p(_f64(uv)), _p(_f64(conic)),
                         _p(_f64(opacity)), _p(_f64(colors)), _p(_f64(depth)), _p(fe), ctypes.c_int(N),
                         _p(_f64(bg)), _p(out["rgb"]), _p(out["depth"]), _p(out["alpha"]), _p(out["feat"]),
                         _p(out["T_final"]), _p(out["last_idx"]), _p(out["n_contrib"]), _p(out["margin"]))
    return out


def edge_mask(rgb, tau):
    """Tracking edge mask m_e (Sec. 3.2) of rgb [3,H,W] (float32), decided in binary32."""
    rgb = np.ascontiguousarray(rgb, np.float32)
    H, W = rgb.shape[1], rgb.shape[2]
    out = np.zeros((H, W), np.uint8)
    lib().ora_edge_mask(ctypes.c_int(W), ctypes.c_int(H), rgb.ctypes.data_as(ctypes.c_void_p), ctypes.c_float(tau),
                        out.ctypes.data_as(ctypes.c_void_p))
    return out


def tracking_grad(rgb, depth, gt_rgb, gt_depth, alpha_ref, alpha_min, m_e, lam):
    """(loss, g_rgb, g_depth) of Eq. 6 in double."""
    H, W = depth.shape
    g_rgb, g_depth = np.zeros((3, H, W)), np.zeros((H, W))
    me = np.ascontiguousarray(m_e, np.uint8)
    lib().ora_tracking_grad.restype = ctypes.c_double
    loss = lib().ora_tracking_grad(ctypes.c_int(W), ctypes.c_int(H), _p(_f64(rgb)), _p(_f64(depth)), _p(_f64(gt_rgb)),
                                   _p(_f64(gt_depth)), _p(_f64(alpha_ref)), ctypes.c_double(alpha_min),
                                   me.ctypes.data_as(ctypes.c_void_p), ctypes.c_double(lam), _p(g_rgb), _p(g_depth))
    return float(loss), g_rgb, g_depth


def pose_update(pose, g, m, v, step, lr_t, lr_r, b1=0.9, b2=0.999, eps=1e-8, tol_t=1e-4, tol_r=1e-4):
    """Adam on the pose tangent then T <- Exp(delta) T; updates pose (12), m, v (6) in place (float64
    arrays); returns the convergence flag."""
    for a in (pose, m, v):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return int(lib().ora_pose_update(_p(pose), _p(_f64(g)), _p(m), _p(v), ctypes.c_int(step), ctypes.c_double(lr_t),
                                     ctypes.c_double(lr_r), ctypes.c_double(b1), ctypes.c_double(b2),
                                     ctypes.c_double(eps), ctypes.c_double(tol_t), ctypes.c_double(tol_r)))


def semantic_ce(feat, labels, hwc=False):
    """(loss, grad) of Eq. 9 on logits feat ([N,H,W], or [H,W,N] with hwc) in double."""
    feat = _f64(feat)
    if hwc:
        H, W, N = feat.shape
    else:
        N, H, W = feat.shape
    lab = np.ascontiguousarray(labels, np.int32)
    grad = np.zeros_like(feat)
    lib().ora_semantic_ce.restype = ctypes.c_double
    loss = lib().ora_semantic_ce(ctypes.c_int(W), ctypes.c_int(H), ctypes.c_int(N), ctypes.c_int(int(hwc)), _p(feat),
                                 lab.ctypes.data_as(ctypes.c_void_p), _p(grad))
    return float(loss), grad


def argmax_labels(feat, hwc=False):
    """Eq. 10: argmax over the channels (first maximum) of the given binary32 values."""
    return np.argmax(np.asarray(feat), axis=-1 if hwc else 0).astype(np.int32)


def label_logits_b32(f, q):
    """Eq. 12 logits replayed in binary32 (the GPU's fused multiply-add order); f [npix, M], q [L, M]."""
    f = np.ascontiguousarray(f, np.float32)
    q = np.ascontiguousarray(q, np.float32)
    z = np.zeros((f.shape[0], q.shape[0]), np.float32)
    lib().ora_label_logits_b32(ctypes.c_longlong(f.shape[0]), ctypes.c_int(f.shape[1]), ctypes.c_int(q.shape[0]),
                               f.ctypes.data_as(ctypes.c_void_p), q.ctypes.data_as(ctypes.c_void_p),
                               z.ctypes.data_as(ctypes.c_void_p))
    return z


def label_probs(f, q):
    """Eq. 12 probabilities in double; f [npix, M], q [L, M]."""
    f, q = _f64(f), _f64(q)
    out = np.zeros((f.shape[0], q.shape[0]))
    lib().ora_label_probs(ctypes.c_longlong(f.shape[0]), ctypes.c_int(f.shape[1]), ctypes.c_int(q.shape[0]), _p(f),
                          _p(q), _p(out))
    return out


def sh_colors(cam, means, sh):
    """View-dependent colours [P,3] from SH coefficients sh [P, K, 3] (K = (lmax+1)^2) in double."""
    sh = _f64(sh)
    P, K = sh.shape[0], sh.shape[1]
    lmax = int(round(K ** 0.5)) - 1
    out = np.zeros((P, 3))
    lib().ora_sh_colors(_p(cam_array(cam)), ctypes.c_int(P), ctypes.c_int(lmax), _p(_f64(means)), _p(sh), _p(out))
    return out


def sh_colors_bwd(cam, means, sh, d_colors):
    """(d_sh [P,K,3], d_means [P,3], d_pose [6]) of the SH colours in double."""
    sh = _f64(sh)
    P, K = sh.shape[0], sh.shape[1]
    lmax = int(round(K ** 0.5)) - 1
    d_sh, d_means, d_pose = np.zeros_like(sh), np.zeros((P, 3)), np.zeros(6)
    lib().ora_sh_colors_bwd(_p(cam_array(cam)), ctypes.c_int(P), ctypes.c_int(lmax), _p(_f64(means)), _p(sh),
                            _p(_f64(d_colors)), _p(d_sh), _p(d_means), _p(d_pose))
    return d_sh, d_means, d_pose


def sh_basis(dirs, lmax=3):
    """Real SH basis values [n, (lmax+1)^2] at unit directions dirs [n,3]."""
    dirs = _f64(dirs)
    out = np.zeros((dirs.shape[0], (lmax + 1) ** 2))
    lib().ora_sh_basis(ctypes.c_int(dirs.shape[0]), ctypes.c_int(lmax), _p(dirs), _p(out))
    return out


def visibility(cam, ranges, gids, uv, conic, opacity):
    """Per Gaussian, the largest transmittance in front of it over the pixels where it is blended
    (0 where blended nowhere); visible in the keyframe sense (Sec. 3.2) when it exceeds 0.5."""
    P = uv.shape[0]
    out = np.zeros(P)
    lib().ora_visibility(_p(cam_array(cam)), ctypes.c_int(cam.tiles_x), _p(np.ascontiguousarray(ranges, np.int32)),
                         _p(np.ascontiguousarray(gids, np.int32)), _p(_f64(uv)), _p(_f64(conic)),
                         _p(_f64(opacity)), ctypes.c_int(P), _p(out))
    return out


def render_bwd(cam, ranges, gids, uv, conic, opacity, colors, depth, feats, g_rgb=None, g_depth=None,
               g_alpha=None, g_feat=None, coupled=False, bg=(0.0, 0.0, 0.0)):
    P = uv.shape[0]
    N = 0 if feats is None else feats.shape[1]
    out = dict(d_uv=np.zeros((P, 2)), d_conic=np.zeros((P, 3)), d_opacity=np.zeros(P),
               d_colors=np.zeros((P, 3)), d_depth=np.zeros(P), d_feats=np.zeros((P, N)))
    fe = _f64(feats) if N > 0 else np.zeros((1,))
    opt = lambda a: None if a is None else _f64(a)
    g_rgb, g_depth, g_alpha = opt(g_rgb), opt(g_depth), opt(g_alpha)
    g_feat = opt(g_feat) if N > 0 else None
    lib().ora_render_bwd(_p(cam_array(cam)), ctypes.c_int(cam.tiles_x), _p(np.ascontiguousarray(ranges, np.int32)),
                         _p(np.ascontiguousarray(gids, np.int32)), _p(_f64(uv)), _p(_f64(conic)),
                         _p(_f64(opacity)), _p(_f64(colors)), _p(_f64(depth)), _p(fe), ctypes.c_int(N),
                         _p(_f64(bg)), _p(g_rgb), _p(g_depth), _p(g_alpha), _p(g_feat),
                         ctypes.c_int(int(coupled)), ctypes.c_int(P), _p(out["d_uv"]), _p(out["d_conic"]),
                         _p(out["d_opacity"]), _p(out["d_colors"]), _p(out["d_depth"]), _p(out["d_feats"]))
    return out


def project_bwd_f64(cam, means, scales, quats, opacity, d_uv, d_conic, d_depth):
    P = means.shape[0]
    out = dict(d_means=np.zeros((P, 3)), d_scales=np.zeros((P, 3)), d_quats=np.zeros((P, 4)),
               d_pose=np.zeros(6))
    lib().ora_project_bwd_f64(_p(cam_array(cam)), ctypes.c_int(P), _p(_f64(means)), _p(_f64(scales)),
                              _p(_f64(quats)), _p(_f64(opacity)), _p(_f64(d_uv)), _p(_f64(d_conic)),
                              _p(_f64(d_depth)), _p(out["d_means"]), _p(out["d_scales"]),
                              _p(out["d_quats"]), _p(out["d_pose"]))
    return out


# ---- whole-pipeline helpers ------------------------------------------------

def render_full(cam, scene, bg=(0.0, 0.0, 0.0), records="f64", feats=None):
    """Project, bin and composite in the oracle.

    records="f64": projection in double (Eq. 1 literally) -- the pipeline the
    finite-difference pins differentiate. records="b32": the projection's
    binary32 replay supplies the discrete decisions and the per-Gaussian
    records (exact binary32 values, then composited in double) -- the pipeline
    the GPU is compared with.
    """
    feats = scene.feats if feats is None else feats
    if records == "f64":
        pr = project_f64(cam, scene.means, scene.scales, scene.quats, scene.opacity)
    else:
        pr = project_b32(cam.as_f32() if hasattr(cam, "as_f32") else cam, scene.means, scene.scales,
                         scene.quats, scene.opacity)
    ranges, gids = bin_lists(cam, pr["rect"], pr["depth"])
    fw = render_fwd(cam, ranges, gids, pr["uv"], pr["conic"], scene.opacity, scene.colors, pr["depth"],
                    feats if feats.shape[1] > 0 else None, bg)
    return pr, ranges, gids, fw


def render_full_grad(cam, scene, g_rgb, g_depth, g_alpha, g_feat, coupled=False, bg=(0.0, 0.0, 0.0),
                     records="f64"):
    """Forward plus the full adjoint (render then projection) in the oracle."""
    pr, ranges, gids, fw = render_full(cam, scene, bg, records)
    feats = scene.feats if scene.feats.shape[1] > 0 else None
    rb = render_bwd(cam, ranges, gids, pr["uv"], pr["conic"], scene.opacity, scene.colors, pr["depth"],
                    feats, g_rgb, g_depth, g_alpha, g_feat, coupled, bg)
    pb = project_bwd_f64(cam, scene.means, scene.scales, scene.quats, scene.opacity, rb["d_uv"],
                         rb["d_conic"], rb["d_depth"])
    grads = dict(means=pb["d_means"], scales=pb["d_scales"], quats=pb["d_quats"], opacity=rb["d_opacity"],
                 colors=rb["d_colors"], feats=rb["d_feats"], pose=pb["d_pose"], uv=rb["d_uv"],
                 conic=rb["d_conic"], depth=rb["d_depth"])
    return pr, ranges, gids, fw, grads


def linear_loss(fw, g_rgb, g_depth, g_alpha, g_feat):
    """L = <g_rgb, C> + <g_depth, D> + <g_alpha, A> + <g_feat, F>."""
    L = float((g_rgb * fw["rgb"]).sum() + (g_depth * fw["depth"]).sum() + (g_alpha * fw["alpha"]).sum())
    if g_feat is not None and fw["feat"].shape[0] > 0:
        L += float((g_feat * fw["feat"]).sum())
    return L


# ---- per-pixel decoder o(.) (Eq. 11) ------------------------------------------

def decoder_fwd(z, W1, b1, W2, b2):
    z = _f64(z)
    n, din = z.shape
    dh, dout = W2.shape
    y = np.zeros((n, dout))
    lib().ora_decoder_fwd(ctypes.c_int(n), ctypes.c_int(din), ctypes.c_int(dh), ctypes.c_int(dout), _p(z),
                          _p(_f64(W1)), _p(_f64(b1)), _p(_f64(W2)), _p(_f64(b2)), _p(y))
    return y


def decoder_bwd(z, W1, b1, W2, g):
    """Gradients of sum(g * y) w.r.t. (W1, b1, W2, b2, z)."""
    z = _f64(z)
    n, din = z.shape
    dh, dout = W2.shape
    out = dict(W1=np.zeros((din, dh)), b1=np.zeros(dh), W2=np.zeros((dh, dout)), b2=np.zeros(dout),
               z=np.zeros((n, din)))
    lib().ora_decoder_bwd(ctypes.c_int(n), ctypes.c_int(din), ctypes.c_int(dh), ctypes.c_int(dout), _p(z),
                          _p(_f64(W1)), _p(_f64(b1)), _p(_f64(W2)), _p(_f64(g)), _p(out["W1"]), _p(out["b1"]),
                          _p(out["W2"]), _p(out["b2"]), _p(out["z"]))
    return out
