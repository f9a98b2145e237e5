"""GB300-native feature-field Gaussian rasterizer (GSFF-SLAM hot path).

Thin Python binding over the C ABI of ``libgsff.so`` (include/gsff.h). Every
step of the path runs in the library's CUDA kernels; this module only
marshals torch tensors (device memory, streams) into the C calls. There is no
CPU fallback: if the library cannot be loaded every entry point raises.

Entry points with the ABI's names: :func:`project`, :func:`bin_sort`,
:func:`render_fwd`, :func:`render_bwd`, :func:`l1_loss_grad`; a frame-level
:class:`Rasterizer` that owns the per-frame buffers; and :func:`render`, a
``torch.autograd.Function`` returning RGB, depth, alpha and the feature map
with gradients for the Gaussians, the features (decoupled, Sec. 3.1) and the
SE(3) pose tangent (Eq. 4).
"""
from __future__ import annotations

import copy
import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# GSFF_CHECKED=1 loads the bounds-checked build (the same kernels with the ids
# they follow checked; see build.py)
LIB_PATH = os.path.join(_HERE, "libgsff_checked.so" if os.environ.get("GSFF_CHECKED") == "1" else "libgsff.so")

GS_OK, GS_ERR_INVALID_ARG, GS_ERR_CAPACITY, GS_ERR_TIMEOUT, GS_ERR_CUDA, GS_ERR_UNSUPPORTED, GS_ERR_BOUNDS = range(7)
GS_FEAT_OFF, GS_FEAT_ON, GS_FEAT_TENSOR_CORE = 0, 1, 2
GS_FEAT_GRAD_DECOUPLED, GS_FEAT_GRAD_COUPLED = 0, 1
GS_F32, GS_BF16 = 0, 1
GS_LAYOUT_CHW, GS_LAYOUT_HWC = 0, 1
TILE = 16

# Every symbol include/gsff.h declares.
EXPORTS = ("gs_project", "gs_bin_sort_workspace_bytes", "gs_bin_sort", "gs_render_fwd",
           "gs_render_bwd_workspace_bytes", "gs_render_bwd", "gs_l1_loss_grad", "gs_trace_enable",
           "gs_trace_reset", "gs_trace_count", "gs_trace_get", "gs_status_string", "gs_version",
           "gs_bin_sort_static", "gs_decoder_workspace_bytes", "gs_decoder_fwd", "gs_decoder_train",
           "gs_adam_step", "gs_decoder_fwd_tc", "gs_visibility_iou", "gs_edge_mask", "gs_tracking_loss_grad",
           "gs_pose_update", "gs_semantic_ce_grad", "gs_argmax_labels", "gs_label_probs", "gs_decoder_labels_tc",
           "gs_sh_colors", "gs_sh_colors_bwd", "gs_render_fwd_l1", "gs_render_bwd_l1", "gs_tile_order",
           "gs_l1_signs", "gs_tracking_loss_signs", "gs_zero",
           "gs_peak_probe", "gs_count_nonfinite", "gs_pair_state_workspace_bytes", "gs_render_fwd_pairs",
           "gs_render_bwd_pairs", "gs_decoder_train_tc_workspace_bytes", "gs_decoder_train_tc",
           "gs_test_hold_tc_producer")


class GsffError(RuntimeError):
    pass


class GsDecoder(ctypes.Structure):
    _fields_ = [("din", ctypes.c_int32), ("dh", ctypes.c_int32), ("dout", ctypes.c_int32),
                ("W1", ctypes.c_void_p), ("b1", ctypes.c_void_p), ("W2", ctypes.c_void_p), ("b2", ctypes.c_void_p)]


class GsCamera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("near_z", ctypes.c_float),
                ("pose_dev", ctypes.c_void_p)]


class GsL1Terms(ctypes.Structure):
    _fields_ = [("target_rgb", ctypes.c_void_p), ("target_depth", ctypes.c_void_p), ("target_feat", ctypes.c_void_p),
                ("w_rgb", ctypes.c_float), ("w_depth", ctypes.c_float), ("w_feat", ctypes.c_float),
                ("loss", ctypes.c_void_p)]


def l1_terms(targets=None, weights=None, loss=None) -> GsL1Terms:
    """The gs_l1_terms of an L1 loss: targets and weights are dicts with any of "rgb", "depth", "feat"."""
    t = GsL1Terms()
    for k, v in (targets or {}).items():
        if v is None:
            continue
        _need(v, torch.float32, "target " + k)
        setattr(t, "target_" + k, v.data_ptr())
        setattr(t, "w_" + k, float(weights[k]))
    if targets is None:
        for k, w in (weights or {}).items():
            setattr(t, "w_" + k, float(w))
    t.loss = None if loss is None else loss.data_ptr()
    return t


def zero_(t, stream=None):
    """gs_zero: clears a contiguous device tensor in the library's launch chain (see gs_zero)."""
    if not (t.is_cuda and t.is_contiguous()):
        raise GsffError("zero_ needs a contiguous CUDA tensor (a strided view would be cleared over the wrong span)")
    _check(lib().gs_zero(_ptr(t), t.numel() * t.element_size(), _stream(stream)), "gs_zero")
    return t


def hold_tc_producer(on):
    """gs_test_hold_tc_producer: while on, the tensor-core feature kernels' producer warps stay idle, so
    their bounded waits run out (the launch flags GS_ERR_TIMEOUT and returns); a failure-detection test hook."""
    _check(lib().gs_test_hold_tc_producer(1 if on else 0), "gs_test_hold_tc_producer")


def count_nonfinite(tensors, stream=None):
    """gs_count_nonfinite over each float32 CUDA tensor given: returns a device int64 [len(tensors)] with the
    number of NaN / infinite values in each (one kernel per tensor, no host round trip)."""
    tensors = list(tensors)
    out = torch.zeros(max(1, len(tensors)), dtype=torch.int64, device=tensors[0].device if tensors else "cuda")
    for i, t in enumerate(tensors):
        _need(t, torch.float32, "scanned tensor")
        _check(lib().gs_count_nonfinite(t.numel(), _ptr(t), _vp(out.data_ptr() + 8 * i), _stream(stream)),
               "gs_count_nonfinite")
    return out[:len(tensors)]


PROBE_KINDS = ("fp32_fma", "fp32_fma2", "ex2", "mma_sync_bf16")


def peak_probe(kind: int, blocks: int, threads: int = 256, iters: int = 4096, stream=None) -> float:
    """gs_peak_probe: launches one probe on the stream and returns the operations it performs; time it with
    CUDA events around the call."""
    sink = torch.empty(blocks, device="cuda")
    ops = ctypes.c_double(0.0)
    _check(lib().gs_peak_probe(int(kind), int(blocks), int(threads), int(iters), _ptr(sink), ctypes.byref(ops),
                               _stream(stream)), "gs_peak_probe")
    return ops.value


def camera_struct(cam) -> GsCamera:
    c = GsCamera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    R = np.asarray(cam.R, dtype=np.float64).reshape(9)
    t = np.asarray(cam.t, dtype=np.float64).reshape(3)
    for i in range(9):
        c.R[i] = float(R[i])
    for i in range(3):
        c.t[i] = float(t[i])
    c.near_z = float(getattr(cam, "near", 0.2))
    pose = getattr(cam, "pose_dev", None)
    if pose is not None:
        _need(pose, torch.float32, "pose_dev", (12,))
        c.pose_dev = pose.data_ptr()
    return c


def with_device_pose(cam, pose):
    """A copy of `cam` whose kernels take R, t from `pose` (CUDA float32 [12]: R row-major, then t)."""
    c = copy.copy(cam)
    c.pose_dev = pose
    return c


_lib = None
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_sz = ctypes.c_size_t
_f32 = ctypes.c_float


def lib():
    """Load libgsff.so (built in-tree by ``build.py``); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise GsffError(f"CUDA library not built: {LIB_PATH} is missing (run paper_2504_19409_gb300/build.py)")
    L = ctypes.CDLL(LIB_PATH)
    cam_p = ctypes.POINTER(GsCamera)
    L.gs_project.argtypes = [cam_p, _i32] + [_vp] * 10 + [_vp]
    L.gs_project.restype = ctypes.c_int
    L.gs_bin_sort_workspace_bytes.argtypes = [_i32, _i64, _i32]
    L.gs_bin_sort_workspace_bytes.restype = _sz
    L.gs_bin_sort.argtypes = [cam_p, _i32, _vp, _vp, _vp, _i64, _vp, _sz, _vp, _vp, _vp, _vp, _vp, _vp]
    L.gs_bin_sort.restype = ctypes.c_int
    L.gs_bin_sort_static.argtypes = [cam_p, _i32, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp]
    L.gs_bin_sort_static.restype = ctypes.c_int
    L.gs_zero.argtypes = [_vp, _sz, _vp]
    L.gs_zero.restype = ctypes.c_int
    L.gs_test_hold_tc_producer.argtypes = [_i32]
    L.gs_test_hold_tc_producer.restype = ctypes.c_int
    L.gs_peak_probe.argtypes = [_i32, _i32, _i32, _i32, _vp, ctypes.POINTER(ctypes.c_double), _vp]
    L.gs_peak_probe.restype = ctypes.c_int
    L.gs_pair_state_workspace_bytes.argtypes = [_i32, _i32]
    L.gs_pair_state_workspace_bytes.restype = _sz
    L.gs_render_fwd_pairs.argtypes = [cam_p, _i32] + [_vp] * 8 + [_sz, _i64, _vp, _vp, _vp, _vp]
    L.gs_render_fwd_pairs.restype = ctypes.c_int
    L.gs_render_bwd_pairs.argtypes = ([cam_p, _i32] + [_vp] * 5 + [_i32, _i32, _i32, _i32, _vp] + [_vp] * 12 +
                                      [_i32, _vp, _vp, _vp, _sz] + [_vp] * 9)
    L.gs_render_bwd_pairs.restype = ctypes.c_int
    L.gs_count_nonfinite.argtypes = [_i64, _vp, _vp, _vp]
    L.gs_count_nonfinite.restype = ctypes.c_int
    L.gs_tile_order.argtypes = [_i32, _vp, _vp, _vp]
    L.gs_tile_order.restype = ctypes.c_int
    L.gs_render_fwd.argtypes = ([cam_p, _i32] + [_vp] * 9 + [_i32, _i32, _i32, _i32, _vp] + [_vp] * 10)
    L.gs_render_fwd.restype = ctypes.c_int
    L.gs_visibility_iou.argtypes = [_i32, _vp, _vp, _vp, _vp]
    L.gs_visibility_iou.restype = ctypes.c_int
    _f = ctypes.c_float
    L.gs_edge_mask.argtypes = [_i32, _i32, _vp, _f, _vp, _vp]
    L.gs_edge_mask.restype = ctypes.c_int
    L.gs_tracking_loss_grad.argtypes = [_i32, _i32] + [_vp] * 5 + [_f, _vp, _f, _vp, _vp, _vp, _vp]
    L.gs_tracking_loss_signs.argtypes = [_i32, _i32] + [_vp] * 5 + [_f, _vp, _f, _vp, _vp, _vp, _vp]
    L.gs_tracking_loss_signs.restype = ctypes.c_int
    L.gs_tracking_loss_grad.restype = ctypes.c_int
    L.gs_pose_update.argtypes = [_vp] * 4 + [_i32] + [_f] * 7 + [_vp, _vp]
    L.gs_pose_update.restype = ctypes.c_int
    L.gs_semantic_ce_grad.argtypes = [_i32, _i32, _i32, _i32, _vp, _vp, _vp, _vp, _vp]
    L.gs_semantic_ce_grad.restype = ctypes.c_int
    L.gs_argmax_labels.argtypes = [_i32, _i32, _i32, _i32, _vp, _vp, _vp]
    L.gs_argmax_labels.restype = ctypes.c_int
    L.gs_label_probs.argtypes = [_i64, _i32, _i32, _vp, _vp, _vp, _vp, _vp]
    L.gs_label_probs.restype = ctypes.c_int
    L.gs_decoder_labels_tc.argtypes = [ctypes.POINTER(GsDecoder), _i64, _vp, _i32, _vp, _vp, _vp, _vp, _vp]
    L.gs_decoder_labels_tc.restype = ctypes.c_int
    L.gs_sh_colors.argtypes = [cam_p, _i32, _i32, _vp, _vp, _vp, _vp]
    L.gs_sh_colors.restype = ctypes.c_int
    L.gs_sh_colors_bwd.argtypes = [cam_p, _i32, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
    L.gs_sh_colors_bwd.restype = ctypes.c_int
    L.gs_render_bwd_workspace_bytes.argtypes = [_i32]
    L.gs_render_bwd_workspace_bytes.restype = _sz
    L.gs_render_bwd.argtypes = ([cam_p, _i32] + [_vp] * 5 + [_i32, _i32, _i32, _i32, _vp] + [_vp] * 13 +
                                [_i32, _vp, _sz] + [_vp] * 9)
    L.gs_render_bwd.restype = ctypes.c_int
    L.gs_render_fwd_l1.argtypes = ([cam_p, _i32] + [_vp] * 9 + [_i32, _i32, _i32, _i32, _vp] + [_vp] * 8 +
                                   [ctypes.POINTER(GsL1Terms), _vp, _vp, _vp])
    L.gs_render_fwd_l1.restype = ctypes.c_int
    L.gs_render_bwd_l1.argtypes = ([cam_p, _i32] + [_vp] * 5 + [_i32, _i32, _i32, _i32, _vp] + [_vp] * 9 +
                                   [ctypes.POINTER(GsL1Terms), _vp, _vp, _sz] + [_vp] * 9)
    L.gs_render_bwd_l1.restype = ctypes.c_int
    L.gs_l1_signs.argtypes = [_i32, _i32, _i32, _i32, _vp, _vp, _vp, ctypes.POINTER(GsL1Terms), _vp, _vp]
    L.gs_l1_signs.restype = ctypes.c_int
    L.gs_l1_loss_grad.argtypes = [_i64, _vp, _vp, _f32, _vp, _vp, _vp]
    L.gs_l1_loss_grad.restype = ctypes.c_int
    L.gs_trace_enable.argtypes = [_i32]
    L.gs_trace_enable.restype = ctypes.c_int
    L.gs_trace_count.restype = _i32
    L.gs_trace_get.argtypes = [_i32, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(_f32)]
    L.gs_trace_get.restype = ctypes.c_int
    dec_p = ctypes.POINTER(GsDecoder)
    L.gs_decoder_workspace_bytes.argtypes = [dec_p, _i64, _i32]
    L.gs_decoder_workspace_bytes.restype = _sz
    L.gs_decoder_fwd.argtypes = [dec_p, _i64, _vp, _vp, _vp, _sz, _vp]
    L.gs_decoder_fwd.restype = ctypes.c_int
    L.gs_decoder_train.argtypes = [dec_p, _i64, _i64, ctypes.c_uint64, _vp, _vp, _f32, _vp, _sz] + [_vp] * 7
    L.gs_decoder_train.restype = ctypes.c_int
    L.gs_decoder_train_tc_workspace_bytes.argtypes = [_i64]
    L.gs_decoder_train_tc_workspace_bytes.restype = _sz
    L.gs_decoder_train_tc.argtypes = [dec_p, _i64, _i64, ctypes.c_uint64, _vp, _vp, _f32, _vp, _sz] + [_vp] * 8
    L.gs_decoder_train_tc.restype = ctypes.c_int
    L.gs_decoder_fwd_tc.argtypes = [dec_p, _i64, _vp, _vp, _vp, _vp]
    L.gs_decoder_fwd_tc.restype = ctypes.c_int
    L.gs_adam_step.argtypes = [_i64, _vp, _vp, _vp, _vp, _f32, _f32, _f32, _f32, _i32, _vp, _vp]
    L.gs_adam_step.restype = ctypes.c_int
    L.gs_status_string.argtypes = [ctypes.c_int]
    L.gs_status_string.restype = ctypes.c_char_p
    L.gs_version.restype = _i32
    _lib = L
    return L


def status_names(word: int):
    """The error kinds OR-ed as bits (1 << gs_status) into a device status word, by name."""
    return [lib().gs_status_string(i).decode() for i in range(1, GS_ERR_BOUNDS + 1) if word & (1 << i)]


def _check(code: int, what: str):
    if code != GS_OK:
        raise GsffError(f"{what}: {lib().gs_status_string(code).decode()} ({code})")


def _ptr(t):
    return None if t is None else _vp(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return _vp(s.cuda_stream)


def _need(t, dtype, name, shape=None):
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise GsffError(f"{name} must be a contiguous CUDA {dtype} tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise GsffError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t


# ---- the four ABI calls -------------------------------------------------------

def project(cam, means, scales, quats, opacity, out=None, stream=None):
    """gs_project: returns dict(uv [P,2], conic_opacity [P,4], depth [P], rect [P,4], tiles_touched [P],
    n_instances [1] int64)."""
    P = means.shape[0]
    dev = means.device
    for t, n, s in ((means, "means", (P, 3)), (scales, "scales", (P, 3)), (quats, "quats", (P, 4)),
                    (opacity, "opacity", (P,))):
        _need(t, torch.float32, n, s)
    o = out if out is not None else dict(
        uv=torch.empty(P, 2, device=dev), conic_opacity=torch.empty(P, 4, device=dev),
        depth=torch.empty(P, device=dev), rect=torch.empty(P, 4, dtype=torch.int32, device=dev),
        tiles_touched=torch.empty(P, dtype=torch.int32, device=dev),
        n_instances=torch.zeros(1, dtype=torch.int64, device=dev))
    c = camera_struct(cam)
    _check(lib().gs_project(ctypes.byref(c), P, _ptr(means), _ptr(scales), _ptr(quats), _ptr(opacity), _ptr(o["uv"]),
                            _ptr(o["conic_opacity"]), _ptr(o["depth"]), _ptr(o["rect"]), _ptr(o["tiles_touched"]),
                            _ptr(o["n_instances"]), _stream(stream)), "gs_project")
    return o


def bin_sort_workspace_bytes(P: int, capacity: int, num_tiles: int) -> int:
    return int(lib().gs_bin_sort_workspace_bytes(P, capacity, num_tiles))


def bin_sort(cam, proj, capacity, workspace=None, out=None, status=None, stream=None, tile_order=True):
    """gs_bin_sort: returns dict(keys [cap] int64, gids [cap] int32, tile_ranges [T,2], n_instances [1]);
    with tile_order also gs_tile_order's launch order of the tiles (tile_order [T] int32); and
    inst_masks [cap] uint8, where the forward leaves each instance's pixel-block skip mask for the
    adjoint of the same frame. The render calls use both."""
    P = proj["depth"].shape[0]
    dev = proj["depth"].device
    T = ((cam.width + TILE - 1) // TILE) * ((cam.height + TILE - 1) // TILE)
    wsb = bin_sort_workspace_bytes(P, capacity, T)
    ws = workspace if workspace is not None else torch.empty(wsb, dtype=torch.uint8, device=dev)
    o = out if out is not None else dict(
        keys=torch.empty(capacity, dtype=torch.int64, device=dev),
        gids=torch.empty(capacity, dtype=torch.int32, device=dev),
        tile_ranges=torch.empty(T, 2, dtype=torch.int32, device=dev),
        n_instances=torch.zeros(1, dtype=torch.int64, device=dev))
    st = status if status is not None else torch.zeros(1, dtype=torch.int32, device=dev)
    c = camera_struct(cam)
    _check(lib().gs_bin_sort(ctypes.byref(c), P, _ptr(proj["depth"]), _ptr(proj["rect"]),
                             _ptr(proj["tiles_touched"]), int(capacity), _ptr(ws), ws.numel(), _ptr(o["keys"]),
                             _ptr(o["gids"]), _ptr(o["tile_ranges"]), _ptr(o["n_instances"]), _ptr(st),
                             _stream(stream)), "gs_bin_sort")
    if o.get("inst_masks") is None:
        o["inst_masks"] = torch.empty(capacity, dtype=torch.uint8, device=dev)
    if tile_order:
        if o.get("tile_order") is None:
            o["tile_order"] = torch.empty(T, dtype=torch.int32, device=dev)
        _check(lib().gs_tile_order(T, _ptr(o["tile_ranges"]), _ptr(o["tile_order"]), _stream(stream)),
               "gs_tile_order")
    o["status"] = st
    return o


def render_fwd(cam, proj, sort, colors, feats=None, flags=None, layout=GS_LAYOUT_CHW, bg=None, out=None,
               status=None, stream=None, visible=None, l1_targets=None, l1_weights=None, l1_loss=None):
    """gs_render_fwd: returns dict(rgb [3,H,W], depth [H,W], alpha [H,W], feat, T_final, last_idx, n_contrib).
    `visible` (uint8 [P], optional) receives 1 for every Gaussian blended with T > 0.5 in front of it;
    the caller zeroes it. With l1_targets (dict with any of "rgb", "depth", "feat") and l1_weights:
    gs_render_fwd_l1, which also adds the weighted L1 loss to l1_loss and leaves the cotangent signs in
    out["l1_signs"] (int32 [H*W, 2]) for render_bwd_l1."""
    H, W = cam.height, cam.width
    dev = colors.device
    P = colors.shape[0]
    N = 0 if feats is None else feats.shape[1]
    if flags is None:
        flags = GS_FEAT_ON if N > 0 else GS_FEAT_OFF
    feat_on = bool(flags & GS_FEAT_ON)
    dtype = GS_BF16 if (feats is not None and feats.dtype == torch.bfloat16) else GS_F32
    _need(colors, torch.float32, "colors", (P, 3))
    o = out
    if o is None:
        o = dict(rgb=torch.empty(3, H, W, device=dev), depth=torch.empty(H, W, device=dev),
                 alpha=torch.empty(H, W, device=dev), T_final=torch.empty(H, W, device=dev),
                 last_idx=torch.empty(H, W, dtype=torch.int32, device=dev),
                 n_contrib=torch.empty(H, W, dtype=torch.int32, device=dev))
        if feat_on:
            o["feat"] = torch.empty((N, H, W) if layout == GS_LAYOUT_CHW else (H, W, N), device=dev)
    bgc = (ctypes.c_float * 3)(*(bg if bg is not None else (0.0, 0.0, 0.0)))
    st = status if status is not None else torch.zeros(1, dtype=torch.int32, device=dev)
    c = camera_struct(cam)
    args = (ctypes.byref(c), P, _ptr(sort["tile_ranges"]), _ptr(sort.get("tile_order")), _ptr(sort["gids"]),
            _ptr(sort.get("inst_masks")), _ptr(proj["uv"]),
            _ptr(proj["conic_opacity"]), _ptr(proj["depth"]), _ptr(colors), _ptr(feats) if feat_on else None,
            N if feat_on else 0, dtype, layout, flags, ctypes.cast(bgc, _vp), _ptr(o["rgb"]), _ptr(o["depth"]),
            _ptr(o["alpha"]), _ptr(o.get("feat")) if feat_on else None, _ptr(o["T_final"]), _ptr(o["last_idx"]),
            _ptr(o["n_contrib"]), _ptr(visible))
    if l1_targets is None:
        _check(lib().gs_render_fwd(*args, _ptr(st), _stream(stream)), "gs_render_fwd")
        return o
    if o.get("l1_signs") is None:
        o["l1_signs"] = torch.empty(H * W, 2, dtype=torch.int32, device=dev)
    terms = l1_terms({k: v for k, v in l1_targets.items() if feat_on or k != "feat"}, l1_weights, l1_loss)
    _check(lib().gs_render_fwd_l1(*args, ctypes.byref(terms), _ptr(o["l1_signs"]), _ptr(st), _stream(stream)),
           "gs_render_fwd_l1")
    return o


def edge_mask(rgb, tau, out=None, stream=None):
    """gs_edge_mask: uint8 [H,W], 1 where the Sobel gradient of (r+g+b)/3 exceeds tau (Sec. 3.2's m_e)."""
    _need(rgb, torch.float32, "rgb")
    H, W = rgb.shape[1], rgb.shape[2]
    m = out if out is not None else torch.empty(H, W, dtype=torch.uint8, device=rgb.device)
    _check(lib().gs_edge_mask(W, H, _ptr(rgb), float(tau), _ptr(m), _stream(stream)), "gs_edge_mask")
    return m


def tracking_loss_grad(rgb, depth, gt_rgb, gt_depth, alpha_ref, m_e, lambda_t=0.9, alpha_min=0.5, g_rgb=None,
                       g_depth=None, loss=None, stream=None):
    """gs_tracking_loss_grad: the cotangents (g_rgb [3,H,W], g_depth [H,W]) of Eq. 6."""
    H, W = depth.shape
    for t_, n_, sh in ((rgb, "rgb", (3, H, W)), (gt_rgb, "gt_rgb", (3, H, W)), (gt_depth, "gt_depth", (H, W)),
                       (alpha_ref, "alpha_ref", (H, W))):
        _need(t_, torch.float32, n_, sh)
    _need(m_e, torch.uint8, "m_e", (H, W))
    gr = g_rgb if g_rgb is not None else torch.empty_like(rgb)
    gd = g_depth if g_depth is not None else torch.empty_like(depth)
    _check(lib().gs_tracking_loss_grad(W, H, _ptr(rgb), _ptr(depth), _ptr(gt_rgb), _ptr(gt_depth), _ptr(alpha_ref),
                                       float(alpha_min), _ptr(m_e), float(lambda_t), _ptr(gr), _ptr(gd), _ptr(loss),
                                       _stream(stream)), "gs_tracking_loss_grad")
    return gr, gd


def tracking_loss_signs(rgb, depth, gt_rgb, gt_depth, alpha_ref, m_e, lambda_t=0.9, alpha_min=0.5, signs=None,
                        loss=None, stream=None):
    """gs_tracking_loss_signs: Eq. 6's cotangents as sign words (int32 [H*W, 2]) and their weights
    ({"rgb": ..., "depth": ...}) for render_bwd_l1."""
    H, W = depth.shape
    for t_, n_, sh in ((rgb, "rgb", (3, H, W)), (gt_rgb, "gt_rgb", (3, H, W)), (gt_depth, "gt_depth", (H, W)),
                       (alpha_ref, "alpha_ref", (H, W))):
        _need(t_, torch.float32, n_, sh)
    _need(m_e, torch.uint8, "m_e", (H, W))
    sg = signs if signs is not None else torch.empty(H * W, 2, dtype=torch.int32, device=depth.device)
    w = (ctypes.c_float * 2)()
    _check(lib().gs_tracking_loss_signs(W, H, _ptr(rgb), _ptr(depth), _ptr(gt_rgb), _ptr(gt_depth), _ptr(alpha_ref),
                                        float(alpha_min), _ptr(m_e), float(lambda_t), _ptr(sg), ctypes.cast(w, _vp),
                                        _ptr(loss), _stream(stream)), "gs_tracking_loss_signs")
    return sg, {"rgb": float(w[0]), "depth": float(w[1]), "feat": 0.0}


def pose_update(pose, d_pose, m, v, step, lr_trans=1e-3, lr_rot=3e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                tol_trans=1e-4, tol_rot=1e-4, converged=None, stream=None):
    """gs_pose_update: Adam on the pose tangent, then pose <- Exp(delta) pose (all on the device)."""
    for t_, n_, sh in ((pose, "pose", (12,)), (d_pose, "d_pose", (6,)), (m, "m", (6,)), (v, "v", (6,))):
        _need(t_, torch.float32, n_, sh)
    _check(lib().gs_pose_update(_ptr(pose), _ptr(d_pose), _ptr(m), _ptr(v), int(step), float(lr_trans),
                                float(lr_rot), float(beta1), float(beta2), float(eps), float(tol_trans),
                                float(tol_rot), _ptr(converged), _stream(stream)), "gs_pose_update")


def sh_colors(cam, means, sh, out=None, stream=None):
    """gs_sh_colors: view-dependent colours [P,3] from SH coefficients sh [P, K, 3] (K = 1, 4, 9 or 16)."""
    P, K = sh.shape[0], sh.shape[1]
    deg = {1: 0, 4: 1, 9: 2, 16: 3}.get(K)
    if deg is None or sh.shape[2] != 3:
        raise GsffError("sh must be [P, K, 3] with K in (1, 4, 9, 16)")
    _need(sh, torch.float32, "sh")
    _need(means, torch.float32, "means", (P, 3))
    o = out if out is not None else torch.empty(P, 3, device=sh.device)
    c = camera_struct(cam)
    _check(lib().gs_sh_colors(ctypes.byref(c), P, deg, _ptr(means), _ptr(sh), _ptr(o), _stream(stream)),
           "gs_sh_colors")
    return o


def sh_colors_bwd(cam, means, sh, d_colors, d_sh=None, d_means=None, d_pose=None, stream=None):
    """gs_sh_colors_bwd: accumulates into d_sh [P,K,3], d_means [P,3], d_pose [6] (any may be None)."""
    P, K = sh.shape[0], sh.shape[1]
    deg = {1: 0, 4: 1, 9: 2, 16: 3}[K]
    _need(d_colors, torch.float32, "d_colors", (P, 3))
    c = camera_struct(cam)
    _check(lib().gs_sh_colors_bwd(ctypes.byref(c), P, deg, _ptr(means), _ptr(sh), _ptr(d_colors), _ptr(d_sh),
                                  _ptr(d_means), _ptr(d_pose), _stream(stream)), "gs_sh_colors_bwd")


def _feat_shape(feat, layout):
    _need(feat, torch.float32, "feat")
    if layout == GS_LAYOUT_CHW:
        N, H, W = feat.shape
    else:
        H, W, N = feat.shape
    return N, H, W


def semantic_ce_grad(feat, labels, layout=GS_LAYOUT_CHW, grad=None, loss=None, stream=None):
    """gs_semantic_ce_grad (Eq. 9): the softmax cross-entropy cotangent of a rendered map; labels < 0 ignored."""
    N, H, W = _feat_shape(feat, layout)
    _need(labels, torch.int32, "labels", (H, W))
    g = grad if grad is not None else torch.empty_like(feat)
    _check(lib().gs_semantic_ce_grad(W, H, N, layout, _ptr(feat), _ptr(labels), _ptr(g), _ptr(loss),
                                     _stream(stream)), "gs_semantic_ce_grad")
    return g


def argmax_labels(feat, layout=GS_LAYOUT_CHW, out=None, stream=None):
    """gs_argmax_labels (Eq. 10): int32 [H,W] labels, ties to the lowest channel."""
    N, H, W = _feat_shape(feat, layout)
    o = out if out is not None else torch.empty(H, W, dtype=torch.int32, device=feat.device)
    _check(lib().gs_argmax_labels(W, H, N, layout, _ptr(feat), _ptr(o), _stream(stream)), "gs_argmax_labels")
    return o


def label_probs(feat, queries, probs=True, labels=True, stream=None):
    """gs_label_probs (Eq. 12): (probs [npix, L], labels [npix]) of pixel features [npix, M] against
    queries [L, M]; either output can be skipped."""
    _need(feat, torch.float32, "feat")
    _need(queries, torch.float32, "queries")
    npix, M = feat.shape
    L = queries.shape[0]
    if queries.shape[1] != M:
        raise GsffError("queries must be [L, M] with the features' M")
    pr = torch.empty(npix, L, device=feat.device) if probs else None
    lb = torch.empty(npix, dtype=torch.int32, device=feat.device) if labels else None
    _check(lib().gs_label_probs(npix, M, L, _ptr(feat), _ptr(queries), _ptr(pr), _ptr(lb), _stream(stream)),
           "gs_label_probs")
    return pr, lb


def visibility_iou(vis_a, vis_b, counts=None, stream=None):
    """gs_visibility_iou: device int64 [2] = (|a and b|, |a or b|) of two uint8 visibility vectors."""
    _need(vis_a, torch.uint8, "vis_a")
    _need(vis_b, torch.uint8, "vis_b", vis_a.shape)
    c = counts if counts is not None else torch.empty(2, dtype=torch.int64, device=vis_a.device)
    _check(lib().gs_visibility_iou(vis_a.numel(), _ptr(vis_a), _ptr(vis_b), _ptr(c), _stream(stream)),
           "gs_visibility_iou")
    return c


def l1_signs(cam, fwd, l1_targets, l1_weights, l1_loss=None, layout=GS_LAYOUT_CHW, stream=None):
    """gs_l1_signs: the L1 terms of render_fwd(..., l1_targets=...) as a pass over the images of a plain
    render_fwd (fwd), for targets that arrive after the forward ran: adds the loss to l1_loss and leaves
    the cotangent signs in fwd["l1_signs"] for render_bwd_l1, exactly as the fused forward would."""
    H, W = cam.height, cam.width
    feat = fwd.get("feat")
    N = 0 if feat is None else (feat.shape[0] if layout == GS_LAYOUT_CHW else feat.shape[2])
    if fwd.get("l1_signs") is None:
        fwd["l1_signs"] = torch.empty(H * W, 2, dtype=torch.int32, device=fwd["rgb"].device)
    terms = l1_terms({k: v for k, v in l1_targets.items() if N > 0 or k != "feat"}, l1_weights, l1_loss)
    _check(lib().gs_l1_signs(W, H, N, layout, _ptr(fwd["rgb"]), _ptr(fwd["depth"]), _ptr(feat), ctypes.byref(terms),
                             _ptr(fwd["l1_signs"]), _stream(stream)), "gs_l1_signs")
    return fwd


def render_bwd_workspace_bytes(P: int) -> int:
    return int(lib().gs_render_bwd_workspace_bytes(P))


def render_bwd(cam, means, scales, quats, colors, feats, proj, sort, fwd, g_rgb=None, g_depth=None, g_alpha=None,
               g_feat=None, flags=None, layout=GS_LAYOUT_CHW, bg=None, coupled=False, grads=None, workspace=None,
               status=None, stream=None):
    """gs_render_bwd: accumulates into grads (zeroed if created here) and returns it. A caller-given grads
    dict needs only "pose" (and "feats" with features on); classes it leaves out are not computed."""
    P = means.shape[0]
    dev = means.device
    N = 0 if feats is None else feats.shape[1]
    if flags is None:
        flags = GS_FEAT_ON if N > 0 else GS_FEAT_OFF
    feat_on = bool(flags & GS_FEAT_ON)
    dtype = GS_BF16 if (feats is not None and feats.dtype == torch.bfloat16) else GS_F32
    g = grads if grads is not None else dict(
        means=torch.zeros(P, 3, device=dev), scales=torch.zeros(P, 3, device=dev),
        quats=torch.zeros(P, 4, device=dev), opacity=torch.zeros(P, device=dev),
        colors=torch.zeros(P, 3, device=dev), feats=torch.zeros(P, max(N, 1), device=dev)[:, :N],
        pose=torch.zeros(6, device=dev))
    ws = workspace if workspace is not None else torch.empty(max(render_bwd_workspace_bytes(P), 256),
                                                             dtype=torch.uint8, device=dev)
    bgc = (ctypes.c_float * 3)(*(bg if bg is not None else (0.0, 0.0, 0.0)))
    st = status if status is not None else torch.zeros(1, dtype=torch.int32, device=dev)
    c = camera_struct(cam)
    cont = lambda t: None if t is None else t.contiguous()
    g_rgb, g_depth, g_alpha, g_feat = cont(g_rgb), cont(g_depth), cont(g_alpha), cont(g_feat)
    _check(lib().gs_render_bwd(
        ctypes.byref(c), P, _ptr(means), _ptr(scales), _ptr(quats), _ptr(colors), _ptr(feats) if feat_on else None,
        N if feat_on else 0, dtype, layout, flags, ctypes.cast(bgc, _vp), _ptr(sort["tile_ranges"]),
        _ptr(sort.get("tile_order")),
        _ptr(sort["gids"]), _ptr(sort.get("inst_masks")), _ptr(proj["uv"]), _ptr(proj["conic_opacity"]), _ptr(proj["depth"]),
        _ptr(fwd["T_final"]), _ptr(fwd["last_idx"]), _ptr(g_rgb), _ptr(g_depth), _ptr(g_alpha),
        _ptr(g_feat) if feat_on else None, GS_FEAT_GRAD_COUPLED if coupled else GS_FEAT_GRAD_DECOUPLED,
        _ptr(ws), ws.numel(), _ptr(g.get("means")), _ptr(g.get("scales")), _ptr(g.get("quats")),
        _ptr(g.get("opacity")), _ptr(g.get("colors")), _ptr(g["feats"]) if feat_on else None, _ptr(g["pose"]),
        _ptr(st), _stream(stream)),
        "gs_render_bwd")
    return g


def render_bwd_l1(cam, means, scales, quats, colors, feats, proj, sort, fwd, weights, flags=None,
                  layout=GS_LAYOUT_CHW, bg=None, grads=None, workspace=None, status=None, stream=None):
    """gs_render_bwd_l1: the adjoint of the L1 loss evaluated by render_fwd(..., l1_targets=...), its
    cotangents rebuilt from fwd["l1_signs"] and weights (dict with "rgb", "depth", "feat"). Gradients as
    render_bwd."""
    P = means.shape[0]
    dev = means.device
    N = 0 if feats is None else feats.shape[1]
    if flags is None:
        flags = GS_FEAT_ON if N > 0 else GS_FEAT_OFF
    feat_on = bool(flags & GS_FEAT_ON)
    dtype = GS_BF16 if (feats is not None and feats.dtype == torch.bfloat16) else GS_F32
    g = grads if grads is not None else dict(
        means=torch.zeros(P, 3, device=dev), scales=torch.zeros(P, 3, device=dev),
        quats=torch.zeros(P, 4, device=dev), opacity=torch.zeros(P, device=dev),
        colors=torch.zeros(P, 3, device=dev), feats=torch.zeros(P, max(N, 1), device=dev)[:, :N],
        pose=torch.zeros(6, device=dev))
    ws = workspace if workspace is not None else torch.empty(max(render_bwd_workspace_bytes(P), 256),
                                                             dtype=torch.uint8, device=dev)
    bgc = (ctypes.c_float * 3)(*(bg if bg is not None else (0.0, 0.0, 0.0)))
    st = status if status is not None else torch.zeros(1, dtype=torch.int32, device=dev)
    terms = l1_terms(None, {k: weights.get(k, 0.0) for k in ("rgb", "depth", "feat")})
    c = camera_struct(cam)
    _check(lib().gs_render_bwd_l1(
        ctypes.byref(c), P, _ptr(means), _ptr(scales), _ptr(quats), _ptr(colors), _ptr(feats) if feat_on else None,
        N if feat_on else 0, dtype, layout, flags, ctypes.cast(bgc, _vp), _ptr(sort["tile_ranges"]),
        _ptr(sort.get("tile_order")),
        _ptr(sort["gids"]), _ptr(sort.get("inst_masks")), _ptr(proj["uv"]), _ptr(proj["conic_opacity"]), _ptr(proj["depth"]),
        _ptr(fwd["T_final"]), _ptr(fwd["last_idx"]), ctypes.byref(terms), _ptr(fwd["l1_signs"]), _ptr(ws), ws.numel(),
        _ptr(g.get("means")), _ptr(g.get("scales")), _ptr(g.get("quats")), _ptr(g.get("opacity")),
        _ptr(g.get("colors")), _ptr(g["feats"]) if feat_on else None, _ptr(g["pose"]), _ptr(st), _stream(stream)),
        "gs_render_bwd_l1")
    return g


def render_fwd_pairs(cam, proj, sort, fwd, capacity=None, out=None, status=None, stream=None):
    """gs_render_fwd_pairs: the per-pair saved state of the last forward: dict(pair_off [H*W+1] int64,
    pair_T [capacity] float32 (the transmittance in front of each blended pair), n_pairs [1] int64 view)."""
    H, W = cam.height, cam.width
    dev = fwd["T_final"].device
    P = proj["depth"].shape[0]
    if capacity is None:
        capacity = int(fwd["n_contrib"].sum().item())
    o = out if out is not None else {}
    if o.get("pair_off") is None or o["pair_off"].numel() != H * W + 1:
        o["pair_off"] = torch.empty(H * W + 1, dtype=torch.int64, device=dev)
    if o.get("pair_T") is None or o["pair_T"].numel() < capacity:
        o["pair_T"] = torch.empty(max(1, capacity), device=dev)
    wsb = int(lib().gs_pair_state_workspace_bytes(W, H))
    if o.get("ws") is None or o["ws"].numel() < wsb:
        o["ws"] = torch.empty(wsb, dtype=torch.uint8, device=dev)
    st = status if status is not None else torch.zeros(1, dtype=torch.int32, device=dev)
    c = camera_struct(cam)
    _check(lib().gs_render_fwd_pairs(ctypes.byref(c), P, _ptr(sort["tile_ranges"]), _ptr(sort.get("tile_order")),
                                     _ptr(sort["gids"]), _ptr(proj["uv"]), _ptr(proj["conic_opacity"]),
                                     _ptr(fwd["last_idx"]), _ptr(fwd["n_contrib"]), _ptr(o["ws"]), o["ws"].numel(),
                                     int(o["pair_T"].numel()), _ptr(o["pair_off"]), _ptr(o["pair_T"]), _ptr(st),
                                     _stream(stream)), "gs_render_fwd_pairs")
    o["n_pairs"] = o["pair_off"][H * W:]
    return o


def render_bwd_pairs(cam, means, scales, quats, colors, feats, proj, sort, fwd, pairs=None, g_rgb=None, g_depth=None,
                     g_alpha=None, g_feat=None, flags=None, layout=GS_LAYOUT_CHW, bg=None, coupled=False, grads=None,
                     workspace=None, status=None, stream=None):
    """gs_render_bwd_pairs: the SIMT adjoint with the transmittance read from pairs (render_fwd_pairs of the same
    frame) or, with pairs=None, recovered by division; gradients as render_bwd."""
    P = means.shape[0]
    dev = means.device
    N = 0 if feats is None else feats.shape[1]
    if flags is None:
        flags = GS_FEAT_ON if N > 0 else GS_FEAT_OFF
    feat_on = bool(flags & GS_FEAT_ON)
    dtype = GS_BF16 if (feats is not None and feats.dtype == torch.bfloat16) else GS_F32
    g = grads if grads is not None else dict(
        means=torch.zeros(P, 3, device=dev), scales=torch.zeros(P, 3, device=dev),
        quats=torch.zeros(P, 4, device=dev), opacity=torch.zeros(P, device=dev),
        colors=torch.zeros(P, 3, device=dev), feats=torch.zeros(P, max(N, 1), device=dev)[:, :N],
        pose=torch.zeros(6, device=dev))
    ws = workspace if workspace is not None else torch.empty(max(render_bwd_workspace_bytes(P), 256),
                                                             dtype=torch.uint8, device=dev)
    bgc = (ctypes.c_float * 3)(*(bg if bg is not None else (0.0, 0.0, 0.0)))
    st = status if status is not None else torch.zeros(1, dtype=torch.int32, device=dev)
    c = camera_struct(cam)
    cont = lambda t: None if t is None else t.contiguous()
    g_rgb, g_depth, g_alpha, g_feat = cont(g_rgb), cont(g_depth), cont(g_alpha), cont(g_feat)
    _check(lib().gs_render_bwd_pairs(
        ctypes.byref(c), P, _ptr(means), _ptr(scales), _ptr(quats), _ptr(colors), _ptr(feats) if feat_on else None,
        N if feat_on else 0, dtype, layout, flags, ctypes.cast(bgc, _vp), _ptr(sort["tile_ranges"]),
        _ptr(sort.get("tile_order")), _ptr(sort["gids"]), _ptr(proj["uv"]), _ptr(proj["conic_opacity"]),
        _ptr(proj["depth"]), _ptr(fwd["T_final"]), _ptr(fwd["last_idx"]), _ptr(g_rgb), _ptr(g_depth), _ptr(g_alpha),
        _ptr(g_feat) if feat_on else None, GS_FEAT_GRAD_COUPLED if coupled else GS_FEAT_GRAD_DECOUPLED,
        _ptr(pairs["pair_off"]) if pairs else None, _ptr(pairs["pair_T"]) if pairs else None, _ptr(ws), ws.numel(),
        _ptr(g.get("means")), _ptr(g.get("scales")), _ptr(g.get("quats")), _ptr(g.get("opacity")),
        _ptr(g.get("colors")), _ptr(g["feats"]) if feat_on else None, _ptr(g["pose"]), _ptr(st), _stream(stream)),
        "gs_render_bwd_pairs")
    return g


def l1_loss_grad(pred, target, scale, grad=None, loss=None, stream=None):
    """gs_l1_loss_grad: grad = scale sign(pred - target); loss += scale sum |pred - target|."""
    _need(pred, torch.float32, "pred")
    _need(target, torch.float32, "target", pred.shape)
    g = grad if grad is not None else torch.empty_like(pred)
    _check(lib().gs_l1_loss_grad(pred.numel(), _ptr(pred), _ptr(target), float(scale), _ptr(g), _ptr(loss),
                                 _stream(stream)), "gs_l1_loss_grad")
    return g


# ---- tracing ------------------------------------------------------------------

def trace_enable(capacity: int) -> None:
    _check(lib().gs_trace_enable(int(capacity)), "gs_trace_enable")


def trace_reset() -> None:
    lib().gs_trace_reset()


def trace_read():
    """[(kernel name, ms)] for every traced launch since the last reset."""
    out = []
    for i in range(lib().gs_trace_count()):
        name = ctypes.c_char_p()
        ms = ctypes.c_float()
        _check(lib().gs_trace_get(i, ctypes.byref(name), ctypes.byref(ms)), "gs_trace_get")
        out.append((name.value.decode(), ms.value))
    return out


# ---- frame-level driver -----------------------------------------------------------

class Rasterizer:
    """Owns the per-frame device buffers for one (P, image, N) shape and runs
    project -> bin_sort -> render_fwd -> render_bwd with no host round trip
    (instance capacity fixed up front; overflow is flagged in ``status``)."""

    def __init__(self, P, width, height, N=0, capacity=None, layout=GS_LAYOUT_CHW, feat_dtype=torch.float32,
                 device="cuda", flags=None):
        self.P, self.W, self.H, self.N = P, width, height, N
        self.layout = layout
        self.flags = flags if flags is not None else (GS_FEAT_ON if N > 0 else GS_FEAT_OFF)
        self.device = torch.device(device)
        self.T = ((width + TILE - 1) // TILE) * ((height + TILE - 1) // TILE)
        self.capacity = int(capacity) if capacity else max(1024, 8 * P)
        dev = self.device
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        self.proj = dict(uv=torch.empty(P, 2, device=dev), conic_opacity=torch.empty(P, 4, device=dev),
                         depth=torch.empty(P, device=dev), rect=torch.empty(P, 4, dtype=torch.int32, device=dev),
                         tiles_touched=torch.empty(P, dtype=torch.int32, device=dev),
                         n_instances=torch.zeros(1, dtype=torch.int64, device=dev))
        self._alloc_sort()
        self.fwd = dict(rgb=torch.empty(3, height, width, device=dev), depth=torch.empty(height, width, device=dev),
                        alpha=torch.empty(height, width, device=dev), T_final=torch.empty(height, width, device=dev),
                        last_idx=torch.empty(height, width, dtype=torch.int32, device=dev),
                        n_contrib=torch.empty(height, width, dtype=torch.int32, device=dev))
        if self.flags & GS_FEAT_ON:
            shape = (N, height, width) if layout == GS_LAYOUT_CHW else (height, width, N)
            self.fwd["feat"] = torch.empty(shape, device=dev)
        self.bwd_ws = torch.empty(max(render_bwd_workspace_bytes(P), 256), dtype=torch.uint8, device=dev)
        # all gradient outputs are views of one buffer (each part starting on a 256-byte boundary), so
        # zeroing them before an adjoint is a single fill
        shapes = dict(means=(P, 3), scales=(P, 3), quats=(P, 4), opacity=(P,), colors=(P, 3), feats=(P, max(N, 1)),
                      pose=(6,))
        offs, n = {}, 0
        for k, shp in shapes.items():
            offs[k] = n
            n += (int(np.prod(shp)) + 63) // 64 * 64
        self.grad_arena = torch.zeros(n, device=dev)
        self.grads = {k: self.grad_arena[offs[k]:offs[k] + int(np.prod(shp))].view(shp) for k, shp in shapes.items()}
        self.grads["feats"] = self.grads["feats"][:, :N]

    def _alloc_sort(self):
        dev = self.device
        self.sort_ws = torch.empty(bin_sort_workspace_bytes(self.P, self.capacity, self.T), dtype=torch.uint8,
                                   device=dev)
        self.sort = dict(keys=torch.empty(self.capacity, dtype=torch.int64, device=dev),
                         gids=torch.empty(self.capacity, dtype=torch.int32, device=dev),
                         tile_ranges=torch.empty(self.T, 2, dtype=torch.int32, device=dev),
                         tile_order=torch.empty(self.T, dtype=torch.int32, device=dev),
                         inst_masks=torch.empty(self.capacity, dtype=torch.uint8, device=dev),
                         n_instances=torch.zeros(1, dtype=torch.int64, device=dev))

    def ensure_capacity(self, cam, means, scales, quats, opacity, slack=1.25):
        """Project once, read the instance count (one sync) and grow the sort buffers if needed."""
        project(cam, means, scales, quats, opacity, out=self.proj)
        need = int(self.proj["n_instances"].item())
        if need > self.capacity:
            self.capacity = int(need * slack) + 1024
            self._alloc_sort()
        return need

    def forward(self, cam, means, scales, quats, opacity, colors, feats=None, bg=None, stream=None, visible=None,
                l1_targets=None, l1_weights=None, l1_loss=None, wait_event=None):
        """Project, bin and composite; with l1_targets also the L1 loss of the images (see render_fwd).
        wait_event (a torch.cuda.Event or a list of them, e.g. recorded after copying the colours and
        targets on other streams) is waited for only before compositing, so projection and binning
        overlap with it."""
        project(cam, means, scales, quats, opacity, out=self.proj, stream=stream)
        bin_sort(cam, self.proj, self.capacity, workspace=self.sort_ws, out=self.sort, status=self.status,
                 stream=stream)
        if wait_event is not None:
            st = stream if stream is not None else torch.cuda.current_stream(self.device)
            for ev in (wait_event if isinstance(wait_event, (list, tuple)) else (wait_event,)):
                st.wait_event(ev)
        render_fwd(cam, self.proj, self.sort, colors, feats, flags=self.flags, layout=self.layout, bg=bg,
                   out=self.fwd, status=self.status, stream=stream, visible=visible, l1_targets=l1_targets,
                   l1_weights=l1_weights, l1_loss=l1_loss)
        return self.fwd

    def backward(self, cam, means, scales, quats, colors, feats=None, g_rgb=None, g_depth=None, g_alpha=None,
                 g_feat=None, bg=None, coupled=False, zero=True, stream=None):
        if zero:
            zero_(self.grad_arena, stream)
        render_bwd(cam, means, scales, quats, colors, feats, self.proj, self.sort, self.fwd, g_rgb, g_depth, g_alpha,
                   g_feat, flags=self.flags, layout=self.layout, bg=bg, coupled=coupled, grads=self.grads,
                   workspace=self.bwd_ws, status=self.status, stream=stream)
        return self.grads

    def l1_loss(self, cam, l1_targets, l1_weights, l1_loss=None, wait_event=None, stream=None):
        """The L1 terms of the last forward's images (gs_l1_signs), for targets copied while the forward
        ran: waits for wait_event (an event or a list of them) first; backward_l1 then differentiates it."""
        if wait_event is not None:
            st = stream if stream is not None else torch.cuda.current_stream(self.device)
            for ev in (wait_event if isinstance(wait_event, (list, tuple)) else (wait_event,)):
                st.wait_event(ev)
        l1_signs(cam, self.fwd, l1_targets, l1_weights, l1_loss, layout=self.layout, stream=stream)
        return self.fwd

    def backward_l1(self, cam, means, scales, quats, colors, feats, weights, bg=None, zero=True, stream=None):
        """The adjoint of the L1 loss that the last forward(..., l1_targets=...) evaluated
        (gs_render_bwd_l1)."""
        if zero:
            zero_(self.grad_arena, stream)
        render_bwd_l1(cam, means, scales, quats, colors, feats, self.proj, self.sort, self.fwd, weights,
                      flags=self.flags, layout=self.layout, bg=bg, grads=self.grads, workspace=self.bwd_ws,
                      status=self.status, stream=stream)
        return self.grads

    def render_pose_grad(self, cam, means, scales, quats, colors, g_rgb, g_depth, grads, stream=None):
        """The adjoint of the last forward into grads["pose"] only (frozen Gaussians, as in tracking)."""
        render_bwd(cam, means, scales, quats, colors, None, self.proj, self.sort, self.fwd, g_rgb, g_depth,
                   flags=GS_FEAT_OFF, grads=grads, workspace=self.bwd_ws, status=self.status, stream=stream)
        return grads

    def render_pose_grad_l1(self, cam, means, scales, quats, colors, weights, grads, stream=None):
        """The pose gradient of the last forward from the L1 sign words in self.fwd["l1_signs"]
        (e.g. tracking_loss_signs's) and their weights: gs_render_bwd_l1 with the Gaussians frozen."""
        render_bwd_l1(cam, means, scales, quats, colors, None, self.proj, self.sort, self.fwd, weights,
                      flags=GS_FEAT_OFF, grads=grads, workspace=self.bwd_ws, status=self.status, stream=stream)
        return grads

    def check_finite(self, grads=True, stream=None):
        """Scans the last forward's images (and, with grads, the gradient arena) for NaN / infinite values;
        raises GsffError naming the buffers that hold any."""
        bufs = {k: v for k, v in self.fwd.items() if v.dtype == torch.float32}
        if grads:
            bufs["gradients"] = self.grad_arena
        counts = count_nonfinite(bufs.values(), stream=stream).cpu().tolist()
        bad = {k: c for k, c in zip(bufs, counts) if c}
        if bad:
            raise GsffError(f"non-finite values: {bad}")

    def check_status(self):
        s = int(self.status.item())
        if s:
            raise GsffError("device status: " + ", ".join(status_names(s)))


# ---- autograd -----------------------------------------------------------------

class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, scales, quats, opacity, colors, feats, pose, cam, opts):
        P = means.shape[0]
        N = 0 if feats is None else feats.shape[1]
        flags = GS_FEAT_ON if (N > 0 and opts.get("render_features", True)) else GS_FEAT_OFF
        layout = opts.get("layout", GS_LAYOUT_CHW)
        bg = opts.get("bg")
        cont = [t.detach().contiguous() for t in (means, scales, quats, opacity, colors)]
        fe = None if feats is None else feats.detach().contiguous()
        proj = project(cam, *cont[:4])
        cap = max(int(proj["n_instances"].item()), 1)
        srt = bin_sort(cam, proj, cap)
        fw = render_fwd(cam, proj, srt, cont[4], fe, flags=flags, layout=layout, bg=bg, status=srt["status"])
        if int(srt["status"].item()):
            raise GsffError("device status flagged during the forward pass")
        ctx.cam, ctx.opts, ctx.flags, ctx.N = cam, opts, flags, N
        ctx.proj, ctx.sort, ctx.fwd = proj, srt, fw
        ctx.save_for_backward(*cont, fe if fe is not None else torch.empty(0, device=means.device))
        ctx.has_feats = fe is not None
        feat = fw.get("feat")
        if feat is None:
            H, W = cam.height, cam.width
            feat = torch.zeros((N, H, W) if layout == GS_LAYOUT_CHW else (H, W, N), device=means.device)
        ctx.mark_non_differentiable(fw["T_final"], fw["n_contrib"])
        return fw["rgb"], fw["depth"], fw["alpha"], feat, fw["T_final"], fw["n_contrib"]

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_alpha, g_feat, _gT, _gn):
        means, scales, quats, opacity, colors, fe = ctx.saved_tensors
        fe = fe if ctx.has_feats else None
        grads = render_bwd(ctx.cam, means, scales, quats, colors, fe, ctx.proj, ctx.sort, ctx.fwd, g_rgb, g_depth,
                           g_alpha, g_feat, flags=ctx.flags, layout=ctx.opts.get("layout", GS_LAYOUT_CHW),
                           bg=ctx.opts.get("bg"), coupled=ctx.opts.get("coupled", False))
        d_feats = grads["feats"] if ctx.has_feats else None
        if ctx.has_feats and d_feats.shape[1] == 0:
            d_feats = torch.zeros_like(fe, dtype=torch.float32)
        return (grads["means"], grads["scales"], grads["quats"], grads["opacity"], grads["colors"], d_feats,
                grads["pose"], None, None)


def render(means, scales, quats, opacity, colors, feats, pose, cam, render_features=True, layout=GS_LAYOUT_CHW,
           bg=None, coupled=False):
    """Differentiable render at camera ``cam``.

    ``pose`` is a 6-vector tangent (rho, theta) of the left perturbation
    T <- Exp(pose) T evaluated at 0: its value is not read, its gradient is
    dL/dtau (Eq. 4). Returns (rgb [3,H,W], depth [H,W], alpha [H,W], feat,
    T_final [H,W], n_contrib [H,W]).
    """
    opts = dict(render_features=render_features, layout=layout, bg=bg, coupled=coupled)
    return _RenderFn.apply(means, scales, quats, opacity, colors, feats, pose, cam, opts)
