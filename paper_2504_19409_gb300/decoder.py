"""Learned per-pixel decoder o(.) of Eq. 11 and its trainer.

A din-channel latent per Gaussian is rendered with the rasterizer (Eq. 3 with
f := latent) and lifted per pixel to the full feature width by
y = W2^T gelu(W1^T z + b1) + b2 (Eq. 11, read as a 1x1 lift). Every step runs
in the library's kernels (gs_render_fwd / gs_render_bwd for the latent
render, gs_decoder_train for the MLP, gs_adam_step for the updates); this
module only owns device buffers and orders the calls.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from . import (GS_FEAT_ON, GS_FEAT_TENSOR_CORE, GS_LAYOUT_HWC, GsDecoder, GsffError, Rasterizer, _check, _ptr,
               _stream, lib)
from .scenegen import Rng


def _bf16_round(t: torch.Tensor) -> torch.Tensor:
    return t.to(torch.bfloat16).to(torch.float32)


class Decoder:
    """MLP din -> dh -> dout with fp32 master weights, bf16-rounded working
    copies (what the products use), gradients and Adam moments."""

    def __init__(self, din=16, dh=128, dout=512, seed=0, device="cuda"):
        self.din, self.dh, self.dout = din, dh, dout
        self.device = torch.device(device)
        rng = Rng(seed)
        W1 = rng.normal(din * dh).reshape(din, dh) / math.sqrt(din)
        W2 = rng.normal(dh * dout).reshape(dh, dout) / math.sqrt(dh)
        t = lambda a: torch.tensor(np.asarray(a, np.float32), device=self.device)
        self.params = dict(W1=t(W1), b1=t(np.zeros(dh)), W2=t(W2), b2=t(np.zeros(dout)))
        self.work = dict(W1=_bf16_round(self.params["W1"]), W2=_bf16_round(self.params["W2"]))
        self.grads = {k: torch.zeros_like(v) for k, v in self.params.items()}
        self.m = {k: torch.zeros_like(v) for k, v in self.params.items()}
        self.v = {k: torch.zeros_like(v) for k, v in self.params.items()}
        self.step = 0
        self._ws = None
        self._ws_tc = None

    def struct(self) -> GsDecoder:
        d = GsDecoder()
        d.din, d.dh, d.dout = self.din, self.dh, self.dout
        d.W1 = self.work["W1"].data_ptr()
        d.b1 = self.params["b1"].data_ptr()
        d.W2 = self.work["W2"].data_ptr()
        d.b2 = self.params["b2"].data_ptr()
        return d

    def workspace(self, n, training):
        d = self.struct()
        need = int(lib().gs_decoder_workspace_bytes(ctypes.byref(d), int(n), int(training)))
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(max(need, 256), dtype=torch.uint8, device=self.device)
        return self._ws

    def forward(self, z: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        n = z.shape[0]
        y = out if out is not None else torch.empty(n, self.dout, device=self.device)
        ws = self.workspace(n, 0)
        d = self.struct()
        _check(lib().gs_decoder_fwd(ctypes.byref(d), n, _ptr(z), _ptr(y), _ptr(ws), ws.numel(), _stream(stream)),
               "gs_decoder_fwd")
        return y

    def forward_tc(self, z: torch.Tensor, out: torch.Tensor | None = None, status=None, stream=None) -> torch.Tensor:
        """The same map on tcgen05 (bf16 operands, fp32 accumulation)."""
        n = z.shape[0]
        y = out if out is not None else torch.empty(n, self.dout, device=self.device)
        d = self.struct()
        _check(lib().gs_decoder_fwd_tc(ctypes.byref(d), n, _ptr(z), _ptr(y), _ptr(status), _stream(stream)),
               "gs_decoder_fwd_tc")
        return y

    def labels_tc(self, z: torch.Tensor, queries: torch.Tensor, probs=True, labels=True, status=None, stream=None):
        """Eq. 12 label probabilities / labels of the decoded field straight from the latents z [n, 16]
        (the 512-d features are never formed): returns (probs [n, L] or None, labels [n] or None)."""
        n, L = z.shape[0], queries.shape[0]
        pr = torch.empty(n, L, device=self.device) if probs else None
        lb = torch.empty(n, dtype=torch.int32, device=self.device) if labels else None
        d = self.struct()
        _check(lib().gs_decoder_labels_tc(ctypes.byref(d), n, _ptr(z), L, _ptr(queries.contiguous()), _ptr(pr),
                                          _ptr(lb), _ptr(status), _stream(stream)), "gs_decoder_labels_tc")
        return pr, lb

    def zero_grad(self):
        for g in self.grads.values():
            g.zero_()

    def train_eval(self, z_map, target, nsample, seed, loss_scale, dz_map=None, loss=None, stream=None):
        """Accumulates the MLP gradients (and dL/dz at the sampled pixels)."""
        ws = self.workspace(nsample, 1)
        d = self.struct()
        g = self.grads
        _check(lib().gs_decoder_train(ctypes.byref(d), int(nsample), int(z_map.shape[0]), ctypes.c_uint64(seed),
                                      _ptr(z_map), _ptr(target), float(loss_scale), _ptr(ws), ws.numel(),
                                      _ptr(g["W1"]), _ptr(g["b1"]), _ptr(g["W2"]), _ptr(g["b2"]), _ptr(dz_map),
                                      _ptr(loss), _stream(stream)), "gs_decoder_train")

    def train_eval_tc(self, z_map, target, nsample, seed, loss_scale, dz_map=None, loss=None, status=None,
                      stream=None):
        """The same accumulation on tcgen05 (gs_decoder_train_tc; bf16 operands, fp32 sums)."""
        need = int(lib().gs_decoder_train_tc_workspace_bytes(int(nsample)))
        if self._ws_tc is None or self._ws_tc.numel() < need:
            self._ws_tc = torch.empty(max(need, 256), dtype=torch.uint8, device=self.device)
        d = self.struct()
        g = self.grads
        _check(lib().gs_decoder_train_tc(ctypes.byref(d), int(nsample), int(z_map.shape[0]), ctypes.c_uint64(seed),
                                         _ptr(z_map), _ptr(target), float(loss_scale), _ptr(self._ws_tc),
                                         self._ws_tc.numel(), _ptr(g["W1"]), _ptr(g["b1"]), _ptr(g["W2"]),
                                         _ptr(g["b2"]), _ptr(dz_map), _ptr(loss), _ptr(status), _stream(stream)),
               "gs_decoder_train_tc")

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        self.step += 1
        for k, p in self.params.items():
            q = self.work.get(k)
            _check(lib().gs_adam_step(p.numel(), _ptr(p), _ptr(self.grads[k]), _ptr(self.m[k]), _ptr(self.v[k]),
                                      float(lr), float(beta1), float(beta2), float(eps), self.step, _ptr(q),
                                      _stream(stream)), "gs_adam_step")


    # ---- checkpoint / resume (raw little-endian binary) ------------------
    # magic "GSFFDEC1", int32 din, dh, dout, step, then for W1, b1, W2, b2 in
    # turn the fp32 parameter, its first and its second Adam moment. The bf16
    # working copies are the parameters' bf16 rounding, rebuilt on load.
    _MAGIC = b"GSFFDEC1"
    _NAMES = ("W1", "b1", "W2", "b2")

    def state_bytes(self) -> bytes:
        head = self._MAGIC + np.array([self.din, self.dh, self.dout, self.step], "<i4").tobytes()
        body = b"".join(t.detach().cpu().numpy().astype("<f4").tobytes()
                        for k in self._NAMES for t in (self.params[k], self.m[k], self.v[k]))
        return head + body

    def load_state_bytes(self, blob: bytes) -> int:
        """Restores the state from state_bytes(); returns the bytes consumed."""
        if blob[:8] != self._MAGIC:
            raise ValueError("not a decoder checkpoint")
        din, dh, dout, step = (int(x) for x in np.frombuffer(blob, "<i4", 4, 8))
        if (din, dh, dout) != (self.din, self.dh, self.dout):
            raise ValueError(f"checkpoint is {din}x{dh}x{dout}, decoder is {self.din}x{self.dh}x{self.dout}")
        off = 24
        for k in self._NAMES:
            for t in (self.params[k], self.m[k], self.v[k]):
                n = t.numel()
                if len(blob) < off + 4 * n:
                    raise ValueError("truncated decoder checkpoint")
                t.copy_(torch.from_numpy(np.frombuffer(blob, "<f4", n, off).reshape(t.shape).copy()))
                off += 4 * n
        for k in self.work:
            self.work[k].copy_(_bf16_round(self.params[k]))
        self.step = step
        return off

    def save(self, path) -> None:
        with open(path, "wb") as f:
            f.write(self.state_bytes())

    def load(self, path) -> None:
        with open(path, "rb") as f:
            self.load_state_bytes(f.read())


def adam_tensor(param, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(lib().gs_adam_step(param.numel(), _ptr(param), _ptr(grad), _ptr(m), _ptr(v), float(lr), float(beta1),
                              float(beta2), float(eps), int(step), None, _stream(stream)), "gs_adam_step")


class LatentFieldTrainer:
    """Joint training of per-Gaussian latents and the decoder against
    full-width renders (targets) of the same Gaussians at training poses.

    Per step: render the latents (din channels, HWC) -> gs_decoder_train on
    `nsample` sampled pixels (MSE to the target) -> gs_render_bwd of the latent
    render with dL/dz as the feature cotangent (decoupled: only the latents
    receive it) -> Adam on the latents and the MLP.
    """

    def __init__(self, scene_tensors, latents0: np.ndarray, cam_like, decoder: Decoder, capacity=None,
                 device="cuda", tensor_core=True):
        self.means, self.scales, self.quats, self.opac, self.cols = scene_tensors
        self.device = torch.device(device)
        self.lat = torch.tensor(np.asarray(latents0, np.float32), device=self.device)
        self.lat_g = torch.zeros_like(self.lat)
        self.lat_m = torch.zeros_like(self.lat)
        self.lat_v = torch.zeros_like(self.lat)
        self.lat_step = 0
        self.dec = decoder
        # the decoder's training on tcgen05 (gs_decoder_train_tc) where its
        # shape allows, else the fp32 SIMT chain (gs_decoder_train)
        self.tensor_core = tensor_core and (decoder.din, decoder.dh, decoder.dout) == (16, 128, 512)
        P, din = self.lat.shape
        self.ras = Rasterizer(P, cam_like.width, cam_like.height, N=din, capacity=capacity, layout=GS_LAYOUT_HWC,
                              device=device)
        HW = cam_like.width * cam_like.height
        self.dz = torch.zeros(HW, din, device=self.device)
        self.loss = torch.zeros(1, device=self.device)

    def ensure_capacity(self, cams):
        for c in cams:
            self.ras.ensure_capacity(c, self.means, self.scales, self.quats, self.opac)

    def render_latents(self, cam):
        fw = self.ras.forward(cam, self.means, self.scales, self.quats, self.opac, self.cols, self.lat)
        return fw["feat"].reshape(-1, self.lat.shape[1])

    def step(self, cam, target, nsample, seed, lr_dec=1e-3, lr_lat=1e-2):
        z = self.render_latents(cam)
        self.dec.zero_grad()
        self.dz.zero_()
        scale = 1.0 / (nsample * self.dec.dout)
        train = self.dec.train_eval_tc if self.tensor_core else self.dec.train_eval
        train(z, target, nsample, seed, scale, dz_map=self.dz, loss=self.loss)
        g_feat = self.dz.reshape(cam.height, cam.width, -1)
        gr = self.ras.backward(cam, self.means, self.scales, self.quats, self.cols, self.lat, g_feat=g_feat)
        self.dec.adam(lr_dec)
        self.lat_step += 1
        adam_tensor(self.lat, gr["feats"], self.lat_m, self.lat_v, self.lat_step, lr_lat)

    # checkpoint: magic "GSFFLAT1", int64 P, int32 din, int32 latent step, the
    # latents and their two Adam moments (fp32), then the decoder's state
    _MAGIC = b"GSFFLAT1"

    def save(self, path) -> None:
        P, din = self.lat.shape
        head = self._MAGIC + np.array([P], "<i8").tobytes() + np.array([din, self.lat_step], "<i4").tobytes()
        body = b"".join(t.detach().cpu().numpy().astype("<f4").tobytes() for t in (self.lat, self.lat_m, self.lat_v))
        with open(path, "wb") as f:
            f.write(head + body + self.dec.state_bytes())

    def load(self, path) -> None:
        with open(path, "rb") as f:
            blob = f.read()
        if blob[:8] != self._MAGIC:
            raise ValueError("not a latent-field checkpoint")
        P = int(np.frombuffer(blob, "<i8", 1, 8)[0])
        din, step = (int(x) for x in np.frombuffer(blob, "<i4", 2, 16))
        if (P, din) != tuple(self.lat.shape):
            raise ValueError(f"checkpoint holds {P}x{din} latents, trainer has {tuple(self.lat.shape)}")
        off, n = 24, P * din
        for t in (self.lat, self.lat_m, self.lat_v):
            t.copy_(torch.from_numpy(np.frombuffer(blob, "<f4", n, off).reshape(P, din).copy()))
            off += 4 * n
        self.lat_step = step
        self.dec.load_state_bytes(blob[off:])

    def decode(self, cam):
        return self.dec.forward(self.render_latents(cam).contiguous())


def render_features(ras: Rasterizer, cam, scene_tensors, feats, tensor_core=False):
    """Full-width feature render (HWC rows [H*W, N]) with the plain fp32 path
    or the tensor-core form (bf16 features)."""
    means, scales, quats, opac, cols = scene_tensors
    if tensor_core:
        ras.flags = GS_FEAT_ON | GS_FEAT_TENSOR_CORE
    fw = ras.forward(cam, means, scales, quats, opac, cols, feats)
    return fw["feat"].reshape(-1, feats.shape[1])


def feature_error(pred: torch.Tensor, ref: torch.Tensor, mask: torch.Tensor | None = None):
    """(relative L2, mean cosine) of per-pixel feature rows, optionally over a mask."""
    if mask is not None:
        pred, ref = pred[mask], ref[mask]
    rel = float(torch.linalg.norm(pred - ref) / torch.linalg.norm(ref).clamp_min(1e-30))
    cos = torch.nn.functional.cosine_similarity(pred, ref, dim=1, eps=1e-12)
    return rel, float(cos.mean())
