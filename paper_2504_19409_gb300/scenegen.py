"""Seeded synthetic scenes and camera trajectories.

This module only draws random numbers and lays out arrays. It holds none of
the renderer's arithmetic, so both the CUDA path and the FP64 CPU oracle can
take their inputs from it without sharing any of the method.

Random numbers come from one counter-based generator: splitmix64 (Steele,
Lea, Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014)
evaluated on consecutive counters, turned into doubles in [0, 1) from the top
53 bits, and into normals by the Box-Muller transform.

Scene shapes follow the paper's workloads (indoor RGB-D sequences rendered
with 3D Gaussians, Sec. 3.1): a view-frustum cloud for the small cases and a
6 x 5 x 3 m box room (four walls and a floor) for SLAM-frame scale.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


_CHUNK = 1 << 22  # draws per piece when a large request is spread over threads


def _pieces(n: int):
    return [(a, min(n, a + _CHUNK)) for a in range(0, n, _CHUNK)]


def _run(fn, pieces):
    """fn over the pieces, on a thread pool for large requests (numpy releases
    the GIL inside its array operations); the result does not depend on it."""
    if len(pieces) <= 2:
        return [fn(a, b) for a, b in pieces]
    import concurrent.futures as cf
    import os
    with cf.ThreadPoolExecutor(max_workers=min(len(pieces), os.cpu_count() or 1)) as ex:
        return list(ex.map(lambda ab: fn(*ab), pieces))


class Rng:
    """splitmix64 stream: draw k returns mix(seed + (c + k + 1) * golden).

    Every draw depends only on its counter, so a large request is computed in
    pieces (on several threads) with the same result as in one piece."""

    def __init__(self, seed: int):
        with np.errstate(over="ignore"):
            self._base = _mix(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64) * _GOLDEN)[0]
        self._ctr = 0

    def _u64_at(self, first: int, n: int) -> np.ndarray:
        idx = np.arange(first + 1, first + 1 + n, dtype=np.uint64)
        with np.errstate(over="ignore"):
            return _mix(self._base + idx * _GOLDEN)

    @staticmethod
    def _to_unit(x: np.ndarray) -> np.ndarray:
        return (x >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def u64(self, n: int) -> np.ndarray:
        c = self._ctr
        self._ctr += n
        return np.concatenate(_run(lambda a, b: self._u64_at(c + a, b - a), _pieces(n))) if n else \
            np.zeros(0, np.uint64)

    def uniform(self, n: int) -> np.ndarray:
        """Doubles in [0, 1) from the top 53 bits."""
        c = self._ctr
        self._ctr += n
        if n == 0:
            return np.zeros(0)
        return np.concatenate(_run(lambda a, b: self._to_unit(self._u64_at(c + a, b - a)), _pieces(n)))

    def normal(self, n: int) -> np.ndarray:
        """Standard normals by Box-Muller (both outputs of each pair used):
        pair i takes draws i and m + i of the next 2m = 2 ceil(n / 2)."""
        m = (n + 1) // 2
        c = self._ctr
        self._ctr += 2 * m
        z = np.empty(2 * m)

        def piece(a, b):
            u1 = 1.0 - self._to_unit(self._u64_at(c + a, b - a))      # (0, 1]
            u2 = self._to_unit(self._u64_at(c + m + a, b - a))
            r = np.sqrt(-2.0 * np.log(u1))
            z[2 * a:2 * b:2] = r * np.cos(2.0 * np.pi * u2)
            z[2 * a + 1:2 * b:2] = r * np.sin(2.0 * np.pi * u2)

        _run(piece, _pieces(m))
        return z[:n]


@dataclasses.dataclass
class Camera:
    """Pinhole camera, world->camera rigid transform mu_c = R mu + t.

    OpenCV axes: x right, y down, z forward. R is row-major 3x3.
    """
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    R: np.ndarray          # (3, 3) float64
    t: np.ndarray          # (3,)   float64
    near: float = 0.2

    @property
    def tiles_x(self) -> int:
        return (self.width + 15) // 16

    @property
    def tiles_y(self) -> int:
        return (self.height + 15) // 16

    @property
    def num_tiles(self) -> int:
        return self.tiles_x * self.tiles_y

    def as_f32(self) -> "Camera":
        """The same camera with every real parameter rounded to binary32."""
        f = lambda x: float(np.float32(x))
        return Camera(self.width, self.height, f(self.fx), f(self.fy), f(self.cx), f(self.cy),
                      self.R.astype(np.float32).astype(np.float64),
                      self.t.astype(np.float32).astype(np.float64), f(self.near))


@dataclasses.dataclass
class Scene:
    """Per-Gaussian parameters as float32 arrays (the layout the GPU reads).

    means [P,3], scales [P,3] (linear, > 0), quats [P,4] (w,x,y,z, not
    normalised), opacity [P] in (0,1), colors [P,3], feats [P,N].
    """
    means: np.ndarray
    scales: np.ndarray
    quats: np.ndarray
    opacity: np.ndarray
    colors: np.ndarray
    feats: np.ndarray

    @property
    def P(self) -> int:
        return self.means.shape[0]

    @property
    def N(self) -> int:
        return self.feats.shape[1]


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _unit_quats(rng: Rng, P: int) -> np.ndarray:
    # Four i.i.d. normals normalised: uniform on S^3.
    q = rng.normal(4 * P).reshape(P, 4)
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def frustum_scene(seed: int, P: int, cam: Camera, N: int, zmin: float = 1.0, zmax: float = 5.0,
                  log_scale_mu: float = -3.0, log_scale_sigma: float = 0.5,
                  opacity_mu: float = 0.0) -> Scene:
    """Gaussians volume-uniform in the view frustum between zmin and zmax.

    z = cbrt(U (zmax^3 - zmin^3) + zmin^3); pixel (u, v) uniform over the
    image; the point is back-projected through the pinhole and moved to world
    coordinates with the inverse of the camera transform.
    """
    rng = Rng(seed)
    z = np.cbrt(rng.uniform(P) * (zmax ** 3 - zmin ** 3) + zmin ** 3)
    u = rng.uniform(P) * cam.width
    v = rng.uniform(P) * cam.height
    pc = np.stack([(u - cam.cx) * z / cam.fx, (v - cam.cy) * z / cam.fy, z], axis=1)
    means = (pc - cam.t[None, :]) @ cam.R            # R^T (pc - t)
    scales = np.exp(log_scale_mu + log_scale_sigma * rng.normal(3 * P)).reshape(P, 3)
    quats = _unit_quats(rng, P)
    opacity = _sigmoid(opacity_mu + rng.normal(P))
    colors = rng.uniform(3 * P).reshape(P, 3)
    feats = rng.normal(N * P).reshape(P, N) if N > 0 else np.zeros((P, 0))
    return Scene(means.astype(np.float32), scales.astype(np.float32), quats.astype(np.float32),
                 opacity.astype(np.float32), colors.astype(np.float32), feats.astype(np.float32))


# Box room [0,6] x [0,5] x [0,3] m: four walls and a floor, no ceiling.
ROOM = (6.0, 5.0, 3.0)


def room_scene(seed: int, P: int, N: int, jitter: float = 0.02, log_scale_mu: float = -4.0,
               log_scale_sigma: float = 0.5, opacity_mu: float = 1.0,
               feat_kind: str = "normal") -> Scene:
    """Gaussians on the walls and floor of the box room, area-proportional,
    with N(0, jitter) displacement along the surface normal.

    feat_kind: "normal" -> i.i.d. N(0,1); "unit" -> N(0,1) rows scaled to unit
    L2 norm; "none" -> N must be 0.
    """
    lx, ly, lz = ROOM
    # surfaces: (area, origin, axis-a, axis-b, normal)
    surfs = [
        (lx * ly, (0, 0, 0), (lx, 0, 0), (0, ly, 0), (0, 0, 1)),     # floor z=0
        (lx * lz, (0, 0, 0), (lx, 0, 0), (0, 0, lz), (0, 1, 0)),     # wall y=0
        (lx * lz, (0, ly, 0), (lx, 0, 0), (0, 0, lz), (0, -1, 0)),   # wall y=ly
        (ly * lz, (0, 0, 0), (0, ly, 0), (0, 0, lz), (1, 0, 0)),     # wall x=0
        (ly * lz, (lx, 0, 0), (0, ly, 0), (0, 0, lz), (-1, 0, 0)),   # wall x=lx
    ]
    areas = np.array([s[0] for s in surfs])
    cdf = np.cumsum(areas) / areas.sum()
    rng = Rng(seed)
    pick = np.searchsorted(cdf, rng.uniform(P), side="right")
    pick = np.minimum(pick, len(surfs) - 1)
    a = rng.uniform(P)
    b = rng.uniform(P)
    j = jitter * rng.normal(P)
    org = np.array([s[1] for s in surfs], dtype=np.float64)[pick]
    ea = np.array([s[2] for s in surfs], dtype=np.float64)[pick]
    eb = np.array([s[3] for s in surfs], dtype=np.float64)[pick]
    nrm = np.array([s[4] for s in surfs], dtype=np.float64)[pick]
    means = org + a[:, None] * ea + b[:, None] * eb + j[:, None] * nrm
    scales = np.exp(log_scale_mu + log_scale_sigma * rng.normal(3 * P)).reshape(P, 3)
    quats = _unit_quats(rng, P)
    opacity = _sigmoid(opacity_mu + rng.normal(P))
    colors = rng.uniform(3 * P).reshape(P, 3)
    if N == 0 or feat_kind == "none":
        feats = np.zeros((P, N))
    elif feat_kind == "prototypes":
        feats = prototype_features(seed + 7919, means, N)
    else:
        feats = rng.normal(N * P).reshape(P, N)
        if feat_kind == "unit":
            feats = feats / np.linalg.norm(feats, axis=1, keepdims=True)
    return Scene(means.astype(np.float32), scales.astype(np.float32), quats.astype(np.float32),
                 opacity.astype(np.float32), colors.astype(np.float32), feats.astype(np.float32))


def prototype_features(seed: int, means: np.ndarray, N: int, n_proto: int = 32, patch: float = 0.75,
                       noise: float = 0.05) -> np.ndarray:
    """Label-structured features: the room surfaces are cut into `patch`-metre
    cells, each cell draws one of `n_proto` unit prototype vectors, and every
    Gaussian carries its cell's prototype plus isotropic noise of expected
    norm `noise` (N(0, noise^2 / N) per channel), renormalised: features that
    come from a small label set, as the paper's GT-label and text-query
    supervision does (Sec. 3.3)."""
    rng = Rng(seed)
    protos = rng.normal(n_proto * N).reshape(n_proto, N)
    protos /= np.linalg.norm(protos, axis=1, keepdims=True)
    cell = np.floor(np.asarray(means, np.float64) / patch).astype(np.int64)
    h = (cell[:, 0] * 73856093) ^ (cell[:, 1] * 19349663) ^ (cell[:, 2] * 83492791)
    labels = np.mod(h, n_proto)
    f = protos[labels] + (noise / math.sqrt(N)) * rng.normal(means.shape[0] * N).reshape(-1, N)
    return f / np.linalg.norm(f, axis=1, keepdims=True)


def pca_basis(feats: np.ndarray, k: int):
    """Mean and top-k principal directions of per-Gaussian features (the
    linear rank-k encode/decode the learned decoder is compared with)."""
    f = np.asarray(feats, np.float64)
    mu = f.mean(0)
    c = np.cov((f - mu).T)
    w, v = np.linalg.eigh(c)
    U = v[:, np.argsort(w)[::-1][:k]]
    return mu, U


def look_camera(width: int, height: int, f: float, centre, yaw: float, pitch: float) -> Camera:
    """Camera at `centre` looking along (cos p cos y, cos p sin y, sin p) with
    world z up; rows of R are the camera's right, down and forward axes."""
    fwd = np.array([math.cos(pitch) * math.cos(yaw), math.cos(pitch) * math.sin(yaw), math.sin(pitch)])
    right = np.cross(fwd, np.array([0.0, 0.0, 1.0]))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd], axis=0)
    c = np.asarray(centre, dtype=np.float64)
    return Camera(width, height, f, f, width / 2.0, height / 2.0, R, -R @ c)


def room_trajectory(k: int, n_frames: int = 100, width: int = 1200, height: int = 680,
                    f: float = 600.0) -> Camera:
    """Frame k of the seeded smooth loop inside the room (>= 0.5 m from walls)."""
    s = 2.0 * math.pi * k / n_frames
    centre = (3.0 + 0.8 * math.sin(s), 2.5 + 0.6 * math.sin(2 * s), 1.5 + 0.2 * math.sin(3 * s))
    yaw = s
    pitch = 0.1 * math.sin(2.0 * math.pi * k / 50.0)
    return look_camera(width, height, f, centre, yaw, pitch)


def perturb_pose(cam: Camera, rho, theta) -> Camera:
    """Left-perturbed camera Exp(tau) T with tau = (rho, theta) (Rodrigues)."""
    th = np.asarray(theta, dtype=np.float64)
    a = np.linalg.norm(th)
    K = np.array([[0, -th[2], th[1]], [th[2], 0, -th[0]], [-th[1], th[0], 0]])
    if a < 1e-12:
        Rd = np.eye(3) + K
        V = np.eye(3) + 0.5 * K
    else:
        Rd = np.eye(3) + math.sin(a) / a * K + (1 - math.cos(a)) / a ** 2 * (K @ K)
        V = np.eye(3) + (1 - math.cos(a)) / a ** 2 * K + (a - math.sin(a)) / a ** 3 * (K @ K)
    td = V @ np.asarray(rho, dtype=np.float64)
    return dataclasses.replace(cam, R=Rd @ cam.R, t=Rd @ cam.t + td)


def identity_camera(width: int, height: int, f: float) -> Camera:
    return Camera(width, height, f, f, width / 2.0, height / 2.0, np.eye(3), np.zeros(3))


# ---- the workloads -------------------------------------------------------

def small_case(seed: int = 1, P: int = 2000, N: int = 16):
    """2,000 Gaussians in the frustum of a 128x96 identity camera, f=100."""
    cam = identity_camera(128, 96, 100.0)
    return frustum_scene(seed, P, cam, N), cam


def fd_case(seed: int = 5, P: int = 500, N: int = 64):
    """500 Gaussians at 64x48, f=50: the finite-difference case."""
    cam = identity_camera(64, 48, 50.0)
    return frustum_scene(seed, P, cam, N), cam


def room_case(seed: int = 3, P: int = 300_000, N: int = 16, feat_kind: str = "normal"):
    """SLAM-frame scale: Gaussians on the room surfaces; frame 0 camera."""
    return room_scene(seed, P, N, feat_kind=feat_kind), room_trajectory(0)


def random_linear_functional(seed: int, H: int, W: int, N: int):
    """Fixed random cotangents (g_rgb [3,H,W], g_depth, g_alpha [H,W], g_feat [N,H,W])."""
    rng = Rng(seed)
    g_rgb = rng.normal(3 * H * W).reshape(3, H, W)
    g_d = rng.normal(H * W).reshape(H, W) * 0.1
    g_a = rng.normal(H * W).reshape(H, W)
    g_f = rng.normal(N * H * W).reshape(N, H, W) if N > 0 else np.zeros((0, H, W))
    return (g_rgb.astype(np.float32), g_d.astype(np.float32), g_a.astype(np.float32),
            g_f.astype(np.float32))
