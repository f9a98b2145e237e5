"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign, a transposed rotation, a wrong tile rule, a missing factor in the
adjoint) fails it:

* closed forms: one Gaussian on the optical axis (axis-aligned and rolled
  about the axis), two Gaussians stacked on the axis (Eq. 2);
* invariants: sum of weights + final transmittance = 1, feature channels that
  copy colour and depth reproduce C and D (Eq. 2 vs Eq. 3), rigid
  re-expression of the camera pose, dtau translation part = R sum dmu;
* brute force: tile rectangles from pixel enumeration and per-tile lists
  ordered by pairwise comparison (front-to-back, Sec. 3.1);
* adjoints: FP64 central finite differences of every parameter class and of
  the six pose components (Eq. 4), decoupled vs coupled feature gradient
  (Sec. 3.1), exact linearity in the features.
"""
import math

import numpy as np
import pytest

from paper_2504_19409_gb300.scenegen import Camera, Scene


def _scene(means, scales, quats, opac, colors, feats):
    f = lambda a: np.asarray(a, dtype=np.float32)
    return Scene(f(means), f(scales), f(quats), f(opac), f(colors), f(feats))


def _pix_centres(cam):
    j, i = np.meshgrid(np.arange(cam.height), np.arange(cam.width), indexing="ij")
    return i + 0.5, j + 0.5


def test_single_gaussian_on_axis_closed_form(ora, sg):
    cam = sg.identity_camera(64, 48, 50.0)
    z, s, o = 2.0, (0.05, 0.08, 0.03), 0.7
    c, f = (0.2, 0.5, 0.9), (1.5, -2.0)
    sc = _scene([[0, 0, z]], [s], [[1, 0, 0, 0]], [o], [c], [f])
    sc = Scene(sc.means, sc.scales, sc.quats, sc.opacity, sc.colors, sc.feats)
    pr, _, _, fw = ora.render_full(cam, sc)
    s64 = np.asarray(sc.scales[0], np.float64)
    a = cam.fx ** 2 * s64[0] ** 2 / z ** 2 + 0.3
    cc = cam.fy ** 2 * s64[1] ** 2 / z ** 2 + 0.3
    assert np.allclose(pr["cov"][0], [a, 0, cc], rtol=1e-12, atol=1e-14)
    assert np.allclose(pr["conic"][0], [1 / a, 0, 1 / cc], rtol=1e-12, atol=1e-14)
    assert np.allclose(pr["uv"][0], [cam.cx, cam.cy])
    assert pr["radius"][0] == math.ceil(3 * math.sqrt(max(a, cc)))
    px, py = _pix_centres(cam)
    dx, dy = cam.cx - px, cam.cy - py
    alpha = np.minimum(0.99, float(sc.opacity[0]) * np.exp(-0.5 * (dx ** 2 / a + dy ** 2 / cc)))
    # tile rectangle of the 3-sigma box; pixels outside it stay empty
    r = pr["radius"][0]
    inside = (np.abs(px - cam.cx) <= r + 16) & (np.abs(py - cam.cy) <= r + 16)
    alpha = np.where(alpha >= 1 / 255, alpha, 0.0)
    tx0, ty0, tx1, ty1 = pr["rect"][0]
    in_rect = (px >= 16 * tx0) & (px < 16 * tx1) & (py >= 16 * ty0) & (py < 16 * ty1)
    alpha = np.where(in_rect, alpha, 0.0)
    assert inside[in_rect].all()
    col = sc.colors[0].astype(np.float64)
    for ch in range(3):
        assert np.allclose(fw["rgb"][ch], alpha * col[ch], rtol=1e-12, atol=1e-15)
    assert np.allclose(fw["depth"], alpha * z, rtol=1e-12, atol=1e-15)
    assert np.allclose(fw["alpha"], alpha, rtol=1e-12, atol=1e-15)
    for k in range(2):
        assert np.allclose(fw["feat"][k], alpha * sc.feats[0, k], rtol=1e-12, atol=1e-15)
    assert (fw["n_contrib"] == (alpha > 0)).all()


def test_rolled_gaussian_on_axis_closed_form(ora, sg):
    """A Gaussian rolled about the optical axis: the 2D covariance is the
    rotated diagonal; pins the off-diagonal conic entry and its sign."""
    cam = sg.identity_camera(64, 48, 50.0)
    z, phi = 2.5, 0.6
    s = np.array([0.12, 0.03, 0.05])
    q = [math.cos(phi / 2), 0, 0, math.sin(phi / 2)]
    sc = _scene([[0, 0, z]], [s], [q], [0.8], [[1, 1, 1]], [[1.0]])
    pr, _, _, fw = ora.render_full(cam, sc)
    s64 = sc.scales[0].astype(np.float64)
    q64 = sc.quats[0].astype(np.float64)
    q64 /= np.linalg.norm(q64)
    ang = 2 * math.atan2(q64[3], q64[0])
    Rz = np.array([[math.cos(ang), -math.sin(ang)], [math.sin(ang), math.cos(ang)]])
    cov = (cam.fx / z) ** 2 * Rz @ np.diag(s64[:2] ** 2) @ Rz.T + 0.3 * np.eye(2)
    K = np.linalg.inv(cov)
    assert np.allclose(pr["conic"][0], [K[0, 0], K[0, 1], K[1, 1]], rtol=1e-11)
    px, py = _pix_centres(cam)
    d = np.stack([cam.cx - px, cam.cy - py], -1)
    power = -0.5 * np.einsum("...i,ij,...j->...", d, K, d)
    alpha = np.minimum(0.99, float(sc.opacity[0]) * np.exp(power))
    alpha = np.where(alpha >= 1 / 255, alpha, 0.0)
    tx0, ty0, tx1, ty1 = pr["rect"][0]
    in_rect = (px >= 16 * tx0) & (px < 16 * tx1) & (py >= 16 * ty0) & (py < 16 * ty1)
    alpha = np.where(in_rect, alpha, 0.0)
    assert np.allclose(fw["alpha"], alpha, rtol=1e-12, atol=1e-15)
    # the footprint is elongated along the rolled major axis
    assert K[0, 1] != 0 and np.sign(K[0, 1]) == -np.sign(math.sin(2 * ang))


def test_two_gaussians_front_to_back(ora, sg):
    """Eq. 2 with two layers: C = a1 c1 + a2 (1 - a1) c2, nearer one first,
    whatever their order in the input."""
    cam = sg.identity_camera(32, 32, 40.0)
    sc = _scene([[0, 0, 3.0], [0, 0, 2.0]], [[0.1, 0.1, 0.1], [0.08, 0.08, 0.08]],
                [[1, 0, 0, 0], [1, 0, 0, 0]], [0.6, 0.5], [[1, 0, 0], [0, 1, 0]], [[1.0], [2.0]])
    pr, _, gids, fw = ora.render_full(cam, sc)
    px, py = _pix_centres(cam)
    a = []
    for g in range(2):
        cv = pr["cov"][g]
        al = float(sc.opacity[g]) * np.exp(-0.5 * ((cam.cx - px) ** 2 / cv[0] + (cam.cy - py) ** 2 / cv[2]))
        a.append(np.where(al >= 1 / 255, np.minimum(al, 0.99), 0.0))
    near, far = a[1], a[0]                 # gaussian 1 is nearer (z=2)
    exp_r = far * (1 - near) * 1.0
    exp_g = near * 1.0
    assert np.allclose(fw["rgb"][0], exp_r, atol=1e-14)
    assert np.allclose(fw["rgb"][1], exp_g, atol=1e-14)
    assert np.allclose(fw["depth"], near * 2.0 + far * (1 - near) * 3.0, atol=1e-13)
    assert np.allclose(fw["feat"][0], near * 2.0 + far * (1 - near) * 1.0, atol=1e-13)


def test_weights_sum_and_feature_copies(ora, sg):
    """sum_i w_i + T_final = 1 and features (c, d, 1) reproduce C - T bg, D, A."""
    sc, cam = sg.small_case(seed=11, P=600, N=0)
    pr = ora.project_f64(cam, sc.means, sc.scales, sc.quats, sc.opacity)
    feats = np.concatenate([sc.colors.astype(np.float64), pr["depth"][:, None], np.ones((sc.P, 1))], 1)
    bg = (0.3, 0.1, 0.7)
    _, _, _, fw = ora.render_full(cam, sc, bg=bg, feats=feats)
    assert np.abs(fw["feat"][4] + fw["T_final"] - 1).max() < 1e-12
    assert np.abs(fw["alpha"] - fw["feat"][4]).max() < 1e-12
    for ch in range(3):
        assert np.abs(fw["feat"][ch] - (fw["rgb"][ch] - fw["T_final"] * bg[ch])).max() < 1e-12
    assert np.abs(fw["feat"][3] - fw["depth"]).max() < 1e-12
    assert fw["n_contrib"].max() > 5 and (fw["T_final"] >= 1e-4).all()


def test_tile_rect_and_lists_brute_force(ora, sg):
    """Rectangles from pixel enumeration; lists by O(n^2) pairwise ordering."""
    for seed in (21, 22, 23):
        sc, cam = sg.small_case(seed=seed, P=40, N=0)
        pr = ora.project_f64(cam, sc.means, sc.scales, sc.quats, sc.opacity)
        px, py = _pix_centres(cam)
        tiles = {}
        for g in range(sc.P):
            if pr["touched"][g] == 0:
                continue
            u, v = pr["uv"][g]
            r = pr["radius"][g]
            m = (np.abs(px - u) <= r) & (np.abs(py - v) <= r)
            ts = set(zip(*np.nonzero(m)))
            tset = {(int(j) // 16) * cam.tiles_x + int(i) // 16 for j, i in ts}
            x0, y0, x1, y1 = pr["rect"][g]
            rset = {ty * cam.tiles_x + tx for ty in range(y0, y1) for tx in range(x0, x1)}
            assert tset == rset, (seed, g)
            for t in rset:
                tiles.setdefault(t, []).append(g)
        ranges, gids = ora.bin_lists(cam, pr["rect"], pr["depth"])
        for t in range(cam.num_tiles):
            members = tiles.get(t, [])
            # position of g = number of members strictly before it in (depth, id)
            want = [None] * len(members)
            for g in members:
                k = sum(1 for h in members if (pr["depth"][h], h) < (pr["depth"][g], g))
                want[k] = g
            s, e = ranges[t]
            assert list(gids[s:e]) == want, (seed, t)


def test_b32_replay_matches_definition(ora, sg):
    """The binary32 replay agrees with the double-precision definition up to
    the conditioning of the 2D covariance; rectangles agree except at
    half-pixel ties."""
    sc, cam = sg.small_case(seed=31, P=3000, N=0)
    a = ora.project_f64(cam, sc.means, sc.scales, sc.quats, sc.opacity)
    b = ora.project_b32(cam.as_f32(), sc.means, sc.scales, sc.quats, sc.opacity)
    vis = a["touched"] > 0
    assert ((b["touched"] > 0) == vis).mean() > 0.995
    both = vis & (b["touched"] > 0)
    assert np.abs(b["uv"][both] - a["uv"][both]).max() < 1e-3
    assert np.max(np.abs(b["depth"][both] - a["depth"][both]) / a["depth"][both]) < 1e-6
    cn = np.linalg.norm(a["conic"][both], axis=1)
    err = np.linalg.norm(b["conic"][both] - a["conic"][both], axis=1) / cn
    assert np.median(err) < 1e-5 and err.max() < 1e-2
    assert (b["rect"][both] == a["rect"][both]).all(1).mean() > 0.99


def _quat_of_rot(R):
    w = math.sqrt(max(0.0, 1 + R[0, 0] + R[1, 1] + R[2, 2])) / 2
    x = math.copysign(math.sqrt(max(0.0, 1 + R[0, 0] - R[1, 1] - R[2, 2])) / 2, R[2, 1] - R[1, 2])
    y = math.copysign(math.sqrt(max(0.0, 1 - R[0, 0] + R[1, 1] - R[2, 2])) / 2, R[0, 2] - R[2, 0])
    z = math.copysign(math.sqrt(max(0.0, 1 - R[0, 0] - R[1, 1] + R[2, 2])) / 2, R[1, 0] - R[0, 1])
    return np.array([w, x, y, z])


def _qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b.T
    return np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], 1)


def test_rigid_reexpression(ora, sg):
    """Rendering world Gaussians at pose (R, t) equals rendering the same
    Gaussians moved into the camera frame (means R mu + t, orientation
    R q) at the identity pose."""
    sc, _ = sg.room_case(seed=41, P=4000, N=2)
    cam = sg.room_trajectory(17, width=96, height=64, f=48.0)
    m64 = sc.means.astype(np.float64)
    q64 = sc.quats.astype(np.float64)
    q64 /= np.linalg.norm(q64, axis=1, keepdims=True)
    means_c = m64 @ cam.R.T + cam.t
    quats_c = _qmul(_quat_of_rot(cam.R), q64)
    cam_id = Camera(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, np.eye(3), np.zeros(3))
    # the oracle takes doubles; feed exact double arrays through a float64 scene
    sc_c = Scene(means_c, sc.scales.astype(np.float64), quats_c, sc.opacity.astype(np.float64),
                 sc.colors.astype(np.float64), sc.feats.astype(np.float64))
    sc_w = Scene(m64, sc.scales.astype(np.float64), q64, sc.opacity.astype(np.float64),
                 sc.colors.astype(np.float64), sc.feats.astype(np.float64))
    pa, _, _, fa = ora.render_full(cam, sc_w)
    pb, _, _, fb = ora.render_full(cam_id, sc_c)
    assert (pa["rect"] == pb["rect"]).all()
    assert np.allclose(pa["conic"], pb["conic"], rtol=1e-9, atol=1e-12)
    assert fa["n_contrib"].sum() > 1000
    ok = np.minimum(fa["margin"], fb["margin"]) > 1e-7
    assert ok.mean() > 0.999
    for k in ("rgb", "feat"):
        assert np.abs(fa[k] - fb[k])[..., ok].max() < 1e-9
    assert np.abs(fa["depth"] - fb["depth"])[ok].max() < 1e-9


def _fd_setup(sg, seed=5):
    sc, cam = sg.fd_case(seed=seed)
    H, W, N = cam.height, cam.width, sc.N
    g = sg.random_linear_functional(seed + 100, H, W, N)
    g = tuple(x.astype(np.float64) for x in g)
    sc64 = Scene(*(a.astype(np.float64) for a in (sc.means, sc.scales, sc.quats, sc.opacity, sc.colors,
                                                   sc.feats)))
    return sc64, cam, g


def _loss(ora, cam, sc, g):
    pr, ranges, gids, fw = ora.render_full(cam, sc, bg=(0.2, 0.4, 0.1))
    key = (fw["n_contrib"].tobytes(), fw["last_idx"].tobytes(), pr["rect"].tobytes(), gids.tobytes())
    return ora.linear_loss(fw, *g), key


def test_finite_differences_all_parameter_classes(ora, sg):
    """FP64 central differences (h = 1e-6) of a random linear functional of
    all outputs against the analytic adjoint in coupled mode, for means,
    scales, quaternions, opacities, colours, features and the pose tangent.
    Coordinates whose +-h evaluations change a discrete decision are skipped
    (and counted)."""
    sc, cam, g = _fd_setup(sg)
    _, _, _, _, grads = ora.render_full_grad(cam, sc, *g, coupled=True, bg=(0.2, 0.4, 0.1))
    rng = np.random.default_rng(7)
    h = 1e-6
    skipped = checked = 0
    worst = {}
    visible = np.nonzero(grads["opacity"] != 0)[0]
    for name, arr in (("means", sc.means), ("scales", sc.scales), ("quats", sc.quats),
                      ("opacity", sc.opacity), ("colors", sc.colors), ("feats", sc.feats)):
        picks = rng.choice(visible, size=12, replace=False)
        for gidx in picks:
            cols = [None] if arr.ndim == 1 else list(rng.choice(arr.shape[1], size=min(arr.shape[1], 3),
                                                                replace=False))
            for col in cols:
                idx = gidx if col is None else (gidx, col)
                orig = arr[idx]
                arr[idx] = orig + h
                lp, kp = _loss(ora, cam, sc, g)
                arr[idx] = orig - h
                lm, km = _loss(ora, cam, sc, g)
                arr[idx] = orig
                if kp != km:
                    skipped += 1
                    continue
                fd = (lp - lm) / (2 * h)
                an = grads[name][idx]
                err = abs(fd - an) / max(abs(an), 1e-3 * np.abs(grads[name]).max(), 1e-9)
                worst[name] = max(worst.get(name, 0.0), err)
                checked += 1
    # pose: left perturbation by Exp(h e_k)
    for k in range(6):
        tau = np.zeros(6)
        tau[k] = h
        lp, kp = _loss(ora, sg.perturb_pose(cam, tau[:3], tau[3:]), sc, g)
        lm, km = _loss(ora, sg.perturb_pose(cam, -tau[:3], -tau[3:]), sc, g)
        assert kp == km
        fd = (lp - lm) / (2 * h)
        an = grads["pose"][k]
        worst["pose"] = max(worst.get("pose", 0.0), abs(fd - an) / max(abs(an), 1e-9))
        checked += 1
    assert checked > 150 and skipped < 0.1 * checked, (checked, skipped)
    for name, err in worst.items():
        assert err < 2e-5, (name, err, worst)


def test_decoupled_feature_gradient(ora, sg):
    """Sec. 3.1: the feature cotangent reaches f only. Decoupled geometry
    gradients equal coupled ones with g_F = 0; feature gradients equal in
    both modes and are exactly linear (F is linear in f)."""
    sc, cam, g = _fd_setup(sg, seed=6)
    g_rgb, g_d, g_a, g_f = g
    _, _, _, fw, dec = ora.render_full_grad(cam, sc, g_rgb, g_d, g_a, g_f, coupled=False)
    _, _, _, _, cou0 = ora.render_full_grad(cam, sc, g_rgb, g_d, g_a, np.zeros_like(g_f), coupled=True)
    _, _, _, _, cou = ora.render_full_grad(cam, sc, g_rgb, g_d, g_a, g_f, coupled=True)
    for k in ("means", "scales", "quats", "opacity", "colors", "pose"):
        assert np.allclose(dec[k], cou0[k], rtol=1e-12, atol=1e-12), k
    assert np.allclose(dec["feats"], cou["feats"], rtol=1e-12, atol=1e-12)
    assert not np.allclose(dec["opacity"], cou["opacity"])
    # linearity: <g_F, F(f)> = <d_feats, f>
    lhs = float((g_f * fw["feat"]).sum())
    rhs = float((dec["feats"] * sc.feats).sum())
    assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(lhs))


def test_pose_translation_equals_rotated_mean_sum(ora, sg):
    """drho = R sum_i dmu_i, since mu_c = R mu + t (Eq. 4, first block)."""
    sc, _ = sg.room_case(seed=51, P=3000, N=0)
    cam = sg.room_trajectory(3, width=96, height=64, f=48.0)
    g = sg.random_linear_functional(52, cam.height, cam.width, 0)
    _, _, _, _, gr = ora.render_full_grad(cam, sc, g[0], g[1], g[2], None)
    lhs = gr["pose"][:3]
    rhs = cam.R @ gr["means"].sum(0)
    assert np.abs(lhs).max() > 1e-3
    assert np.allclose(lhs, rhs, rtol=1e-10, atol=1e-12)


def test_finite_differences_guard_band(ora, sg):
    """Large Gaussians centred outside the guard band (|x/z| > 1.3 tan(fov/2))
    whose footprint still reaches the image: pins the derivative of the
    clamped Jacobian entries (the clamped x' = +-lim z depends on z)."""
    cam = sg.identity_camera(64, 48, 50.0)
    rng = sg.Rng(61)
    P = 24
    z = 1.5 + 2.0 * rng.uniform(P)
    limx, limy = 1.3 * 64 / 100.0, 1.3 * 48 / 100.0
    side = np.where(rng.uniform(P) < 0.5, -1.0, 1.0)
    tx = side * limx * (1.04 + 0.15 * rng.uniform(P))
    ty = (rng.uniform(P) - 0.5) * 2 * limy * 1.1
    means = np.stack([tx * z, ty * z, z], 1)
    scales = np.exp(np.log(0.35) + 0.2 * rng.normal(3 * P)).reshape(P, 3)
    q = rng.normal(4 * P).reshape(P, 4)
    sc = Scene(means, scales, q / np.linalg.norm(q, axis=1, keepdims=True), 0.3 + 0.5 * rng.uniform(P),
               rng.uniform(3 * P).reshape(P, 3), rng.normal(2 * P).reshape(P, 2))
    g = tuple(x.astype(np.float64) for x in sg.random_linear_functional(62, cam.height, cam.width, 2))
    _, _, _, fw, grads = ora.render_full_grad(cam, sc, *g, coupled=True, bg=(0.2, 0.4, 0.1))
    vis = np.nonzero(grads["opacity"] != 0)[0]
    assert len(vis) >= 8 and fw["n_contrib"].sum() > 500
    h = 1e-6
    worst = 0.0
    n = 0
    for gi in vis:
        for col in range(3):
            orig = sc.means[gi, col]
            sc.means[gi, col] = orig + h
            lp, kp = _loss(ora, cam, sc, g)
            sc.means[gi, col] = orig - h
            lm, km = _loss(ora, cam, sc, g)
            sc.means[gi, col] = orig
            if kp != km:
                continue
            an = grads["means"][gi, col]
            worst = max(worst, abs((lp - lm) / (2 * h) - an) / max(abs(an), 1e-3 * np.abs(grads["means"]).max()))
            n += 1
    assert n >= 20 and worst < 2e-5, (n, worst)


def test_stop_rule_closed_form(ora, sg):
    """Four broad, near-opaque layers on the axis. Where the third layer
    would take T below 1e-4 it is not blended and the walk stops: C, T_final
    and the contributor count follow from the first two layers alone."""
    cam = sg.identity_camera(32, 32, 40.0)
    zs = [2.0, 2.5, 3.0, 3.5]
    cols = [[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]]
    sc = _scene([[0, 0, z] for z in zs], [[1.5, 1.5, 1.5]] * 4, [[1, 0, 0, 0]] * 4, [0.99] * 4, cols,
                [[1.0]] * 4)
    pr, _, _, fw = ora.render_full(cam, sc)
    px, py = _pix_centres(cam)
    al = []
    for g in range(4):
        cv = pr["cov"][g]
        a = float(sc.opacity[g]) * np.exp(-0.5 * ((cam.cx - px) ** 2 / cv[0] + (cam.cy - py) ** 2 / cv[2]))
        al.append(np.minimum(a, 0.99))
    T2 = (1 - al[0]) * (1 - al[1])
    stop3 = T2 * (1 - al[2]) < 1e-4
    assert stop3.sum() > 50
    assert (fw["n_contrib"][stop3] == 2).all()
    assert np.allclose(fw["T_final"][stop3], T2[stop3], rtol=1e-12)
    assert np.allclose(fw["rgb"][1][stop3], (al[1] * (1 - al[0]))[stop3], rtol=1e-12)
    assert np.allclose(fw["rgb"][2][stop3], 0.0)


# ---- keyframe visibility (Sec. 3.2): blended somewhere with T > 0.5 in front --

def test_visibility_behind_opaque_and_translucent_layer(ora, sg):
    """A wide front Gaussian covers the whole 32x32 image with alpha_f(p),
    a small one sits behind it on the axis. The largest transmittance in
    front of the back one is max over its blended pixels of 1 - alpha_f(p):
    exactly 1 - 0.99 when the front one is clamped (o = 0.995, invisible
    behind it), about 0.7 when o = 0.3 (visible). The front one is first at
    every pixel: T = 1 in front."""
    cam = sg.identity_camera(32, 32, 40.0)
    px, py = _pix_centres(cam)
    for o_front, visible_back in ((0.995, False), (0.3, True)):
        sc = _scene([[0, 0, 1.5], [0, 0, 3.0]], [[50.0, 50.0, 50.0], [0.1, 0.1, 0.1]],
                    [[1, 0, 0, 0], [1, 0, 0, 0]], [o_front, 0.7], [[1, 0, 0], [0, 1, 0]], [[0.0], [0.0]])
        pr = ora.project_f64(cam, sc.means, sc.scales, sc.quats, sc.opacity)
        ranges, gids = ora.bin_lists(cam, pr["rect"], pr["depth"])
        maxT = ora.visibility(cam, ranges, gids, pr["uv"], pr["conic"], sc.opacity)
        assert maxT[0] == 1.0
        cf, cb = pr["cov"][0], pr["cov"][1]
        a_f = np.minimum(0.99, float(sc.opacity[0]) * np.exp(-0.5 * ((cam.cx - px) ** 2 / cf[0] +
                                                                      (cam.cy - py) ** 2 / cf[2])))
        a_b = float(sc.opacity[1]) * np.exp(-0.5 * ((cam.cx - px) ** 2 / cb[0] + (cam.cy - py) ** 2 / cb[2]))
        tx0, ty0, tx1, ty1 = pr["rect"][1]
        in_rect = (px >= 16 * tx0) & (px < 16 * tx1) & (py >= 16 * ty0) & (py < 16 * ty1)
        blended = in_rect & (a_b >= 1 / 255)
        assert blended.sum() > 10
        want = float((1 - a_f)[blended].max())
        assert abs(maxT[1] - want) < 1e-14, (maxT[1], want)
        assert (maxT[1] > 0.5) == visible_back
    assert abs((1 - 0.99) - 0.01) < 1e-15


def _walk_max_T(cam, pr, ranges, gids, opac):
    """Eq. 2's front-to-back walk written out again in numpy, one tile at a
    time over its pixels: the largest T in front of each blended Gaussian."""
    P = pr["uv"].shape[0]
    out = np.zeros(P)
    px_all, py_all = _pix_centres(cam)
    for t in range(cam.tiles_x * cam.tiles_y):
        s, e = ranges[t]
        tx, ty = t % cam.tiles_x, t // cam.tiles_x
        px = px_all[16 * ty:16 * ty + 16, 16 * tx:16 * tx + 16].ravel()
        py = py_all[16 * ty:16 * ty + 16, 16 * tx:16 * tx + 16].ravel()
        T = np.ones(px.shape)
        done = np.zeros(px.shape, bool)
        for g in gids[s:e]:
            A, B, C = pr["conic"][g]
            dx, dy = pr["uv"][g, 0] - px, pr["uv"][g, 1] - py
            power = -0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy
            alpha = np.minimum(0.99, opac[g] * np.exp(power))
            ok = (power <= 0) & (alpha >= 1 / 255) & ~done
            Tn = T * (1 - alpha)
            stop = ok & (Tn < 1e-4)
            bl = ok & ~stop
            if bl.any():
                out[g] = max(out[g], T[bl].max())
            done |= stop
            T = np.where(bl, Tn, T)
    return out


def test_visibility_brute_force(ora, sg):
    """The oracle's per-Gaussian max T against the walk written out in numpy
    on a random frustum scene; visibility (> 0.5) agrees exactly."""
    sc, cam = sg.small_case(seed=21, P=2000, N=0)
    pr = ora.project_f64(cam, sc.means, sc.scales, sc.quats, sc.opacity)
    ranges, gids = ora.bin_lists(cam, pr["rect"], pr["depth"])
    maxT = ora.visibility(cam, ranges, gids, pr["uv"], pr["conic"], sc.opacity)
    want = _walk_max_T(cam, pr, ranges, gids, sc.opacity.astype(np.float64))
    assert np.abs(maxT - want).max() < 1e-12
    vis = maxT > 0.5
    assert 20 < vis.sum() < sc.P and (maxT[~vis] > 0).any()
    assert np.array_equal(vis, want > 0.5)
