"""Pins of the oracle's spherical-harmonic colour (Sec. 3.1).

* the basis against the real harmonics built from scipy.special.sph_harm_y
  (sqrt2 Re / Im of the complex Y_l^|m|, Condon-Shortley phase included);
* orthonormality on the sphere by a product quadrature (Gauss-Legendre in
  z, uniform in the azimuth) that is exact for these degrees;
* closed forms: degree 0 gives the same colour from every view, a negative
  channel is clamped to 0 and passes no gradient;
* finite differences of the adjoint in the coefficients, the means and the
  pose (through the left perturbation of the camera).
"""
import math

import numpy as np
import pytest

from paper_2504_19409_gb300.scenegen import Camera

special = pytest.importorskip("scipy.special")


def _dirs(n, seed):
    d = np.random.default_rng(seed).normal(size=(n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def test_basis_matches_scipy_real_harmonics(ora):
    d = _dirs(50, 1)
    Y = ora.sh_basis(d)
    th, ph = np.arccos(d[:, 2]), np.arctan2(d[:, 1], d[:, 0])
    for l in range(4):
        for m in range(-l, l + 1):
            z = special.sph_harm_y(l, abs(m), th, ph)
            want = z.real if m == 0 else math.sqrt(2) * (z.real if m > 0 else z.imag)
            assert np.abs(Y[:, l * l + l + m] - want).max() < 1e-13, (l, m)


def test_basis_orthonormal_on_the_sphere(ora):
    zs, wz = np.polynomial.legendre.leggauss(12)
    nphi = 24
    phi = 2 * np.pi * np.arange(nphi) / nphi
    Z, PH = np.meshgrid(zs, phi, indexing="ij")
    r = np.sqrt(1 - Z ** 2)
    d = np.stack([r * np.cos(PH), r * np.sin(PH), Z], -1).reshape(-1, 3)
    w = (wz[:, None] * np.full(nphi, 2 * np.pi / nphi)[None, :]).ravel()
    Y = ora.sh_basis(d)
    G = (Y * w[:, None]).T @ Y
    assert np.abs(G - np.eye(16)).max() < 1e-12


def _cam(seed):
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    return Camera(64, 48, 50.0, 50.0, 32.0, 24.0, q, rng.normal(size=3))


def test_degree_zero_is_view_independent_and_clamped(ora):
    c0 = 0.5 / math.sqrt(math.pi)
    means = np.random.default_rng(2).normal(size=(6, 3)) * 3
    sh = np.zeros((6, 1, 3))
    sh[:, 0] = [[1.0, -2.0, 0.3]]
    for seed in (3, 4):
        col = ora.sh_colors(_cam(seed), means, sh)
        assert np.allclose(col, np.maximum(c0 * sh[:, 0] + 0.5, 0), atol=1e-15)
    d_sh, _, _ = ora.sh_colors_bwd(_cam(3), means, sh, np.ones((6, 3)))
    assert np.allclose(d_sh[:, 0, 0], c0) and not d_sh[:, 0, 1].any()  # channel 1 is clamped


def test_adjoint_finite_differences(ora, sg):
    rng = np.random.default_rng(5)
    P = 7
    cam = _cam(6)
    means = rng.normal(size=(P, 3)) * 2
    sh = rng.normal(size=(P, 16, 3)) * 0.3
    sh[:, 0] += 3.0  # stay above the clamp
    G = rng.normal(size=(P, 3))
    loss = lambda c, m, s: float((ora.sh_colors(c, m, s) * G).sum())
    d_sh, d_means, d_pose = ora.sh_colors_bwd(cam, means, sh, G)
    h = 1e-6
    for idx in [(0, 0, 0), (2, 5, 1), (6, 15, 2), (4, 9, 0)]:
        a, b = sh.copy(), sh.copy()
        a[idx] += h
        b[idx] -= h
        assert abs((loss(cam, means, a) - loss(cam, means, b)) / (2 * h) - d_sh[idx]) < 1e-8
    for idx in [(0, 0), (3, 1), (6, 2)]:
        a, b = means.copy(), means.copy()
        a[idx] += h
        b[idx] -= h
        fd = (loss(cam, a, sh) - loss(cam, b, sh)) / (2 * h)
        assert abs(fd - d_means[idx]) < 1e-7 * max(1.0, abs(fd))
    for i in range(6):
        e = np.zeros(6)
        e[i] = h
        cp = sg.perturb_pose(cam, e[:3], e[3:])
        cm = sg.perturb_pose(cam, -e[:3], -e[3:])
        fd = (loss(cp, means, sh) - loss(cm, means, sh)) / (2 * h)
        assert abs(fd - d_pose[i]) < 1e-7 * max(1.0, abs(fd)), (i, fd, d_pose[i])
    assert np.abs(d_pose[:3]).max() > 1e-3 and not d_pose[3:].any()
