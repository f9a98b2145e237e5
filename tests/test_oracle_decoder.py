"""Pins of the oracle's per-pixel decoder (Eq. 11 read as a 1x1 lift,
y = W2^T gelu(W1^T z + b1) + b2 with the exact erf GELU)."""
import math

import numpy as np


def _params(rng, din=16, dh=128, dout=64):
    return (rng.normal(size=(din, dh)) / math.sqrt(din), rng.normal(size=dh) * 0.1,
            rng.normal(size=(dh, dout)) / math.sqrt(dh), rng.normal(size=dout) * 0.1)


def test_gelu_closed_form_values(ora):
    """One hidden unit with unit weights: y = gelu(z). gelu(0) = 0,
    gelu(1) = Phi(1) = (1 + erf(1/sqrt2))/2 = 0.8413447460685429,
    gelu(-1) = -(1 - 0.8413447460685429), gelu(x) -> x for large x."""
    z = np.array([[0.0], [1.0], [-1.0], [8.0], [-8.0]])
    y = ora.decoder_fwd(z, np.ones((1, 1)), np.zeros(1), np.ones((1, 1)), np.zeros(1))[:, 0]
    assert abs(y[0]) < 1e-15
    assert abs(y[1] - 0.8413447460685429) < 1e-15
    assert abs(y[2] + (1 - 0.8413447460685429)) < 1e-15
    assert abs(y[3] - 8.0) < 1e-12 and abs(y[4]) < 1e-12


def test_linear_regime_is_affine(ora):
    """With large positive pre-activations gelu is the identity, so the
    decoder reduces to the affine map z -> W2^T (W1^T z + b1) + b2."""
    rng = np.random.default_rng(1)
    W1, b1, W2, b2 = _params(rng)
    W1 = np.abs(W1) * 0.01
    b1 = b1 * 0 + 40.0
    z = np.abs(rng.normal(size=(20, 16)))
    y = ora.decoder_fwd(z, W1, b1, W2, b2)
    assert np.allclose(y, (z @ W1 + b1) @ W2 + b2, rtol=1e-12, atol=1e-10)


def test_decoder_finite_differences(ora):
    rng = np.random.default_rng(2)
    W1, b1, W2, b2 = _params(rng, dout=24)
    z = rng.normal(size=(7, 16))
    g = rng.normal(size=(7, 24))
    gr = ora.decoder_bwd(z, W1, b1, W2, g)
    L = lambda z_, W1_, b1_, W2_, b2_: float((g * ora.decoder_fwd(z_, W1_, b1_, W2_, b2_)).sum())
    h = 1e-6
    args = dict(z=z, W1=W1, b1=b1, W2=W2, b2=b2)
    order = ("z", "W1", "b1", "W2", "b2")
    worst = 0.0
    for name in order:
        arr = args[name]
        for idx in [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(12)]:
            orig = arr[idx]
            arr[idx] = orig + h
            lp = L(*(args[k] for k in order))
            arr[idx] = orig - h
            lm = L(*(args[k] for k in order))
            arr[idx] = orig
            fd = (lp - lm) / (2 * h)
            an = gr[name][idx]
            worst = max(worst, abs(fd - an) / max(abs(an), 1e-6))
    assert worst < 1e-6, worst
