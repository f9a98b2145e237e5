"""Pins of the oracle's semantic pieces (Sec. 3.3): the Eq. 9 cross-entropy
on per-pixel logits, the Eq. 10 argmax and the Eq. 12 label probabilities.

* closed forms: two classes give loss = softplus(b - a) for label 0 and the
  gradient (sigmoid(a - b) - 1, sigmoid(b - a)) / HW; identity queries make
  the label probabilities the softmax of the features themselves;
* invariants: adding a constant to all of a pixel's logits changes nothing,
  the gradient sums to zero over the channels, ignored pixels give nothing,
  CHW and HWC agree, probabilities sum to one;
* finite differences of the loss;
* the binary32 replay of the logits against exact rational arithmetic
  (fractions) rounded once per fused multiply-add.
"""
import math
from fractions import Fraction

import numpy as np


def test_two_class_closed_form(ora):
    a, b = 0.3, -1.2
    feat = np.array([[[a]], [[b]]])          # [N=2, H=1, W=1]
    loss, g = ora.semantic_ce(feat, np.array([[0]]))
    assert abs(loss - math.log1p(math.exp(b - a))) < 1e-15
    s = 1 / (1 + math.exp(-(a - b)))
    assert abs(g[0, 0, 0] - (s - 1)) < 1e-15 and abs(g[1, 0, 0] - (1 - s)) < 1e-15


def test_ce_invariants(ora):
    rng = np.random.default_rng(3)
    N, H, W = 7, 5, 6
    feat = rng.normal(size=(N, H, W)) * 3
    labels = rng.integers(-1, N, size=(H, W)).astype(np.int32)
    labels[0, 0] = N        # out of range: ignored as well
    loss, g = ora.semantic_ce(feat, labels)
    ign = (labels < 0) | (labels >= N)
    assert ign.sum() >= 2 and not g[:, ign].any()
    assert np.abs(g.sum(0)).max() < 1e-15
    shift = rng.normal(size=(1, H, W)) * 50
    loss2, g2 = ora.semantic_ce(feat + shift, labels)
    assert abs(loss2 - loss) < 1e-12 and np.abs(g2 - g).max() < 1e-15
    loss3, g3 = ora.semantic_ce(np.transpose(feat, (1, 2, 0)), labels, hwc=True)
    assert abs(loss3 - loss) < 1e-15 and np.abs(np.transpose(g3, (2, 0, 1)) - g).max() < 1e-17


def test_ce_finite_differences(ora):
    rng = np.random.default_rng(4)
    N, H, W = 5, 3, 4
    feat = rng.normal(size=(N, H, W))
    labels = rng.integers(0, N, size=(H, W)).astype(np.int32)
    _, g = ora.semantic_ce(feat, labels)
    h = 1e-6
    for idx in [(0, 0, 0), (3, 1, 2), (4, 2, 3), (1, 2, 0)]:
        fp, fm = feat.copy(), feat.copy()
        fp[idx] += h
        fm[idx] -= h
        fd = (ora.semantic_ce(fp, labels)[0] - ora.semantic_ce(fm, labels)[0]) / (2 * h)
        assert abs(fd - g[idx]) < 1e-8


def test_argmax_ties_take_the_lowest_channel(ora):
    feat = np.array([[[1.0, 2.0]], [[3.0, 2.0]], [[3.0, -1.0]]], np.float32)   # [3,1,2]
    assert np.array_equal(ora.argmax_labels(feat), [[1, 0]])
    assert np.array_equal(ora.argmax_labels(np.transpose(feat, (1, 2, 0)), hwc=True), [[1, 0]])


def test_label_probs_closed_form_and_invariants(ora):
    rng = np.random.default_rng(5)
    M = 8
    f = rng.normal(size=(20, M))
    p = ora.label_probs(f, np.eye(M))
    e = np.exp(f - f.max(1, keepdims=True))
    assert np.abs(p - e / e.sum(1, keepdims=True)).max() < 1e-15
    q = rng.normal(size=(5, M))
    p = ora.label_probs(f, q)
    assert np.abs(p.sum(1) - 1).max() < 1e-15
    # a constant feature channel whose query entries all equal c adds c to
    # every logit of a pixel: the probabilities do not change
    f2 = np.concatenate([f, np.ones((20, 1))], 1)
    q2 = np.concatenate([q, np.full((5, 1), 0.0)], 1)
    q3 = np.concatenate([q, np.full((5, 1), 7.5)], 1)
    assert np.abs(ora.label_probs(f2, q2) - ora.label_probs(f2, q3)).max() < 1e-13


def test_label_logits_b32_against_exact_rounding(ora):
    """Each step rounds the exact value of fma(f, q, acc) to binary32 once;
    recompute that exactly with fractions and numpy's float32 rounding."""
    rng = np.random.default_rng(6)
    f = rng.normal(size=(3, 12)).astype(np.float32)
    q = rng.normal(size=(2, 12)).astype(np.float32)
    z = ora.label_logits_b32(f, q)
    for p in range(3):
        for l in range(2):
            acc = np.float32(0)
            for c in range(12):
                exact = Fraction(float(f[p, c])) * Fraction(float(q[l, c])) + Fraction(float(acc))
                # nearest binary32 of the exact value: via double when it is
                # exact in double, else by comparing the two float32 neighbours
                d = float(exact)
                cand = np.float32(d)
                lo, hi = np.nextafter(cand, np.float32(-np.inf)), np.nextafter(cand, np.float32(np.inf))
                acc = min((lo, cand, hi), key=lambda v: (abs(Fraction(float(v)) - exact),
                                                         int(np.float32(v).view(np.uint32)) & 1))
            assert z[p, l] == acc
