"""Learned decoder o(.) (Eq. 11 as a per-pixel 1x1 lift, 16 -> 128 -> 512,
exact-erf GELU, bf16 weights, fp32 accumulation) on the GPU vs the FP64
oracle, and what training it gains.

Bars: forward and gradients within 1e-5 / 1e-4 (normwise) of the oracle on
the same bf16 weights (products of bf16 values are exact in fp32; the rest is
fp32 accumulation over <= 2000 samples). Sample indices are reproduced here
from splitmix64's published definition, independently of the kernel.
"""
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

GOLD = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1


def _normal_(t, sd, seed):
    """Fill t with N(0, sd^2) draws of a seeded numpy generator (independent of
    the torch generators' state, hence of which tests ran before)."""
    t.copy_(torch.from_numpy(np.random.default_rng(seed).normal(0.0, sd, size=tuple(t.shape)).astype(np.float32)))


def _splitmix(z):
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9 & M64
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB & M64
    return z ^ (z >> 31)


def _samples(seed, S, npix):
    return np.array([_splitmix((seed + (s + 1) * GOLD) & M64) % npix for s in range(S)], dtype=np.int64)


@pytest.fixture(scope="module")
def dec_mod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_19409_gb300 import build
    build.build()
    import paper_2504_19409_gb300.decoder as d
    return d


def _np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def test_decoder_forward_matches_oracle(dec_mod, ora):
    dec = dec_mod.Decoder(seed=3)
    _normal_(dec.params["b1"], 0.1, 101)
    _normal_(dec.params["b2"], 0.1, 102)
    rng = np.random.default_rng(4)
    z = torch.tensor(rng.normal(size=(3000, 16)).astype(np.float32), device="cuda")
    y = dec.forward(z)
    torch.cuda.synchronize()
    ref = ora.decoder_fwd(_np(z), _np(dec.work["W1"]), _np(dec.params["b1"]), _np(dec.work["W2"]),
                          _np(dec.params["b2"]))
    err = np.linalg.norm(_np(y) - ref) / np.linalg.norm(ref)
    assert err < 1e-5, err
    assert np.abs(_np(y) - ref).max() < 1e-4 * np.abs(ref).max()


def test_decoder_training_gradients_match_oracle(dec_mod, ora):
    dec = dec_mod.Decoder(seed=5)
    _normal_(dec.params["b1"], 0.1, 103)
    rng = np.random.default_rng(6)
    npix, S, seed = 2500, 2000, 77
    z = torch.tensor(rng.normal(size=(npix, 16)).astype(np.float32), device="cuda")
    tgt = torch.tensor(rng.normal(size=(npix, 512)).astype(np.float32), device="cuda")
    dz = torch.zeros(npix, 16, device="cuda")
    loss = torch.zeros(1, device="cuda")
    scale = 1.0 / (S * 512)
    dec.zero_grad()
    dec.train_eval(z, tgt, S, seed, scale, dz_map=dz, loss=loss)
    torch.cuda.synchronize()
    idx = _samples(seed, S, npix)
    W1, b1, W2, b2 = _np(dec.work["W1"]), _np(dec.params["b1"]), _np(dec.work["W2"]), _np(dec.params["b2"])
    zs, ts = _np(z)[idx], _np(tgt)[idx]
    y = ora.decoder_fwd(zs, W1, b1, W2, b2)
    g = 2 * scale * (y - ts)
    gr = ora.decoder_bwd(zs, W1, b1, W2, g)
    dz_ref = np.zeros((npix, 16))
    np.add.at(dz_ref, idx, gr["z"])
    want_loss = scale * ((y - ts) ** 2).sum()
    assert abs(loss.item() - want_loss) < 1e-4 * want_loss
    got = dict(W1=dec.grads["W1"], b1=dec.grads["b1"], W2=dec.grads["W2"], b2=dec.grads["b2"], z=dz)
    want = dict(W1=gr["W1"], b1=gr["b1"], W2=gr["W2"], b2=gr["b2"], z=dz_ref)
    for k in want:
        a, b = _np(got[k]).ravel(), want[k].ravel()
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert rel < 1e-4, (k, rel)


U_BF16 = 2.0 ** -8
GAMMA_F32 = 2.0 ** -24  # per term of an fp32 sum (with the term count as factor)


def _gelu(x):
    return 0.5 * x * (1.0 + np.vectorize(math.erf)(x / math.sqrt(2.0)))


def _gelu_d(x):
    phi = np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)
    return 0.5 * (1.0 + np.vectorize(math.erf)(x / math.sqrt(2.0))) + x * phi


def _gelu_dd(x):
    return np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi) * (2.0 - x * x)


def _tc_training_bound(zs, W1, b1, W2, t_minus_b2, scale, idx, npix):
    """First-order bound of the tensor-core training's error: z, H, dY and dPRE
    enter the products rounded to bf16 (relative error <= u each), every sum
    is fp32 (gamma = k 2^-24 of the sum of |terms| over its k terms). The
    magnitudes propagate through the step in its order, with |gelu'| and
    |gelu''| at the exact pre-activation."""
    u, S = U_BF16, zs.shape[0]
    pre = zs @ W1 + b1
    H = _gelu(pre)
    r = H @ W2 - t_minus_b2  # = y - target
    g = 2 * scale * r
    aW1, aW2, az = np.abs(W1), np.abs(W2), np.abs(zs)
    d_pre = u * az @ aW1 + 16 * GAMMA_F32 * (az @ aW1)
    d_H = u * np.abs(H) + np.abs(_gelu_d(pre)) * d_pre
    d_Y = d_H @ aW2 + 128 * GAMMA_F32 * (np.abs(H) @ aW2)
    d_g = 2 * scale * d_Y                  # the fp32 cotangent (loss, db2)
    d_gb = u * np.abs(g) + d_g              # the bf16 dY of the products
    dH = g @ W2.T
    d_dH = d_gb @ aW2.T + 512 * GAMMA_F32 * (np.abs(g) @ aW2.T)
    dpre = dH * _gelu_d(pre)
    d_dpre = u * np.abs(dpre) + np.abs(_gelu_d(pre)) * d_dH + np.abs(dH) * np.abs(_gelu_dd(pre)) * d_pre
    gS = S * GAMMA_F32
    b = dict(
        W2=d_H.T @ np.abs(g) + np.abs(H).T @ d_gb + gS * (np.abs(H).T @ np.abs(g)),
        b2=d_g.sum(0) + gS * np.abs(g).sum(0),
        W1=(u * az).T @ np.abs(dpre) + az.T @ d_dpre + gS * (az.T @ np.abs(dpre)),
        b1=d_dpre.sum(0) + gS * np.abs(dpre).sum(0),
    )
    dz_rows = d_dpre @ aW1.T + 128 * GAMMA_F32 * (np.abs(dpre) @ aW1.T)
    b["z"] = np.zeros((npix, zs.shape[1]))
    np.add.at(b["z"], idx, dz_rows)
    b["loss"] = scale * (2 * np.abs(r) * d_Y).sum() + S * 512 * GAMMA_F32 * scale * (r * r).sum()
    return b


@pytest.mark.parametrize("S", [100, 2000])
def test_decoder_training_tc_within_bf16_bound(dec_mod, ora, S):
    """gs_decoder_train_tc against the FP64 oracle's loss and gradients (exact
    fp32 z, the same bf16-exact weights):
    * element by element within twice the first-order worst-case bound of
      _tc_training_bound (the factor covers second-order terms). That bound
      adds |terms|, so for these sums of random-sign terms it is loose (of the
      order of the gradients themselves);
    * normwise within u = 2^-8, one bf16 rounding: every gradient passes
      through at most four rounded operands with independent errors of
      relative size <= u, which mostly cancel (a numpy emulation of the same
      roundings and fp32 sums lands at 0.03-0.6 u on the S = 2000 case).
    S = 100 is one partial tile; 2000 is 16 tiles with a ragged last one,
    spread over several CTAs."""
    dec = dec_mod.Decoder(seed=5)
    _normal_(dec.params["b1"], 0.1, 103)
    _normal_(dec.params["b2"], 0.1, 104)
    rng = np.random.default_rng(6)
    npix, seed = 2500, 77
    z = torch.tensor(rng.normal(size=(npix, 16)).astype(np.float32), device="cuda")
    tgt = torch.tensor(rng.normal(size=(npix, 512)).astype(np.float32), device="cuda")
    dz = torch.zeros(npix, 16, device="cuda")
    loss = torch.zeros(1, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    scale = 1.0 / (S * 512)
    dec.zero_grad()
    dec.train_eval_tc(z, tgt, S, seed, scale, dz_map=dz, loss=loss, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    idx = _samples(seed, S, npix)
    W1, b1, W2, b2 = _np(dec.work["W1"]), _np(dec.params["b1"]), _np(dec.work["W2"]), _np(dec.params["b2"])
    zs, ts = _np(z)[idx], _np(tgt)[idx]
    y = ora.decoder_fwd(zs, W1, b1, W2, b2)
    g = 2 * scale * (y - ts)
    gr = ora.decoder_bwd(zs, W1, b1, W2, g)
    dz_ref = np.zeros((npix, 16))
    np.add.at(dz_ref, idx, gr["z"])
    bound = _tc_training_bound(zs, W1, b1, W2, ts - b2, scale, idx, npix)
    want_loss = scale * ((y - ts) ** 2).sum()
    assert abs(loss.item() - want_loss) <= 2 * bound["loss"] + 1e-6 * want_loss
    got = dict(W1=dec.grads["W1"], b1=dec.grads["b1"], W2=dec.grads["W2"], b2=dec.grads["b2"], z=dz)
    want = dict(W1=gr["W1"], b1=gr["b1"], W2=gr["W2"], b2=gr["b2"], z=dz_ref)
    for k in want:
        a, b = _np(got[k]), want[k]
        err = np.abs(a - b)
        assert np.all(err <= 2 * bound[k] + 1e-12), (k, float((err / (bound[k] + 1e-30)).max()))
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert rel <= U_BF16, (k, rel)


def test_checkpoint_resume_reproduces_the_next_step(dec_mod, tmp_path):
    """Three tensor-core training steps with Adam, a checkpoint, then the next
    step twice: from the live decoder and from a decoder of another seed
    loaded from the file. Given the same gradients (the gradient sums use
    float atomics, whose order may differ between runs), the resumed Adam
    step gives bit-identical weights, moments and bf16 copies."""
    rng = np.random.default_rng(12)
    npix, S = 3000, 1000
    z = torch.tensor(rng.normal(size=(npix, 16)).astype(np.float32), device="cuda")
    tgt = torch.tensor(rng.normal(size=(npix, 512)).astype(np.float32), device="cuda")
    a = dec_mod.Decoder(seed=9)
    for step in range(3):
        a.zero_grad()
        a.train_eval_tc(z, tgt, S, 100 + step, 1.0 / (S * 512))
        a.adam(1e-3)
    path = tmp_path / "dec.bin"
    a.save(path)
    b = dec_mod.Decoder(seed=10)
    b.load(path)
    a.zero_grad()
    a.train_eval_tc(z, tgt, S, 103, 1.0 / (S * 512))
    for k in a.grads:
        b.grads[k].copy_(a.grads[k])
    a.adam(1e-3)
    b.adam(1e-3)
    torch.cuda.synchronize()
    assert a.step == b.step == 4
    for k in a.params:
        for x, y in ((a.params[k], b.params[k]), (a.m[k], b.m[k]), (a.v[k], b.v[k])):
            assert torch.equal(x.view(torch.int32), y.view(torch.int32)), k
    for k in a.work:
        assert torch.equal(a.work[k], b.work[k]), k


def test_adam_step_formula(dec_mod):
    rng = np.random.default_rng(8)
    p0 = rng.normal(size=1000).astype(np.float32)
    g = rng.normal(size=1000).astype(np.float32)
    p = torch.tensor(p0, device="cuda")
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    for step in (1, 2):
        dec_mod.adam_tensor(p, torch.tensor(g, device="cuda"), m, v, step, 1e-2)
    torch.cuda.synchronize()
    mm, vv, pp = np.zeros(1000), np.zeros(1000), p0.astype(np.float64)
    for step in (1, 2):
        mm = 0.9 * mm + 0.1 * g
        vv = 0.999 * vv + 0.001 * g.astype(np.float64) ** 2
        pp = pp - 1e-2 * (mm / (1 - 0.9 ** step)) / (np.sqrt(vv / (1 - 0.999 ** step)) + 1e-8)
    assert np.abs(_np(p) - pp).max() < 1e-5


def test_trained_decoder_beats_linear_and_untrained(dec_mod):
    """Config-5 pattern at small scale: 16-d latents rendered and decoded to
    512 channels, trained on the GPU by the project's kernels against the
    plain 512-d render of prototype-structured features; on held-out poses
    the trained decoder beats (a) the rank-16 PCA linear decode of rendered
    PCA latents and (b) the untrained decoder."""
    import paper_2504_19409_gb300 as g
    from paper_2504_19409_gb300 import scenegen as sg
    P, W, H, f = 30_000, 160, 96, 80.0
    sc = sg.room_scene(41, P, 512, feat_kind="prototypes")
    t = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    scene = tuple(t(x) for x in (sc.means, sc.scales, sc.quats, sc.opacity, sc.colors))
    feats = t(sc.feats)
    mu, U = sg.pca_basis(sc.feats, 16)
    lat0 = ((sc.feats - mu) @ U).astype(np.float32)
    cams = [sg.room_trajectory(k, 100, W, H, f).as_f32() for k in range(0, 100, 5)]
    train, held = cams[::2] + cams[1::4], cams[3::4]
    plain = g.Rasterizer(P, W, H, N=512, layout=g.GS_LAYOUT_HWC)
    for c in cams:
        plain.ensure_capacity(c, *scene[:4])
    targets = [dec_mod.render_features(plain, c, scene, feats).clone() for c in cams]
    alphas = []
    for c in cams:
        plain.forward(c, *scene, feats)
        alphas.append(plain.fwd["alpha"].reshape(-1).clone())
    tgt = {id(c): tt for c, tt in zip(cams, targets)}
    alp = {id(c): a for c, a in zip(cams, alphas)}

    dec = dec_mod.Decoder(seed=11)
    tr = dec_mod.LatentFieldTrainer(scene, lat0, cams[0], dec)
    tr.ensure_capacity(cams)

    def evaluate(fn):
        rels, coss = [], []
        for c in held:
            pred = fn(c)
            rel, cos = dec_mod.feature_error(pred, tgt[id(c)], alp[id(c)] > 0.5)
            rels.append(rel)
            coss.append(cos)
        return float(np.mean(rels)), float(np.mean(coss))

    mu_t, U_t = t(mu.astype(np.float32)), t(U.astype(np.float32))
    pca = evaluate(lambda c: alp[id(c)][:, None] * mu_t[None, :] + tr.render_latents(c) @ U_t.T)
    untrained = evaluate(tr.decode)
    for step in range(1500):
        c = train[step % len(train)]
        tr.step(c, tgt[id(c)], 16384, 1000 + step, lr_dec=3e-3, lr_lat=5e-3)
    torch.cuda.synchronize()
    trained = evaluate(tr.decode)
    print(f"held-out rel-L2 / cosine: PCA-16 {pca}, untrained {untrained}, trained {trained}")
    assert trained[0] < 0.5 * pca[0], (trained, pca)
    assert trained[1] > 0.95 and trained[0] < untrained[0] and trained[1] > pca[1]


@pytest.mark.parametrize("n", [1000 + 37, 3 * 152 * 128 + 37])
def test_decoder_tensor_core_forward_within_bound(dec_mod, ora, n):
    """gs_decoder_fwd_tc rounds z and the GELU output h to bf16 (weights are
    bf16 already); against the oracle on the bf16-rounded z the remaining
    difference is the rounding of h, |fl(h) - h| <= u |h| with u = 2^-8 the
    unit roundoff of bf16 (8 significant bits), the bf16 x bf16 products being
    exact in fp32: |y_tc - y| <= u |h| |W2| + 1e-6 per output, the 1e-6
    covering the fp32 arithmetic of h and of the accumulation. Both sizes end
    in a ragged tile; the larger gives every CTA about three tiles, so each
    tile's drain overlaps the next tile's products."""
    from math import sqrt
    from scipy.special import erf
    dec = dec_mod.Decoder(seed=13)
    _normal_(dec.params["b1"], 0.2, 104)
    _normal_(dec.params["b2"], 0.2, 105)
    rng = np.random.default_rng(14)
    z = torch.tensor(rng.normal(size=(n, 16)).astype(np.float32), device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    buf = torch.full((n + 40, 512), 7.0, device="cuda")  # rows past n must stay untouched
    y = dec.forward_tc(z, out=buf[:n], status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert (buf[n:] == 7.0).all()
    zb = z.to(torch.bfloat16).double().cpu().numpy()
    W1, b1, W2, b2 = _np(dec.work["W1"]), _np(dec.params["b1"]), _np(dec.work["W2"]), _np(dec.params["b2"])
    ref = ora.decoder_fwd(zb, W1, b1, W2, b2)
    pre = zb @ W1 + b1
    h = 0.5 * pre * (1 + erf(pre / sqrt(2)))
    bound = 2.0 ** -8 * (np.abs(h) @ np.abs(W2)) + 1e-6
    err = np.abs(_np(y) - ref)
    assert (err <= bound).all(), float((err / bound).max())
    assert (err / bound).max() > 0.01


def test_decoder_labels_from_latents_within_bound(dec_mod, ora):
    """gs_decoder_labels_tc against the oracle's decoded field dotted with the
    queries: z rounded to bf16 (as in the tensor-core decoder), and both
    factors of each product, the hidden layer h and the folded G = W2 q^T,
    rounded to bf16, |fl(h) fl(G) - h G| <= (2u + u^2) |h| |G| with u = 2^-8
    the unit roundoff of bf16, so each logit lies within
    (2u + u^2) sum_k |h_k| |G_kl| + 1e-5 (sum_k |h_k| |G_kl| + |c_l|) + 1e-6 of
    the exact one (the 1e-5 term: the fp32 fold and accumulation). Labels must
    agree wherever the oracle's two largest logits are more than twice that
    apart (80 % of this seeded case's pixels); probabilities within twice the
    pixel's largest bound."""
    from math import erf, sqrt
    dec = dec_mod.Decoder(seed=17)
    _normal_(dec.params["b1"], 0.2, 106)
    _normal_(dec.params["b2"], 0.2, 107)
    rng = np.random.default_rng(18)
    n, L = 1000 + 37, 24
    z = torch.tensor(rng.normal(size=(n, 16)).astype(np.float32), device="cuda")
    q = torch.tensor((rng.normal(size=(L, 512)) / np.sqrt(512) * 4).astype(np.float32), device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    probs, labels = dec.labels_tc(z, q, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    zb = z.to(torch.bfloat16).double().cpu().numpy()
    W1, b1, W2, b2 = _np(dec.work["W1"]), _np(dec.params["b1"]), _np(dec.work["W2"]), _np(dec.params["b2"])
    qn = _np(q)
    y = ora.decoder_fwd(zb, W1, b1, W2, b2)
    logits = y @ qn.T
    h = zb @ W1 + b1
    h = 0.5 * h * (1 + np.vectorize(erf)(h / sqrt(2)))
    G, c = W2 @ qn.T, b2 @ qn.T
    hg = np.abs(h) @ np.abs(G)
    u = 2.0 ** -8
    bound = (2 * u + u * u) * hg + 1e-5 * (hg + np.abs(c)) + 1e-6
    srt = np.sort(logits, axis=1)
    sure = (srt[:, -1] - srt[:, -2]) > 2 * bound.max(axis=1)
    assert sure.mean() > 0.75
    assert np.array_equal(labels.cpu().numpy()[sure], np.argmax(logits, axis=1)[sure])
    e = np.exp(logits - logits.max(1, keepdims=True))
    p_ref = e / e.sum(1, keepdims=True)
    err = np.abs(probs.cpu().numpy() - p_ref)
    assert (err <= 2 * bound.max(axis=1, keepdims=True) + 1e-6).all(), float(err.max())
    _, lab_only = dec.labels_tc(z, q, probs=False)
    assert torch.equal(lab_only, labels)
