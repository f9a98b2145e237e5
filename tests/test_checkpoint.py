"""Decoder checkpoints (raw binary: the fp32 weights and biases, both Adam
moments and the step counter; the bf16 working copies are rebuilt as the
weights' bf16 rounding), on the host: a state written and read back into a
differently initialised decoder is bit-identical, and a checkpoint of another
shape or a truncated one is refused."""
import numpy as np
import pytest
import torch


def _randomise(dec, seed):
    rng = np.random.default_rng(seed)
    for k in dec.params:
        for t in (dec.params[k], dec.m[k], dec.v[k]):
            t.copy_(torch.from_numpy(rng.normal(size=tuple(t.shape)).astype(np.float32)))
    for k in dec.work:
        dec.work[k].copy_(dec.params[k].to(torch.bfloat16).to(torch.float32))
    dec.step = 37


def test_decoder_state_round_trip(tmp_path):
    from paper_2504_19409_gb300.decoder import Decoder
    a = Decoder(seed=1, device="cpu")
    _randomise(a, 5)
    path = tmp_path / "dec.bin"
    a.save(path)
    assert path.stat().st_size == 24 + 3 * 4 * (16 * 128 + 128 + 128 * 512 + 512)
    b = Decoder(seed=2, device="cpu")
    assert not torch.equal(a.params["W1"], b.params["W1"])
    b.load(path)
    assert b.step == 37
    for k in a.params:
        for x, y in ((a.params[k], b.params[k]), (a.m[k], b.m[k]), (a.v[k], b.v[k])):
            assert torch.equal(x.view(torch.int32), y.view(torch.int32)), k
    for k in a.work:
        assert torch.equal(a.work[k], b.work[k]), k


def test_decoder_state_refuses_other_shapes_and_truncation(tmp_path):
    from paper_2504_19409_gb300.decoder import Decoder
    a = Decoder(seed=1, device="cpu")
    blob = a.state_bytes()
    with pytest.raises(ValueError):
        Decoder(din=8, seed=1, device="cpu").load_state_bytes(blob)
    with pytest.raises(ValueError):
        Decoder(seed=1, device="cpu").load_state_bytes(blob[:-4])
    with pytest.raises(ValueError):
        Decoder(seed=1, device="cpu").load_state_bytes(b"XXXXXXXX" + blob[8:])
