"""gs_zero, the clearing kernel of the launch chain (it clears the gradient
arena before every adjoint): the requested words become zero and nothing
around them changes, for spans past the kernel's grid stride (1216 blocks of
256 threads, one 16-byte store per thread per round), odd word counts and
slices that start off a 16-byte boundary (single-word head and tail)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

GRID_WORDS = 1216 * 256 * 4
PATTERN = 0x5A5A5A5A


@pytest.mark.parametrize("offset,count", [(0, 3 * GRID_WORDS + 37), (1, 5), (3, GRID_WORDS + 1), (7, 1),
                                          (2, 2 * GRID_WORDS)])
def test_zero_clears_exactly_the_span(gs, offset, count):
    guard = 1024
    buf = torch.full((offset + count + guard,), PATTERN, dtype=torch.int32, device="cuda")
    gs.zero_(buf[offset:offset + count])
    torch.cuda.synchronize()
    h = buf.cpu().numpy()
    assert np.all(h[:offset] == PATTERN)
    assert np.all(h[offset:offset + count] == 0)
    assert np.all(h[offset + count:] == PATTERN)


def test_zero_rejects_strided_views(gs):
    buf = torch.ones(64, 4, device="cuda")
    with pytest.raises(gs.GsffError):
        gs.zero_(buf[:, 1])
    torch.cuda.synchronize()
    assert torch.all(buf == 1)
