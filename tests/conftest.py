import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU check")


@pytest.fixture(scope="session")
def ora():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def sg():
    from paper_2504_19409_gb300 import scenegen
    return scenegen


@pytest.fixture(scope="session")
def gs():
    """The package with its CUDA library built and loaded (skips without a GPU)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_19409_gb300 import build
    build.build()
    import paper_2504_19409_gb300 as g
    g.lib()
    return g
