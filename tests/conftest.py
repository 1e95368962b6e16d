import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA library)")
    config.addinivalue_line("markers", "slow: large inputs")


def read_golden(name):
    """Parse a tests/golden/*.txt fixture: 'key: value' lines, '#' comments."""
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = line.split(":", 1)
            out[k.strip()] = v.strip()
    return out


@pytest.fixture(scope="session")
def ctx():
    """A gbx context on cuda:0 (GPU tests only)."""
    import torch
    import paper_1908_01407_gb300 as gb
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    c = gb.Context(0)
    yield c
    c.close()
