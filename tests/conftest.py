import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def load_matrix(name):
    """A numeric matrix from tests/golden (comment lines start with '#')."""
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#", ndmin=2)


def load_table(name):
    """key value pairs from tests/golden."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split()[:2]
            out[k] = float(v)
    return out


@pytest.fixture
def golden():
    return load_matrix


@pytest.fixture(scope="session")
def rg_ctx():
    """A library context on cuda:0 (GPU tests only)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_04277_gb300 import api
    ctx = api.Context(0)
    yield ctx
    ctx.close()
