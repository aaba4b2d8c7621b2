import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU test")


import pytest


@pytest.fixture(scope="session")
def ctx():
    """A libtbmd context on cuda:0 (builds the library first)."""
    import torch
    from paper_1203_6836_gb300 import build, tbmd
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    c = tbmd.Context()
    yield c
    c.close()
