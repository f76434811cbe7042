import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running case")


@pytest.fixture(scope="session")
def A():
    """The built library's Python binding on a GB300 (GPU tests only): builds
    libaccord.so if needed and checks the device.  Skips without a GPU."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_11554_gb300 import build
    build.build()
    import paper_2412_11554_gb300 as pkg
    assert pkg.accord_device_check() == 0, "libaccord needs an sm_103 (GB300) device"
    return pkg
