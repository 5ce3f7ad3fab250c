import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU test")


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_golden(name):
    import numpy as np
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#")


def gpu_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def to_dev(a):
    """numpy n x c (or n) -> torch (c, n) float64 CUDA block."""
    import numpy as np
    import torch
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        a = a[:, None]
    return torch.tensor(np.ascontiguousarray(a.T), dtype=torch.float64, device="cuda").contiguous()


def from_dev(t):
    """torch (c, n) block -> numpy n x c."""
    return t.detach().cpu().numpy().T.copy()


@pytest.fixture(scope="session")
def built_lib():
    from paper_2506_08355_gb300 import build, lrep
    build.build()
    return lrep.lib()
