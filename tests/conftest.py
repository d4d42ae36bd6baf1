import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def ed():
    """The CUDA library binding, built in-tree if needed (GPU tests only)."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test selected but no CUDA device is visible")
    from paper_2105_06806_gb300 import _build
    _build.build()
    import paper_2105_06806_gb300 as E
    E.lib()
    return E


@pytest.fixture(autouse=True, scope="module")
def _release_device_memory():
    """After each GPU test module, the library pool's cached blocks and
    PyTorch's go back to the device, so that one module's peak does not
    crowd the next module's allocations (a no-op where the library was not
    loaded)."""
    yield
    E = sys.modules.get("paper_2105_06806_gb300")
    if E is None or getattr(E, "_lib", None) is None:
        return
    import torch
    if torch.cuda.is_available():
        torch.cuda.synchronize()
        E.trim_memory()
        torch.cuda.empty_cache()
