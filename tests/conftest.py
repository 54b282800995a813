import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    # the library's autotuner keeps its decisions in a file: a private one per
    # test session, so that runs neither read nor leave a cache elsewhere
    import tempfile
    if "STAG_TUNE_CACHE" not in os.environ:
        os.environ["STAG_TUNE_CACHE"] = os.path.join(tempfile.mkdtemp(prefix="stag_tune_"), "tune.json")
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: larger CPU oracle runs")


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def stag():
    """The CUDA library's Python binding; fails loudly when the GPU or library is missing."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("gpu test collected without a CUDA device")
    import paper_2502_03249_gb300 as stag_mod
    stag_mod.load()
    return stag_mod
