import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


# The property-based pins are CPU tests built on hypothesis. An image without it
# (the Arm GPU image has none) leaves the module out at collection, instead of
# reporting a module-level skip inside GPU-only runs.
collect_ignore = [] if importlib.util.find_spec("hypothesis") else ["test_oracle_properties.py"]


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


@pytest.fixture(scope="session")
def lib():
    """The built CUDA library (skips on machines without a GPU)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_19742_gb300 import nhcbct
    return nhcbct
