import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_collection_modifyitems(config, items):
    import torch
    if torch.cuda.is_available():
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


_ERRORS = {}


@pytest.fixture
def record_error(request):
    """Record a measured parity error; written to $PARITY_LOG (JSON) at exit."""
    def rec(name, value):
        _ERRORS[f"{request.node.name}:{name}"] = float(value)
    return rec


def pytest_sessionfinish(session, exitstatus):
    import json
    path = os.environ.get("PARITY_LOG")
    if path and _ERRORS:
        with open(path, "w") as f:
            json.dump(_ERRORS, f, indent=1, sort_keys=True)
