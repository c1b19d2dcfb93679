import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA GPU in this environment")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


@pytest.fixture(autouse=True)
def output_guard_bands(request, monkeypatch):
    """GPU tests: every output from binding.alloc_outputs sits between guard bands, checked
    after the test (tests/guard_util.py)."""
    if "gpu" not in request.keywords:
        yield
        return
    from guard_util import GuardRegistry, guarded_alloc_outputs
    from paper_1507_07733_gb300 import binding
    reg = GuardRegistry()
    monkeypatch.setattr(binding, "alloc_outputs", guarded_alloc_outputs(reg, binding.outputs_struct))
    yield reg
    reg.check()
