import os
import sys

import pytest

# one hardware work queue per scheduler stream, before any CUDA context exists
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# The oracle's mutation tests run its pins against a mutated copy of the
# oracle package: ORACLE_UNDER_TEST names the directory holding that copy,
# which is loaded as `oracle` in place of the repository's own.
if os.environ.get("ORACLE_UNDER_TEST"):
    import importlib.util

    _pkg = os.path.join(os.environ["ORACLE_UNDER_TEST"], "oracle")
    _spec = importlib.util.spec_from_file_location("oracle", os.path.join(_pkg, "__init__.py"),
                                                   submodule_search_locations=[_pkg])
    _mod = importlib.util.module_from_spec(_spec)
    sys.modules["oracle"] = _mod
    _spec.loader.exec_module(_mod)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a)")
    config.addinivalue_line("markers", "slow: full-size parity case")


def pytest_collection_modifyitems(config, items):
    have_gpu = False
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:
        pass
    if have_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)
