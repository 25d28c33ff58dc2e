import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: long CPU run; enabled with BDDC_SLOW=1")


def pytest_collection_modifyitems(config, items):
    if os.environ.get("BDDC_SLOW") == "1":
        return
    skip = pytest.mark.skip(reason="slow oracle run; set BDDC_SLOW=1")
    for item in items:
        if "slow" in item.keywords:
            item.add_marker(skip)


def pytest_sessionstart(session):
    """Build the in-tree library if it is missing or stale (nvcc is on both
    the build host and the GPU machine)."""
    try:
        from paper_1901_02090_gb300.build import build
        build()
    except Exception as exc:  # the import of the binding will report it
        sys.stderr.write(f"[conftest] building libbddc.so failed: {exc}\n")
