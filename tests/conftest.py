"""Shared pytest configuration: the ``gpu`` marker and repository import path."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU oracle check")


@pytest.fixture(scope="session")
def root():
    return ROOT


def pytest_sessionfinish(session, exitstatus):
    """Under the index-checking build (GBPME_BOUNDS=1) write which build ran and the kernels'
    index-check flags to the file named by GBPME_BOUNDS_REPORT."""
    path = os.environ.get("GBPME_BOUNDS_REPORT")
    if not path or os.environ.get("GBPME_BOUNDS") != "1":
        return
    import json
    try:
        import paper_2606_01598_gb300 as g
        lib = g.load_library()
        rep = {"checking": int(lib.pme_bounds_checking()), "flags": int(lib.pme_bounds_flags()),
               "exitstatus": int(exitstatus)}
    except Exception as e:  # reported, the outer test fails on it
        rep = {"error": str(e)}
    with open(path, "w") as f:
        json.dump(rep, f)
