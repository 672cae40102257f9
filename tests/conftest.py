import os
import sys

import pytest

# Native plans are range-checked on the host before every launch in tests.
os.environ.setdefault("QED_VALIDATE", "1")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_collection_modifyitems(config, items):
    # Run files in name order so tests/test_zz_*.py come last.
    items.sort(key=lambda it: (os.path.basename(str(it.fspath)), ))
