import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
TESTS = os.path.dirname(os.path.abspath(__file__))
if TESTS not in sys.path:
    sys.path.insert(0, TESTS)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


def pytest_runtest_setup(item):
    import margins
    margins.set_test(item.nodeid)


def pytest_sessionfinish(session, exitstatus):
    import margins
    margins.dump()


@pytest.fixture(scope="session")
def lib():
    """The CUDA library's ctypes handle (built in-tree on first use)."""
    from paper_2505_21319_gb300 import _binding
    return _binding.load()
