import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


_ORACLE_MEMO = {}


@pytest.fixture(scope="session")
def oracle_memo():
    """Oracle results shared by the tests of one session: memo(key, fn) runs fn() once per
    key.  The oracle is deterministic, so FP64 and mixed-precision parity tests of the same
    seeded LP can compare against one oracle solve."""
    def memo(key, fn):
        if key not in _ORACLE_MEMO:
            _ORACLE_MEMO[key] = fn()
        return _ORACLE_MEMO[key]
    return memo
