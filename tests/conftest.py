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


@pytest.fixture(scope="session")
def oracle_pool():
    """run(jobs) -> oracle results: jobs are (A, b, c, Params) tuples, solved by
    oracle.abip_oracle.solve in a pool of spawned processes (spawned, not forked: the
    parent holds a CUDA context)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor

    from oracle import abip_oracle as O

    ex = ProcessPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1)), mp_context=mp.get_context("spawn"))

    def run(jobs):
        futs = [ex.submit(O.solve, A, b, c, prm) for (A, b, c, prm) in jobs]
        return [f.result() for f in futs]

    yield run
    ex.shutdown()
