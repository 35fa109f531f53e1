"""The batch autotuner of abip_solve_batch (abip_params.autotune) and the hand-out order
(abip_params.batch_order): the occupancy variants of the solve kernel and the order in
which CTAs take instances change the time, never the arithmetic, so every per-instance
result must be bitwise the same; the choice is timed once and then served from the cache
(in the process, and in the JSON file named by ABIP_TUNE_CACHE)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1805_12344_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def abip():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1805_12344_gb300 import build, abip as _abip
    build.build()
    _abip.lib()
    return _abip


def _batch():
    return W.batch_uneven(count=40, infeasible_frac=0.1, m_lo=16, m_hi=64, seed=W.seed_for(W.BATCH_UNEVEN, 40))


@pytest.mark.parametrize("precision", [0, 1])
def test_autotune_and_order_leave_results_unchanged(abip, precision):
    lps = _batch()
    args = ([l.A for l in lps], [l.b for l in lps], [l.c for l in lps])
    base = abip.abip_solve_batch(*args, abip.default_params(precision=precision, batch_order=0, max_admm_iters=20000))
    tuned = abip.abip_solve_batch(*args, abip.default_params(precision=precision, autotune=1, max_admm_iters=20000))
    again = abip.abip_solve_batch(*args, abip.default_params(precision=precision, autotune=1, max_admm_iters=20000))
    assert all(f["tuned"] == 1 for f in tuned[0]) and all(f["tuned"] == 2 for f in again[0])
    assert all(f["ctas_per_sm"] >= 1 for f in tuned[0])
    for run in (tuned, again):
        for k in range(len(lps)):
            a, b = base[0][k], run[0][k]
            assert (a["status"], a["admm_iters"], a["obj"]) == (b["status"], b["admm_iters"], b["obj"])
            assert np.array_equal(base[1][k], run[1][k]) and np.array_equal(base[2][k], run[2][k])


def test_autotune_cache_file(tmp_path):
    """A fresh process with ABIP_TUNE_CACHE writes its choice to the file; a second
    process reads it and does not time the variants again."""
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    cache = tmp_path / "tune.json"
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_1805_12344_gb300 import abip, workloads as W\n"
            "lps = W.batch_uneven(count=12, infeasible_frac=0.0, m_lo=16, m_hi=32, seed=5)\n"
            "infos, *_ = abip.abip_solve_batch([l.A for l in lps], [l.b for l in lps], [l.c for l in lps],\n"
            "                                   abip.default_params(autotune=1, max_admm_iters=2000), want_solution=False)\n"
            "print('TUNED', infos[0]['tuned'])\n") % ROOT
    env = dict(os.environ, ABIP_TUNE_CACHE=str(cache))
    first = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert first.returncode == 0, first.stderr
    assert "TUNED 1" in first.stdout
    entries = json.loads(cache.read_text())
    assert len(entries) == 1 and list(entries.values())[0] in (0, 1, 2)
    second = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert second.returncode == 0, second.stderr
    assert "TUNED 2" in second.stdout
