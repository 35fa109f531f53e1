"""The CUDA library (dense per-CTA path, FP64) against the stored expected values of
tests/golden/: the basis-enumeration optima of twelve tiny LPs (Sec. 2; certificates of
Thm 2.2 / Sec. 4.1 for the infeasible ones) and the oracle's first five iterates of
Algorithm 2 on an 8 x 20 planted LP.

Bars: iterates within 1e-10 relative; the status of the enumeration (an LP that is both
primal and dual infeasible may certify either way); objective within 1e-5 relative.
"""
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden as G  # noqa: E402

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abip():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1805_12344_gb300 import build, abip as _abip
    build.build()
    _abip.lib()
    return _abip


def test_gpu_iterates_match_golden(abip):
    lp = G.iter_lp()
    want = np.loadtxt(os.path.join(HERE, "golden", "planted_8x20_iterates.txt"))
    for k in range(1, G.ITERATES + 1):
        s = abip.Solver(lp.A, lp.b, lp.c, max_admm_iters=k)
        info, *_ = s.solve()
        got = s.stacked_state()
        s.close()
        assert info["admm_iters"] == k
        assert np.linalg.norm(got - want[k - 1]) <= 1e-10 * np.linalg.norm(want[k - 1]), k


def test_gpu_tiny_lps_match_golden(abip):
    codes = {"optimal": (abip.ABIP_OPTIMAL,),
             "primal_infeasible": (abip.ABIP_PRIMAL_INFEASIBLE, abip.ABIP_DUAL_INFEASIBLE),
             "dual_infeasible": (abip.ABIP_DUAL_INFEASIBLE,)}
    with open(os.path.join(HERE, "golden", "tiny_lp_optima.txt")) as f:
        rows = [ln.split() for ln in f if not ln.startswith("#")]
    for seed, m, n, status, p in rows:
        lp = G.tiny_lp(int(seed))
        s = abip.Solver(lp.A, lp.b, lp.c)
        info, *_ = s.solve()
        s.close()
        assert info["status"] in codes[status], (seed, info["status"])
        if status == "optimal":
            assert abs(info["obj"] - float(p)) <= 1e-5 * max(1.0, abs(float(p))), seed
