"""The stored expected values of tests/golden/ (written by tests/golden/make_golden.py
from the oracle alone) against the oracle as it stands, on the CPU.

tiny_lp_optima.txt holds the basis-enumeration optimum of twelve tiny LPs (the
fundamental theorem of LP on the pair (P)/(D) of Sec. 2): the enumeration must reproduce
it (ABIP's oracle against the same enumeration, live, is a pin in test_oracle_pins.py;
the GPU against the stored values is test_gpu_golden.py).  planted_8x20_iterates.txt holds the
oracle's first five iterates of Algorithm 2 (Sec. 4.2 relaxation, alpha = 1.8); a change
of the oracle's arithmetic shows here first.
"""
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

from oracle import abip_oracle as O  # noqa: E402
from oracle.lp_bruteforce import enumerate_lp  # noqa: E402
import make_golden as G  # noqa: E402

def _tiny_rows():
    rows = []
    with open(os.path.join(HERE, "golden", "tiny_lp_optima.txt")) as f:
        for line in f:
            if line.startswith("#"):
                continue
            seed, m, n, status, p = line.split()
            rows.append((int(seed), int(m), int(n), status, float(p)))
    return rows


def _iterates():
    return np.loadtxt(os.path.join(HERE, "golden", "planted_8x20_iterates.txt"))


@pytest.mark.parametrize("row", _tiny_rows(), ids=lambda r: f"seed{r[0]}")
def test_tiny_optima_reproduce(row):
    seed, m, n, status, p = row
    lp = G.tiny_lp(seed)
    assert (lp.m, lp.n) == (m, n)
    ref = enumerate_lp(lp.A, lp.b, lp.c)
    assert ref["status"] == status
    if status == "optimal":
        assert abs(ref["p_star"] - p) <= 1e-12 * max(1.0, abs(p))
        # the stored optimum is attained: a primal-feasible vertex with that value
        x = ref["optimal_vertices"][-1]
        assert np.all(x >= -1e-12) and np.allclose(lp.A @ x, lp.b, atol=1e-9)
        assert abs(float(lp.c @ x) - p) <= 1e-12 * max(1.0, abs(p))


def test_oracle_iterates_reproduce():
    lp = G.iter_lp()
    want = _iterates()
    ref = O.solve(lp.A, lp.b, lp.c, O.Params(max_admm_iters=G.ITERATES), trace_iters=G.ITERATES)
    assert want.shape == (G.ITERATES, 2 * lp.n + lp.m + 3)
    for k in range(G.ITERATES):
        got = np.asarray(ref.trace[k])
        assert np.linalg.norm(got - want[k]) <= 1e-12 * np.linalg.norm(want[k]), k
