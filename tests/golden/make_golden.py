"""Writes the stored expected values of tests/golden/ from the oracle alone.

Run from the repository root:  python tests/golden/make_golden.py
Inputs come from the seeded generators of paper_1805_12344_gb300/workloads.py (no ABIP
arithmetic there); every expected value comes from oracle/ (test infrastructure):

  tiny_lp_optima.txt       status and optimal value of twelve tiny standard-form LPs by
                           enumerating every basis (oracle/lp_bruteforce.py): the
                           fundamental theorem of LP applied to the primal-dual pair
                           (P)/(D) of Sec. 2; ABIP's certificates follow Thm 2.2 / Sec. 4.1
  planted_8x20_iterates.txt the first five ADMM iterates (y, x, tau, theta, s, kappa) of
                           Algorithm 2 with the relaxation of Sec. 4.2 (alpha = 1.8,
                           beta = 1, mu0 = beta) on an 8 x 20 planted LP, by the FP64 oracle
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import abip_oracle as O  # noqa: E402
from oracle.lp_bruteforce import enumerate_lp  # noqa: E402
from paper_1805_12344_gb300 import workloads as W  # noqa: E402

TINY_SEEDS = range(12)
ITER_LP_SEED = W.seed_for(W.TINY, 100)
ITERATES = 5


def tiny_lp(seed):
    """The tiny LP of a seed: shape from default_rng(seed); odd seeds unplanted random
    signs (optimal, infeasible or unbounded), even seeds planted."""
    rng = np.random.default_rng(seed)
    m = int(rng.integers(1, 5))
    n = int(rng.integers(m + 1, m + 7))
    if seed % 2:
        return W.tiny_random(m, n, seed=W.seed_for(W.TINY, seed))
    return W.tiny_planted(m, n, W.seed_for(W.TINY, seed))


def iter_lp():
    return W.planted_dense(8, 20, seed=ITER_LP_SEED)


def main():
    with open(os.path.join(HERE, "tiny_lp_optima.txt"), "w") as f:
        f.write("# seed m n status p_star   (basis enumeration; p_star nan unless optimal)\n")
        for seed in TINY_SEEDS:
            lp = tiny_lp(seed)
            ref = enumerate_lp(lp.A, lp.b, lp.c)
            p = ref.get("p_star", float("nan"))
            f.write(f"{seed} {lp.m} {lp.n} {ref['status']} {p:.17e}\n")
    lp = iter_lp()
    ref = O.solve(lp.A, lp.b, lp.c, O.Params(max_admm_iters=ITERATES), trace_iters=ITERATES)
    with open(os.path.join(HERE, "planted_8x20_iterates.txt"), "w") as f:
        f.write(f"# rows: ADMM update 1..{ITERATES}; columns: y (8), x (20), tau, theta, s (20), kappa\n")
        for k in range(ITERATES):
            f.write(" ".join(f"{v:.17e}" for v in ref.trace[k]) + "\n")


if __name__ == "__main__":
    main()
