"""GPU parity of the adaptive decrease ratio (gamma_max > 0: the ratio of mu <- gamma mu
taken from the residual of the iterate, Sec. 5) on every path, against the FP64 oracle
with the same rule.

Bars: the FP64 paths keep the 1e-10 (dense) and 1e-9 (hundreds of updates, several
decreases) relative iterate bars of the fixed-ratio tests; every path ends with the
oracle's status and an objective within 1e-5 relative of the oracle's.
"""
import numpy as np
import pytest

from oracle import abip_oracle as O
from paper_1805_12344_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OBJ_TOL = 1e-5
GMAX = 0.4


@pytest.fixture(scope="module")
def abip():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1805_12344_gb300 import build, abip as _abip
    build.build()
    _abip.lib()
    return _abip


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _end(info, ref):
    assert info["status"] == ref.status
    if ref.status == O.OPTIMAL:
        assert max(info["pres"], info["dres"], info["dgap"]) <= 1e-6
        assert abs(info["obj"] - ref.obj) <= OBJ_TOL * max(1.0, abs(ref.obj))


def test_dense_iterates_across_adaptive_decreases(abip):
    """400 updates of the dense FP64 path span several decreases with ratios between
    gamma and gamma_max; the iterate matches the oracle's, and so do the decrease count
    and mu."""
    lp = W.planted_dense(8, 20, seed=5)
    K = 400
    ref = O.solve(lp.A, lp.b, lp.c, O.Params(gamma_max=GMAX, max_admm_iters=K), trace_iters=K)
    gam = ref.raw["gammas"]
    assert len(gam) >= 3 and max(gam) > 0.1              # the rule moved the ratio
    s = abip.Solver(lp.A, lp.b, lp.c, gamma_max=GMAX, max_admm_iters=K)
    info, *_ = s.solve()
    assert info["admm_iters"] == len(ref.trace)
    assert info["outer_iters"] == ref.outer_iters
    assert abs(info["mu"] - ref.mu) <= 1e-12 * ref.mu
    assert _rel(s.stacked_state(), ref.trace[-1]) <= 1e-9


def test_dense_end_to_end_and_batch(abip):
    """End to end on the dense path, single and batched (FP64 and mixed), with the
    warm start of either rule."""
    lps = [W.planted_dense(m, n, seed=W.seed_for(W.BATCH_UNEVEN, 40 + k))
           for k, (m, n) in enumerate([(12, 30), (30, 80), (50, 120)])]
    lps.append(W.infeasible_twin(12, 25, seed=W.seed_for(W.BATCH_UNEVEN, 98)))
    refs = [O.solve(l.A, l.b, l.c, O.Params(gamma_max=GMAX)) for l in lps]
    s = abip.Solver(lps[2].A, lps[2].b, lps[2].c, gamma_max=GMAX)
    info, *_ = s.solve()
    _end(info, refs[2])
    assert abs(info["admm_iters"] - refs[2].admm_iters) <= max(2, refs[2].admm_iters // 100)
    for prec in (abip.ABIP_PREC_F64, abip.ABIP_PREC_MIXED):
        prm = abip.default_params(gamma_max=GMAX, precision=prec)
        infos, *_ = abip.abip_solve_batch([l.A for l in lps], [l.b for l in lps], [l.c for l in lps], prm)
        for f, r in zip(infos, refs):
            _end(f, r)
    w = O.solve(lps[0].A, lps[0].b, lps[0].c, O.Params(gamma_max=GMAX, warmstart=1))
    s1 = abip.Solver(lps[0].A, lps[0].b, lps[0].c, gamma_max=GMAX, warmstart=1)
    f1, *_ = s1.solve()
    _end(f1, w)


def test_sparse_fp64_iterates_across_adaptive_decreases(abip):
    """The persistent grid kernel (FP64, Jacobi-PCG) over 300 updates of a sparse LP."""
    lp = W.planted_sparse(80, seed=W.seed_for(W.SPARSE_PLANTED, 10))
    K = 300
    prm = O.Params(linsys=1, cg_tol=1e-13, gamma_max=GMAX, max_admm_iters=K)
    ref = O.solve(lp.A.to_scipy(), lp.b, lp.c, prm, trace_iters=K)
    assert len(ref.raw["gammas"]) >= 2
    s = abip.Solver(lp.A, lp.b, lp.c, cg_tol=1e-13, gamma_max=GMAX, max_admm_iters=K)
    info, *_ = s.solve()
    assert info["outer_iters"] == ref.outer_iters
    assert _rel(s.stacked_state(), ref.trace[-1]) <= 1e-9


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_sparse_end_to_end(abip, oracle_memo, precision):
    lp = W.planted_sparse(80, seed=W.seed_for(W.SPARSE_PLANTED, 10))
    ref = oracle_memo(("sparse-gamma", 80, 10),
                      lambda: O.solve(lp.A.to_scipy(), lp.b, lp.c, O.Params(linsys=1, cg_tol=1e-10, gamma_max=GMAX)))
    prec = abip.ABIP_PREC_MIXED if precision == "mixed" else abip.ABIP_PREC_F64
    s = abip.Solver(lp.A, lp.b, lp.c, cg_tol=1e-10, gamma_max=GMAX, precision=prec)
    info, *_ = s.solve()
    _end(info, ref)
    assert abs(info["obj"] - lp.p_star) <= OBJ_TOL * max(1.0, abs(lp.p_star))


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_shared_end_to_end(abip, precision):
    sb = W.basis_pursuit(32, 128, batch=4, seed=5)
    prec = abip.ABIP_PREC_MIXED if precision == "mixed" else abip.ABIP_PREC_F64
    prm = abip.default_params(precision=prec, gamma_max=GMAX)
    infos, xs, ys, ss = abip.abip_solve_batch_shared(sb.A, sb.bs, sb.cs, prm)
    for k in range(4):
        ref = O.solve(sb.A, sb.bs[k], sb.cs[k], O.Params(gamma_max=GMAX))
        _end(infos[k], ref)
        if precision == "f64":
            assert infos[k]["outer_iters"] == ref.outer_iters
