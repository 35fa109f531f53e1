"""Presolve (host, abip_presolve) -> GPU solve of the standard form -> postsolve
(abip_postsolve), on general-form LPs with bounds and on the SICE LPs of Sec. 5.2, against
the planted optimum, scipy's HiGHS optimum of the original LP and the FP64 oracle.

Bars: the postsolved objective within 1e-5 relative of HiGHS's (the solves stop at
eps = 1e-7 on the scaled standard form); the postsolved point feasible to 1e-5 relative.
"""
import numpy as np
import pytest

from oracle import abip_oracle as O
from paper_1805_12344_gb300 import workloads as W

torch = pytest.importorskip("torch")
linprog = pytest.importorskip("scipy.optimize").linprog
pytestmark = pytest.mark.gpu

OBJ_TOL = 1e-5


@pytest.fixture(scope="module")
def abip():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1805_12344_gb300 import build, abip as _abip
    build.build()
    _abip.lib()
    return _abip


def _highs(g):
    bounds = [(None if not np.isfinite(lo) else lo, None if not np.isfinite(hi) else hi) for lo, hi in zip(g.l, g.w)]
    r = linprog(g.c, A_eq=g.A, b_eq=g.b, bounds=bounds, method="highs")
    assert r.status == 0
    return r.fun


def _feasible(g, x, tol):
    scale = 1.0 + np.abs(g.b).max()
    assert np.abs(g.A @ x - g.b).max() <= tol * scale
    assert np.all(x >= g.l - tol * scale) and np.all(x <= g.w + tol * scale)


@pytest.mark.parametrize("seed", [1, 2])
@pytest.mark.parametrize("path", ["dense_f64", "sparse_f64", "sparse_mixed"])
def test_general_lp_through_presolve(abip, seed, path):
    g = W.general_lp(seed=seed)
    P = abip.Presolved(g.A, g.b, g.c, g.l, g.w)
    assert P.status == 0
    M, b, c = P.lp()
    if path == "dense_f64":
        s = abip.Solver(M.to_dense(), b, c, eps=1e-7)
    elif path == "sparse_f64":
        s = abip.Solver(M, b, c, eps=1e-7, cg_tol=1e-12)
    else:
        s = abip.Solver(M, b, c, eps=1e-7, cg_tol=1e-12, precision=abip.ABIP_PREC_MIXED)
    info, x, y, _ = s.solve()
    assert info["status"] == O.OPTIMAL
    xo, yo, zo, obj = P.postsolve(x, y)
    assert abs(obj - (info["obj"] + P.info["obj_offset"])) <= 1e-9 * (1 + abs(obj))
    ref = _highs(g)
    assert abs(obj - ref) <= OBJ_TOL * (1 + abs(ref))
    assert abs(obj - g.p_star) <= OBJ_TOL * (1 + abs(g.p_star))
    _feasible(g, xo, 1e-5)


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_sice_columns_as_one_shared_batch(abip, precision):
    """The d columns of SICE presolve to one scaled matrix and d right-hand sides: one
    abip_solve_batch_shared call solves them all; each postsolved optimum matches HiGHS
    and, for one column, the oracle's ABIP on the same standard form."""
    d = 16
    S, lam = W.sice(d)
    gs = [W.sice_general_lp(S, lam, j) for j in range(d)]
    Ps = [abip.Presolved(g.A, g.b, g.c, g.l, g.w) for g in gs]
    lps = [P.lp() for P in Ps]
    A0 = lps[0][0]
    for M, _, _ in lps[1:]:
        assert np.array_equal(M.val, A0.val) and np.array_equal(M.col_idx, A0.col_idx)
    prec = abip.ABIP_PREC_MIXED if precision == "mixed" else abip.ABIP_PREC_F64
    prm = abip.default_params(eps=1e-7, precision=prec)
    infos, xs, ys, ss = abip.abip_solve_batch_shared(A0.to_dense(), [b for _, b, _ in lps], [c for _, _, c in lps], prm)
    for j in range(d):
        assert infos[j]["status"] == O.OPTIMAL, (j, infos[j]["status"])
        xo, yo, zo, obj = Ps[j].postsolve(xs[j], ys[j])
        ref = _highs(gs[j])
        assert abs(obj - ref) <= OBJ_TOL * (1 + abs(ref)), (j, obj, ref)
        _feasible(gs[j], xo, 1e-5)
    r = O.solve(A0.to_dense(), lps[3][1], lps[3][2], O.Params(eps=1e-7))
    assert abs(infos[3]["obj"] - r.obj) <= OBJ_TOL * (1 + abs(r.obj))
