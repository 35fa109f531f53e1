"""The presolve of Sec. 4.5: the oracle (oracle/presolve.py) against facts that fix it, and the
library's host presolve (abip_presolve, no GPU needed) against the oracle.

Pins: every reduction fires on a general LP built to contain its structure; the optimum
after presolve -> solve -> postsolve equals the planted optimum and scipy's HiGHS optimum
of the original LP; the postsolved point satisfies the KKT conditions of the bounded LP
(primal feasibility, bounds, reduced-cost signs, strong duality); each infeasibility rule
reports on a constructed LP; Ruiz passes equilibrate.  Parity: the library's standard form
and postsolve equal the oracle's (structure exactly, values to rounding).
"""
import numpy as np
import pytest

from oracle import abip_oracle as O
from oracle import presolve as PS
from paper_1805_12344_gb300 import workloads as W

linprog = pytest.importorskip("scipy.optimize").linprog


@pytest.fixture(scope="module")
def abip():
    from paper_1805_12344_gb300 import build, abip as _abip
    build.build()
    _abip.lib()
    return _abip


def _linprog(g):
    bounds = [(None if not np.isfinite(lo) else lo, None if not np.isfinite(hi) else hi) for lo, hi in zip(g.l, g.w)]
    r = linprog(g.c, A_eq=g.A, b_eq=g.b, bounds=bounds, method="highs")
    assert r.status == 0
    return r.fun


def _kkt(g, x, y, z, tol):
    """KKT conditions of min c^T x, A x = b, l <= x <= w at (x, y, z = c - A^T y)."""
    scale = 1.0 + np.abs(g.b).max()
    assert np.abs(g.A @ x - g.b).max() <= tol * scale
    assert np.all(x >= g.l - tol * scale) and np.all(x <= g.w + tol * scale)
    zs = tol * (1.0 + np.abs(g.c).max() + np.abs(y).max())
    at_l = np.isfinite(g.l) & (x <= g.l + 1e-4)
    at_w = np.isfinite(g.w) & (x >= g.w - 1e-4)
    assert np.all(z[~at_l] <= zs * 100)           # z > 0 only at a lower bound
    assert np.all(z[~at_w] >= -zs * 100)          # z < 0 only at an upper bound
    dual = g.b @ y + np.sum(np.where(z > 0, z * np.where(np.isfinite(g.l), g.l, 0.0), 0.0)) \
        + np.sum(np.where(z < 0, z * np.where(np.isfinite(g.w), g.w, 0.0), 0.0))
    assert abs(dual - g.c @ x) <= 1e-5 * (1.0 + abs(g.c @ x))


def test_each_reduction_fires():
    g = W.general_lp(seed=1)
    P = PS.presolve(g.A, g.b, g.c, g.l, g.w)
    assert P.status == 0
    nfree = int(np.sum(~np.isfinite(g.l) & ~np.isfinite(g.w)))
    assert P.removed == dict(P1=2, P2=2, P4=2, P6=2, P7=1, P5=nfree)
    m_eq = g.A.shape[0] - 2 - 2 - 1              # less the empty, singleton and dependent rows
    n_up = sum(1 for j, kind, _ in P.cols if kind == "lo" and np.isfinite(g.w[j]))
    n_str = sum(2 if kind == "free" else 1 for _, kind, _ in P.cols)
    assert len(P.cols) == g.A.shape[1] - 2 - 2 - 2   # less the fixed, empty and singleton-fixed columns
    assert P.A.shape == (m_eq + n_up, n_str + n_up)


@pytest.mark.parametrize("seed", [1, 2])
def test_presolve_solve_postsolve_reaches_the_optimum(seed):
    """Presolve, the oracle's ABIP on the standard form (eps 1e-8), postsolve: the planted
    optimum, HiGHS's optimum, and the KKT conditions of the original bounded LP."""
    g = W.general_lp(seed=seed)
    P = PS.presolve(g.A, g.b, g.c, g.l, g.w)
    r = O.solve(P.A, P.b, P.c, O.Params(eps=1e-8))
    assert r.status == O.OPTIMAL
    x, y, z, obj = PS.postsolve(P, r.x, r.y, r.s)
    assert abs(obj - (r.obj + P.obj_offset)) <= 1e-9 * (1 + abs(obj))
    assert abs(obj - g.p_star) <= 1e-6 * (1 + abs(g.p_star))
    assert abs(obj - _linprog(g)) <= 1e-6 * (1 + abs(g.p_star))
    _kkt(g, x, y, z, 1e-6)


def test_presolve_without_reductions_against_highs():
    """A general LP with only bound rewriting to do (no structure to remove)."""
    g = W.general_lp(m=12, n=30, seed=5, extras=False)
    P = PS.presolve(g.A, g.b, g.c, g.l, g.w)
    assert P.removed["P1"] == P.removed["P6"] == P.removed["P7"] == 0
    r = O.solve(P.A, P.b, P.c, O.Params(eps=1e-8))
    x, y, z, obj = PS.postsolve(P, r.x, r.y, r.s)
    assert abs(obj - _linprog(g)) <= 1e-6 * (1 + abs(obj))
    _kkt(g, x, y, z, 1e-6)


def _infeasible_cases():
    A = np.array([[1.0, 1.0, 0.0], [0.0, 1.0, 1.0]])
    b = np.array([1.0, 1.0])
    c = np.ones(3)
    l = np.zeros(3)
    w = np.full(3, np.inf)
    out = []
    out.append(("P3", A, b, c, np.array([0.0, 2.0, 0.0]), np.array([np.inf, 1.0, np.inf]), PS.PRIMAL_INFEASIBLE))
    Ae = np.vstack([A, np.zeros(3)])
    out.append(("P1", Ae, np.array([1.0, 1.0, 0.5]), c, l, w, PS.PRIMAL_INFEASIBLE))
    As = np.vstack([A, [0.0, 0.0, 2.0]])
    out.append(("P6", As, np.array([1.0, 1.0, -1.0]), c, l, w, PS.PRIMAL_INFEASIBLE))
    Ad = np.array([[1.0, 1.0], [1.0, -1.0], [1.0, 2.0]])
    out.append(("P7", Ad, np.array([2.0, 0.0, 5.0]), np.ones(2), np.zeros(2), np.full(2, np.inf), PS.PRIMAL_INFEASIBLE))
    Ac = np.hstack([A, np.zeros((2, 1))])
    out.append(("P2", Ac, b, np.array([1.0, 1.0, 1.0, -1.0]), np.zeros(4), np.full(4, np.inf), PS.DUAL_INFEASIBLE))
    return out


@pytest.mark.parametrize("case", _infeasible_cases(), ids=lambda c: c[0])
def test_infeasibility_found_by_the_rule(abip, case):
    rule, A, b, c, l, w, status = case
    P = PS.presolve(A, b, c, l, w)
    assert P.status == status and P.why.startswith(rule), P.why
    Q = abip.Presolved(A, b, c, l, w)
    assert Q.status == status and Q.why.startswith(rule), Q.why


def test_dependent_block_kept_rows_and_consistency():
    """Three rows on two columns: the third is 1.5 r1 - 0.5 r2; with a consistent b the
    first two (in index order) are kept and the third is dropped."""
    A = np.array([[1.0, 1.0], [1.0, -1.0], [1.0, 2.0]])
    x0 = np.array([1.5, 0.5])
    P = PS.presolve(A, A @ x0, np.array([1.0, 2.0]), np.zeros(2), np.full(2, np.inf))
    assert P.status == 0 and P.removed["P7"] == 1 and list(P.rows) == [0, 1]


def test_ruiz_passes_equilibrate():
    g = W.general_lp(seed=3)
    g.A[:, :5] *= 1e3
    g.A[3] *= 1e-2
    g.b = g.A @ g.x0
    g.c = g.A.T @ g.y0 + g.z0
    P0 = PS.presolve(g.A, g.b, g.c, g.l, g.w, ruiz=0)
    assert np.all(P0.D == 1.0) and np.all(P0.E == 1.0)
    P = PS.presolve(g.A, g.b, g.c, g.l, g.w, ruiz=20)
    Ab = abs(P.A)
    rmax = np.asarray(Ab.max(axis=1).todense()).ravel()
    cmax = np.asarray(Ab.max(axis=0).todense()).ravel()
    assert np.all(np.abs(np.log(rmax)) <= np.log(1.5)) and np.all(np.abs(np.log(cmax)) <= np.log(1.5))
    r0 = np.asarray(abs(P0.A).max(axis=1).todense()).ravel()
    assert r0.max() / r0.min() > 1e3


@pytest.mark.parametrize("make", [lambda: W.general_lp(seed=1), lambda: W.general_lp(seed=2),
                                  lambda: W.general_lp(m=12, n=30, seed=5, extras=False),
                                  lambda: W.sice_general_lp(*W.sice(12), 4)], ids=["g1", "g2", "g5", "sice"])
def test_library_presolve_matches_oracle(abip, make):
    g = make()
    P = PS.presolve(g.A, g.b, g.c, g.l, g.w)
    Q = abip.Presolved(g.A, g.b, g.c, g.l, g.w)
    assert Q.status == P.status == 0
    i = Q.info
    assert (i["empty_rows"], i["empty_cols"], i["fixed_cols"], i["singleton_rows"], i["dependent_rows"],
            i["free_split"]) == (P.removed["P1"], P.removed["P2"], P.removed["P4"], P.removed["P6"],
                                 P.removed["P7"], P.removed["P5"])
    M, b, c = Q.lp()
    assert (M.m, M.n) == P.A.shape
    assert np.array_equal(M.row_ptr, P.A.indptr) and np.array_equal(M.col_idx, P.A.indices)
    assert np.abs(M.val - P.A.data).max() <= 1e-15 * np.abs(P.A.data).max()
    assert np.abs(b - P.b).max() <= 1e-14 * (1 + np.abs(P.b).max())
    assert np.abs(c - P.c).max() <= 1e-14 * (1 + np.abs(P.c).max())
    assert abs(i["obj_offset"] - P.obj_offset) <= 1e-14 * (1 + abs(P.obj_offset))
    # postsolve of one and the same standard-form point
    rng = np.random.default_rng(0)
    xs, ys = rng.uniform(0, 2, M.n), rng.standard_normal(M.m)
    xo, yo, zo, obj = PS.postsolve(P, xs, ys, None)
    x2, y2, z2, obj2 = Q.postsolve(xs, ys)
    assert np.abs(x2 - xo).max() <= 1e-13 * (1 + np.abs(xo).max())
    assert np.abs(y2 - yo).max() <= 1e-13 * (1 + np.abs(yo).max())
    assert np.abs(z2 - zo).max() <= 1e-12 * (1 + np.abs(zo).max())


def test_sice_columns_share_one_standard_form():
    """Every column j of SICE presolves to the same scaled matrix (the bounds on r become
    d upper-bound rows; nothing is removed), so the d subproblems form a shared-A batch;
    the optimum of one column agrees with HiGHS."""
    S, lam = W.sice(12)
    Ps = [PS.presolve(*(lambda g: (g.A, g.b, g.c, g.l, g.w))(W.sice_general_lp(S, lam, j))) for j in range(12)]
    for P in Ps:
        assert P.A.shape == (24, 48) and sum(P.removed.values()) == 0
        assert (P.A != Ps[0].A).nnz == 0
    g = W.sice_general_lp(S, lam, 4)
    r = O.solve(Ps[4].A, Ps[4].b, Ps[4].c, O.Params(eps=1e-8))
    x, y, z, obj = PS.postsolve(Ps[4], r.x, r.y, r.s)
    assert abs(obj - _linprog(g)) <= 1e-6 * (1 + abs(obj))


def test_reductions_alone_solve_a_determined_lp(abip):
    """Singleton rows fix every variable (one only after another's substitution leaves its
    row a singleton): no row is left, the status is decided in presolve, and the postsolve
    of the empty standard form returns the unique feasible point and duals that make the
    reduced cost of every fixed column zero."""
    A = np.array([[2.0, 0.0, 0.0], [1.0, 1.0, 0.0], [0.0, 1.0, -1.0]])
    x0 = np.array([1.0, 2.0, 0.5])
    b, c = A @ x0, np.array([1.0, -1.0, 2.0])
    l, w = np.full(3, -np.inf), np.full(3, np.inf)
    P = PS.presolve(A, b, c, l, w)
    assert P.status == PS.OPTIMAL_BY_REDUCTION and P.removed["P6"] == 3 and P.A.shape == (0, 0)
    x, y, z, obj = PS.postsolve(P, np.zeros(0), np.zeros(0), None)
    assert np.allclose(x, x0, rtol=0, atol=1e-15) and abs(obj - c @ x0) <= 1e-14
    assert np.abs(z).max() <= 1e-14                      # c - A^T y = 0: y certifies x0
    Q = abip.Presolved(A, b, c, l, w)
    assert Q.status == abip.ABIP_OPTIMAL and Q.info["m"] == 0 and Q.info["n"] == 0
    x2, y2, z2, obj2 = Q.postsolve(np.zeros(0), np.zeros(0))
    assert np.allclose(x2, x) and np.allclose(y2, y) and abs(obj2 - obj) <= 1e-14


def test_library_presolve_takes_csr_and_refuses_bad_arguments(abip):
    """The same LP as a CSR matrix (float64 and float32 values exact in float32) gives the
    standard form of the dense input; malformed bounds and tolerances are refused."""
    g = W.general_lp(m=12, n=30, seed=6)
    g.A = g.A.astype(np.float32).astype(np.float64)
    g.b = g.A @ g.x0
    g.c = g.A.T @ g.y0 + g.z0
    Pd = abip.Presolved(g.A, g.b, g.c, g.l, g.w)
    Md, bd, cd = Pd.lp()
    for dtype in (np.float64, np.float32):
        Pc = abip.Presolved(W.dense_to_csr(g.A, dtype), g.b, g.c, g.l, g.w)
        Mc, bc, cc = Pc.lp()
        assert np.array_equal(Mc.row_ptr, Md.row_ptr) and np.array_equal(Mc.col_idx, Md.col_idx)
        assert np.array_equal(Mc.val, Md.val) and np.array_equal(bc, bd) and np.array_equal(cc, cd)
    bad_l = g.l.copy()
    bad_l[0] = np.inf
    bad_w = g.w.copy()
    bad_w[1] = np.nan
    for args, kw in (((g.A, g.b, g.c, bad_l, g.w), {}), ((g.A, g.b, g.c, g.l, bad_w), {}),
                     ((g.A, g.b, g.c, g.l, g.w), {"tol": 0.0}), ((g.A, g.b, g.c, g.l, g.w), {"ruiz": -1})):
        with pytest.raises(abip.AbipError) as e:
            abip.Presolved(*args, **kw)
        assert e.value.code == abip.ABIP_E_INVALID_ARG


def test_oracle_refuses_a_gamma_max_below_gamma():
    lp = W.planted_dense(6, 14, seed=7)
    with pytest.raises(ValueError):
        O.solve(lp.A, lp.b, lp.c, O.Params(gamma=0.2, gamma_max=0.1))


def test_empty_columns_take_the_bound_their_cost_prefers(abip):
    """P2 (reading P-A): an empty column sits at l for c_j > 0, at w for c_j < 0 and, with
    c_j = 0, at the point of [l, w] nearest 0; the objective constant follows."""
    A = np.array([[1.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0]])
    b = np.array([1.0])
    c = np.array([1.0, 1.0, 2.0, -3.0, 0.0, 0.0, 0.0])
    l = np.array([0.0, 0.0, 1.5, -np.inf, 2.0, -3.0, -np.inf])
    w = np.array([np.inf, np.inf, np.inf, 4.0, 5.0, -1.0, np.inf])
    want = {2: 1.5, 3: 4.0, 4: 2.0, 5: -1.0, 6: 0.0}
    P = PS.presolve(A, b, c, l, w)
    assert P.status == 0 and P.removed["P2"] == 5
    assert {j: P.fixed[j] for j in want} == want
    assert P.obj_offset == pytest.approx(2.0 * 1.5 - 3.0 * 4.0)
    Q = abip.Presolved(A, b, c, l, w)
    assert Q.info["empty_cols"] == 5 and Q.info["obj_offset"] == pytest.approx(P.obj_offset)
    r = O.solve(P.A, P.b, P.c, O.Params(eps=1e-9))
    x, y, z, obj = PS.postsolve(P, r.x, r.y, r.s)
    assert all(x[j] == v for j, v in want.items())
    assert obj == pytest.approx(1.0 + P.obj_offset, abs=1e-7)      # x0 + x1 = 1 at cost 1
