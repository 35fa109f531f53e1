"""Pins for the FP64 oracle against facts the paper and the mathematics fix.

Each test names the passage it follows.  None of them re-types the formula it
checks: they use identities (skew-symmetry, the central start, Theorem 2.1(i),
Theorem 3.1), an independent scalar root finder, a dense linear solve, brute-force
basis enumeration and planted optima.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import abip_oracle as O
from oracle.lp_bruteforce import enumerate_lp
from paper_1805_12344_gb300 import workloads as W


def _problem(m=7, n=15, seed=11):
    lp = W.planted_dense(m, n, seed=seed)
    return lp, O.Problem(lp.A, lp.b, lp.c)


# --- Sec. 3.1: the embedding -------------------------------------------------

def test_central_start_satisfies_Qu_eq_v():
    """Algorithm 2 starts on {Q u = v}: u = (0, e, 1, 1), v = (0, e, 1, -n-1) (Sec. 3.1,
    Theorem 2.1(ii)).  This fixes bbar, cbar, zbar and xi with their signs."""
    for seed in range(3):
        lp, P = _problem(6 + seed, 13 + 2 * seed, seed)
        ry, rx, rt, rth = O.residual_Qu_v(P, np.zeros(P.m), np.ones(P.n), 1.0, 1.0,
                                          np.zeros(P.m), np.ones(P.n), 1.0, P.xi)
        scale = 1 + np.abs(lp.A).sum() + np.abs(lp.b).sum() + np.abs(lp.c).sum()
        assert np.max(np.abs(ry)) <= 1e-13 * scale
        assert np.max(np.abs(rx)) <= 1e-13 * scale
        assert abs(rt) <= 1e-13 * scale and abs(rth) <= 1e-13 * scale


def test_Q_is_skew_symmetric():
    """Q^T = -Q (Sec. 3.1), so u^T Q u = 0 for every u."""
    lp, P = _problem()
    Q = O.dense_Q(P)
    assert np.max(np.abs(Q + Q.T)) == 0.0
    rng = np.random.default_rng(0)
    for _ in range(5):
        u = rng.standard_normal(Q.shape[0])
        assert abs(u @ Q @ u) <= 1e-12 * (u @ u) * np.abs(Q).max()
    # Q's blocks are A, b, c and the embedding constants in the places Sec. 3.1 puts them
    m, n = P.m, P.n
    assert np.array_equal(Q[:m, m:m + n], lp.A)
    assert np.array_equal(Q[:m, m + n], -lp.b) and np.array_equal(Q[m:m + n, m + n], lp.c)


def test_theorem_2_1_identity_at_central_point():
    """Theorem 2.1(i): at any point with Q u = v, r = 0, xi = -(x0)^T s0 - 1,
    ((x0)^T s0 + 1) theta = x^T s + tau kappa; on the central path (system HSD-log-kkt)
    this forces theta = mu/beta."""
    lp, P = _problem(8, 18, 3)
    for mu in (0.5, 1e-2):
        cp = O.central_point(lp.A, lp.b, lp.c, mu)
        assert cp["residual"] < 1e-11
        lhs = (P.n + 1) * cp["theta"]
        rhs = cp["x"] @ cp["s"] + cp["tau"] * cp["kappa"]
        assert abs(lhs - rhs) <= 1e-11 * (1 + abs(rhs))
        assert abs(cp["theta"] - mu) <= 1e-11


# --- Eq. Simple-Update:Affine and Sec. 4.4: the projection -------------------

@pytest.mark.parametrize("linsys", [0, 1])
def test_projection_equals_dense_inverse(linsys):
    """Block elimination with the cached M^{-1} H (Sec. 4.4) reproduces (I+Q)^{-1} w
    from a dense solve, and (I+Q^T Q)^{-1} (I-Q) w (Eq. Simple-Update:Affine)."""
    lp, P = _problem(9, 21, 5)
    prm = O.Params(linsys=linsys, cg_tol=1e-14)
    proj = O.Projection(P, O.make_linsys(P, prm))
    rng = np.random.default_rng(1)
    Q = O.dense_Q(P)
    N = Q.shape[0]
    for _ in range(3):
        w = rng.standard_normal(N) * 3
        uy, ux, ut, uth = proj(w[:P.m], w[P.m:P.m + P.n], w[-2], w[-1])
        u = np.concatenate([uy, ux, [ut, uth]])
        ref = np.linalg.solve(np.eye(N) + Q, w)
        ref2 = np.linalg.solve(np.eye(N) + Q.T @ Q, (np.eye(N) - Q) @ w)
        assert np.linalg.norm(u - ref) <= 1e-11 * np.linalg.norm(ref)
        assert np.linalg.norm(u - ref2) <= 1e-10 * np.linalg.norm(ref)


def test_projection_is_euclidean_projection():
    """(u~, Q u~) is the closest point of {Q u = v} to (w, w): the optimality condition
    (u~ - w) + Q^T (Q u~ - w) = 0 (proof of Theorem 3.1, Step 1)."""
    lp, P = _problem(5, 12, 8)
    proj = O.Projection(P, O.make_linsys(P, O.Params()))
    Q = O.dense_Q(P)
    w = np.random.default_rng(2).standard_normal(Q.shape[0])
    u = np.concatenate(list(proj(w[:P.m], w[P.m:P.m + P.n], w[-2], w[-1])[:2]) +
                       [np.array(proj(w[:P.m], w[P.m:P.m + P.n], w[-2], w[-1])[2:])])
    g = (u - w) + Q.T @ (Q @ u - w)
    assert np.linalg.norm(g) <= 1e-11 * np.linalg.norm(w)


def test_pcg_matches_library_solve():
    """Jacobi-PCG on G = I + A A^T converges to the dense solution (Sec. 4.4)."""
    lp = W.planted_sparse(300, seed=5)
    A = lp.A.to_scipy()
    P = O.Problem(A, lp.b, lp.c)
    pcg = O.JacobiPCG(P, 1e-13, 1000)
    q = np.random.default_rng(3).standard_normal(P.m)
    z = pcg.solve(q)
    G = np.eye(P.m) + (A @ A.T).toarray()
    ref = np.linalg.solve(G, q)
    assert np.linalg.norm(z - ref) <= 1e-11 * np.linalg.norm(ref)


# --- Eqs. Simple-Update:Barrier-X and Simple-Update:Dual ----------------------

def _scalar_root(omega, c):
    """Positive root of f(x) = x - omega - c/x by bisection then Newton, in plain floats."""
    lo, hi = 0.0, max(1.0, abs(omega)) * 2 + math.sqrt(c) * 2 + 1.0
    for _ in range(3000):
        mid = 0.5 * (lo + hi)
        if mid == lo or mid == hi:
            break
        if mid - omega - c / mid > 0 if mid > 0 else False:
            hi = mid
        else:
            lo = mid
    x = hi
    for _ in range(5):
        f = x - omega - c / x
        x = x - f / (1 + c / (x * x))
    return x


def test_barrier_prox_matches_scalar_root():
    """x = argmin -c log x + (x - omega)^2 / 2 solves x - omega - c/x = 0, and the dual
    step gives s = x - omega with x s = c (Thm 3.1 invariant x o s = mu/beta)."""
    omegas = [s * 10.0 ** k for k in range(-12, 13, 3) for s in (-1, 1)] + [0.0]
    cs = [1e-20, 1e-12, 1e-6, 1e-2, 1.0, 1e2]
    for c in cs:
        x, s = O.barrier_prox(np.array(omegas), c)
        for om, xi, si in zip(omegas, x, s):
            ref = _scalar_root(om, c)
            assert abs(xi - ref) <= 4 * np.spacing(ref) + 1e-300, (om, c, xi, ref)
            assert abs(xi * si - c) <= 4e-15 * c
            assert xi > 0 and si > 0


# --- Theorem 3.1: Algorithm 1 with explicit multipliers -----------------------

@pytest.mark.parametrize("alpha", [1.0, 1.8])
def test_theorem_3_1_multiplier_elimination(alpha):
    """With p0 = v0, q0 = u0 and x o s = tau kappa = mu/beta, Algorithm 1 keeps p = v,
    q = u, x o s = mu/beta, tau kappa = mu/beta, r = 0, xi = -n-1 (Theorem 3.1) and its
    iterates equal those of Algorithm 2 (with the Sec. 4.2 relaxation when alpha != 1)."""
    lp, P = _problem(6, 14, 21)
    gamma = 0.2
    st = O.initial_state(P)
    O.warm_start(st, gamma, 0)                      # now x o s = gamma = mu/beta
    mu = gamma
    start = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in st.items()}
    alg1 = O.algorithm1(lp.A, lp.b, lp.c, mu, 25, alpha=alpha, start=start)
    prm = O.Params(alpha=alpha)
    proj = O.Projection(P, O.make_linsys(P, prm))
    m, n = P.m, P.n
    for (u, v, p, q) in alg1:
        O.admm_step(P, proj, st, mu, prm)
        u2 = np.concatenate([st["y"], st["x"], [st["tau"], st["theta"]]])
        v2 = np.concatenate([np.zeros(m), st["s"], [st["kappa"], P.xi]])
        sc = 1 + np.linalg.norm(u)
        assert np.linalg.norm(p - v) <= 1e-11 * sc
        assert np.linalg.norm(q - u) <= 1e-11 * sc
        assert np.max(np.abs(u[m:m + n] * v[m:m + n] - mu)) <= 1e-12
        assert abs(u[m + n] * v[m + n] - mu) <= 1e-12
        assert np.all(v[:m] == 0) and v[-1] == -(n + 1)
        assert np.linalg.norm(u - u2) <= 1e-10 * sc
        assert np.linalg.norm(v - v2) <= 1e-10 * (1 + np.linalg.norm(v))


# --- Lemma 3.3: monotone decrease at fixed mu --------------------------------

def test_lemma_3_3_monotone_distance_to_central_point():
    """||u_i - u*||^2 + ||v_i - v*||^2 is non-increasing and tends to 0, with (u*, v*)
    the central point at mu (Lemma 3.3; alpha = 1 as analysed)."""
    lp, P = _problem(8, 18, 3)
    mu = 0.1
    st = O.initial_state(P)
    O.warm_start(st, mu, 0)
    prm = O.Params(alpha=1.0)
    proj = O.Projection(P, O.make_linsys(P, prm))
    # reference point: run ADMM a while, then polish with Newton
    tmp = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in st.items()}
    for _ in range(3000):
        O.admm_step(P, proj, tmp, mu, prm)
    cp = O.central_point(lp.A, lp.b, lp.c, mu, start=tmp)
    assert cp["residual"] < 1e-12
    zs = np.concatenate([cp["y"], cp["x"], [cp["tau"], cp["theta"]], cp["s"], [cp["kappa"]]])
    proj = O.Projection(P, O.make_linsys(P, prm))
    d_prev = np.inf
    d0 = None
    for i in range(400):
        d = np.sum((O.stacked(st) - zs) ** 2)
        d0 = d if d0 is None else d0
        assert d <= d_prev * (1 + 1e-12) + 1e-28
        d_prev = d
        O.admm_step(P, proj, st, mu, prm)
    assert d_prev < 0.5 * d0
    for _ in range(20000):
        O.admm_step(P, proj, st, mu, prm)
    assert np.sum((O.stacked(st) - zs) ** 2) < 1e-16
    assert abs(st["theta"] - mu) < 1e-8           # theta -> mu/beta (system HSD-log-kkt)


# --- Theorem 3.6: number of outer iterations --------------------------------

def test_outer_count_theorem_3_6():
    """Stopping once mu^k <= eps takes T_IPM = ceil(log(mu0/eps)/log(1/gamma)) outer steps."""
    lp, P = _problem(5, 11, 4)
    for gamma, eps in ((0.5, 1e-3), (0.3, 2e-4)):
        r = O.solve(lp.A, lp.b, lp.c, O.Params(gamma=gamma, eps=eps, stop_rule=1))
        assert r.outer_iters == math.ceil(math.log(1.0 / eps) / math.log(1.0 / gamma))


# --- Sec. 4.1 end to end: planted optima, certificates, brute force ----------

def test_planted_dense_optimum():
    """The planted pair is optimal (strong duality: c^T x0 = b^T y0); with |supp x0| < m
    the primal optimum x0 is unique.  The relative objective error stays within 1e-5 and the
    returned residuals are within eps (Sec. 4.1)."""
    lp = W.planted_dense()
    r = O.solve(lp.A, lp.b, lp.c)
    assert r.status == O.OPTIMAL
    assert abs(r.obj - lp.p_star) <= 1e-5 * abs(lp.p_star)
    assert max(r.pres, r.dres, r.dgap) <= 1e-6
    assert np.linalg.norm(r.x - lp.x0) <= 1e-3 * np.linalg.norm(lp.x0)
    assert r.kappa / r.tau < 1e-6                   # kappa -> 0 at optimality (Thm 2.2(i))
    assert r.x @ r.s <= 1e-5 * (1 + abs(lp.p_star))  # complementarity x^T s -> 0


def test_planted_sparse_optimum_small():
    """[R I] planted LP (m = 80): the returned objective matches p* = c^T x0 = b^T y0."""
    lp = W.planted_sparse(80, seed=W.seed_for(W.SPARSE_PLANTED, 10))
    A = lp.A.to_scipy()
    r = O.solve(A, lp.b, lp.c, O.Params(linsys=1, cg_tol=1e-10))
    assert r.status == O.OPTIMAL
    assert abs(r.obj - lp.p_star) <= 1e-5 * abs(lp.p_star)
    assert max(r.pres, r.dres, r.dgap) <= 1e-6


def test_sparse_and_dense_storage_give_same_iterates():
    lp = W.planted_sparse(40, seed=3)
    Ad = lp.A.to_dense()
    a = O.run_iterations(Ad, lp.b, lp.c, 30)
    b = O.run_iterations(sp.csr_matrix(Ad), lp.b, lp.c, 30)
    assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(a)


def test_primal_infeasible_twin_certificate():
    """The twin has A_1 >= 0, b_1 = -1: primal infeasible.  ABIP ends with kappa > 0,
    tau -> 0 (Thm 2.2(ii)) and y / b^T y is an approximate Farkas certificate (Sec. 4.1)."""
    lp = W.infeasible_twin()
    r = O.solve(lp.A, lp.b, lp.c)
    assert r.status == O.PRIMAL_INFEASIBLE
    assert r.kappa > 0 and r.tau < 1e-6 * r.kappa
    y = r.y
    assert abs(lp.b @ y - 1.0) < 1e-12
    assert np.linalg.norm(lp.A.T @ y + r.s) <= 1e-6 / np.linalg.norm(lp.b) * 1.0001
    assert np.all(r.s >= 0)


def test_dual_infeasible_certificate():
    lp = W.dual_infeasible()
    r = O.solve(lp.A, lp.b, lp.c)
    assert r.status == O.DUAL_INFEASIBLE
    assert r.kappa > 0 and r.tau < 1e-6 * r.kappa
    assert abs(lp.c @ r.x + 1.0) < 1e-12
    assert np.all(r.x >= 0)
    assert np.linalg.norm(lp.A @ r.x) <= 1e-6 / np.linalg.norm(lp.c) * 1.0001


@pytest.mark.parametrize("seed", range(12))
def test_tiny_lps_against_basis_enumeration(seed):
    """p* from enumerating every basis equals ABIP's objective; infeasible or unbounded
    instances give the matching certificate status (Thm 2.2, Sec. 4.1)."""
    rng = np.random.default_rng(seed)
    m = int(rng.integers(1, 5))
    n = int(rng.integers(m + 1, m + 7))
    lp = W.tiny_random(m, n, seed=W.seed_for(W.TINY, seed)) if seed % 2 else W.tiny_planted(m, n, W.seed_for(W.TINY, seed))
    ref = enumerate_lp(lp.A, lp.b, lp.c)
    r = O.solve(lp.A, lp.b, lp.c)
    if ref["status"] == "optimal":
        assert r.status == O.OPTIMAL
        assert abs(r.obj - ref["p_star"]) <= 1e-5 * max(1.0, abs(ref["p_star"]))
    elif ref["status"] == "primal_infeasible":
        assert r.status in (O.PRIMAL_INFEASIBLE, O.DUAL_INFEASIBLE)
    else:
        assert r.status == O.DUAL_INFEASIBLE


# --- Differentiation of the central point (system HSD-log-kkt, Sec. 3.2) -------------

def test_central_point_gradient_matches_central_differences():
    """The adjoint gradient of L(x*) = ||x* - x_t||^2 agrees with FP64 central differences
    (step 1e-6 max(1, |p|)) of the Newton-polished solution map, for every entry of b, c, A."""
    lp = W.l1_svm(d=3, N=8, seed=5)
    mu = 1e-3
    xt = lp.meta["x_target"]
    g = O.central_point_grad(lp.A, lp.b, lp.c, mu, lambda xs: 2.0 * (xs - xt))
    start = {k: g["point"][k] for k in ("y", "x", "tau", "theta", "s", "kappa")}

    def loss(A, b, c):
        cp = O.central_point(A, b, c, mu, start=start, tol=1e-15)
        return float(np.sum((cp["x"] / cp["tau"] - xt) ** 2))

    base = {"A": lp.A, "b": lp.b, "c": lp.c}
    for which, key in (("b", "db"), ("c", "dc"), ("A", "dA")):
        P = base[which]
        fd = np.zeros_like(P)
        for idx in np.ndindex(P.shape):
            h = 1e-6 * max(1.0, abs(P[idx]))
            args = {}
            for sgn in (1, -1):
                Pp = P.copy()
                Pp[idx] += sgn * h
                args[sgn] = dict(base, **{which: Pp})
            fd[idx] = (loss(**args[1]) - loss(**args[-1])) / (2 * h)
        err = np.abs(fd - g[key]).max() / np.abs(g[key]).max()
        assert err <= 1e-5, (which, err)


def test_central_point_gradient_vertex_limit():
    """At a nondegenerate vertex x0 (basis B, strictly complementary) the central point tends
    to x0 with x0_B = B^{-1} b, so as mu -> 0 the gradient tends to dL/db = B^{-T} g_B,
    dL/dA = -(B^{-T} g_B) x0^T and dL/dc = 0 (g = dL/dx at x0); the gap is O(mu)."""
    m, n = 6, 14
    rng = np.random.default_rng(7)
    A = rng.standard_normal((m, n))
    basic = np.zeros(n, dtype=bool)
    basic[rng.permutation(n)[:m]] = True
    x0 = np.where(basic, rng.uniform(0.5, 2.0, n), 0.0)
    s0 = np.where(basic, 0.0, rng.uniform(0.5, 2.0, n))
    y0 = rng.standard_normal(m)
    b, c = A @ x0, A.T @ y0 + s0
    xt = rng.standard_normal(n)
    g = O.central_point_grad(A, b, c, 1e-8, lambda xs: 2.0 * (xs - xt))
    w = np.linalg.solve(A[:, basic].T, 2.0 * (x0 - xt)[basic])
    scale = np.abs(w).max()
    assert np.abs(g["db"] - w).max() <= 1e-6 * scale
    assert np.abs(g["dc"]).max() <= 1e-6 * scale
    dA = -np.outer(w, x0)
    assert np.abs(g["dA"] - dA).max() <= 1e-6 * np.abs(dA).max()


def test_random_udv_lp_reaches_its_planted_value():
    """The random LP of Sec. 5.1: x0 >= 0, s0 >= 0 with x0 o s0 = 0, b = A x0, c = A^T y0 + s0,
    so x0 and (y0, s0) are optimal and the optimum is c^T x0 = b^T y0 exactly.  (At m = 20
    the 0.2-dense U is singular for some seeds; seed 12 gives A full row rank, as the
    paper's sizes do with high probability.)"""
    lp = W.random_udv(20, 60, seed=12)
    assert np.all(lp.x0 >= 0) and np.all(lp.s0 >= 0) and np.all(lp.x0 * lp.s0 == 0)
    assert (lp.x0 == 0).sum() == 36 and abs(lp.c @ lp.x0 - lp.b @ lp.y0) <= 1e-9 * abs(lp.c @ lp.x0)
    assert np.linalg.matrix_rank(lp.A) == 20
    r = O.solve(lp.A, lp.b, lp.c)
    assert r.status == O.OPTIMAL
    assert abs(r.obj - lp.p_star) <= 1e-5 * max(1.0, abs(lp.p_star))


def test_basis_pursuit_recovers_sparse_vector():
    """Basis pursuit LP (min ||x||_1, D x = b as [D, -D] in standard form): x_true is feasible,
    so the optimum is at most ||x_true||_1; with 5 % nonzeros and m = n_d / 4 Gaussian
    measurements l1 recovery succeeds, so the oracle's solution is x_true itself."""
    sb = W.basis_pursuit(32, 128, batch=1, density=0.05, seed=7)
    r = O.solve(sb.A, sb.bs[0], sb.cs[0])
    assert r.status == O.OPTIMAL
    xt = sb.meta["x_true"][0]
    nd = sb.meta["n_d"]
    assert r.obj <= np.abs(xt).sum() * (1 + 1e-6) + 1e-9
    assert np.abs((r.x[:nd] - r.x[nd:]) - xt).max() <= 1e-4
    assert abs(r.obj - np.abs(xt).sum()) <= 1e-5 * np.abs(xt).sum()


# --- special cases whose optimum the mathematics fixes ---------------------------------

def test_square_system_has_the_unique_feasible_point():
    """m = n with A nonsingular: x = A^{-1} b is the only feasible point; when it is
    positive it is the optimum whatever c is."""
    rng = np.random.default_rng(41)
    n = 6
    A = rng.standard_normal((n, n)) + 3.0 * np.eye(n)
    x0 = rng.uniform(0.5, 2.0, n)
    b = A @ x0
    c = rng.standard_normal(n)
    r = O.solve(A, b, c)
    assert r.status == O.OPTIMAL
    assert np.abs(r.x - x0).max() <= 1e-4 * np.abs(x0).max()
    assert abs(r.obj - c @ x0) <= 1e-5 * max(1.0, abs(c @ x0))


def test_duplicated_row_leaves_the_optimum_unchanged():
    """Repeating an equality (a redundant row of A, b) changes neither the feasible set nor
    the optimal value; I + A A^T stays positive definite."""
    lp = W.planted_dense(8, 20, seed=17)
    A2 = np.vstack([lp.A, lp.A[2:3]])
    b2 = np.concatenate([lp.b, lp.b[2:3]])
    r1 = O.solve(lp.A, lp.b, lp.c)
    r2 = O.solve(A2, b2, lp.c)
    assert r1.status == r2.status == O.OPTIMAL
    p_star = lp.c @ lp.x0
    for r in (r1, r2):
        assert abs(r.obj - p_star) <= 1e-5 * max(1.0, abs(p_star))


def test_scaling_the_cost_scales_the_optimal_value():
    """min (2c)^T x has the same solution set as min c^T x and twice its optimal value."""
    lp = W.planted_dense(8, 20, seed=19)
    r1 = O.solve(lp.A, lp.b, lp.c)
    r2 = O.solve(lp.A, lp.b, 2.0 * lp.c)
    assert r1.status == r2.status == O.OPTIMAL
    assert abs(r2.obj - 2.0 * r1.obj) <= 1e-5 * max(1.0, abs(r2.obj))
    assert np.abs(r2.x - r1.x).max() <= 1e-3 * max(1.0, np.abs(r1.x).max())


# --- Barzilai-Borwein choice of beta (Sec. 4.3) ----------------------------------------

def test_bb_estimate_collinear_and_orthogonal_cases():
    """Collinear curvature pairs dv = c1 du_tilde and dv = c2 du (the equality case of
    Cauchy-Schwarz): both spectral steps equal the scale, the hybrid keeps it, both
    correlations are 1, so beta_hat = sqrt(c1 c2).  Orthogonal pairs (correlation 0) fail
    the safeguard and keep beta."""
    rng = np.random.default_rng(5)
    d = rng.standard_normal(40)
    # dv = 3 du_tilde and dv = (3 / 0.75) du
    assert O.bb_estimate(3.0 * d, d, 0.75 * d, 1.0, 0.2) == pytest.approx(np.sqrt(3.0 * (3.0 / 0.75)), rel=1e-12)
    e = rng.standard_normal(40)
    e -= (e @ d) / (d @ d) * d
    assert O.bb_estimate(d, e, e, 0.7, 0.2) == 0.7
    # one reliable pair: its own hybrid step
    assert O.bb_estimate(2.0 * d, d, e, 0.7, 0.2) == pytest.approx(2.0, rel=1e-12)


def test_bb_hybrid_step_rule():
    """The hybrid spectral step of Sec. 4.3: the minimum-gradient step when 2 MG > SD, else
    SD - MG/2.  With du = d and dv = d + t e (e orthogonal to d, |e| = |d|):
    SD = 1 + t^2, MG = 1; t = 0.5 gives MG, t = 1.5 gives SD - MG/2 = 2.75."""
    rng = np.random.default_rng(8)
    d = rng.standard_normal(30)
    e = rng.standard_normal(30)
    e -= (e @ d) / (d @ d) * d
    e *= np.linalg.norm(d) / np.linalg.norm(e)
    orth = rng.standard_normal(30)
    orth -= (orth @ d) / (d @ d) * d + (orth @ e) / (e @ e) * e
    # psi's pair is orthogonal (fails the safeguard), so beta_hat = phi alone
    assert O.bb_estimate(d + 0.5 * e, d, orth, 1.0, 0.2) == pytest.approx(1.0, rel=1e-12)
    assert O.bb_estimate(d + 1.5 * e, d, orth, 1.0, 0.2) == pytest.approx(1.0 + 1.5 ** 2 - 0.5, rel=1e-12)


class _ScriptedBB:
    """Stand-ins for admm_step and bb_estimate that let a test drive bb_select's branches:
    every trial update adds its beta to theta (so the returned state tells which beta
    advanced it), and the estimates come from a script."""

    def __init__(self, monkeypatch, estimates):
        self.betas = []
        self.estimates = iter(estimates)
        monkeypatch.setattr(O, "admm_step", self.step)
        monkeypatch.setattr(O, "bb_estimate", lambda *a, **k: next(self.estimates))

    def step(self, P, proj, st, mu, prm, beta=None):
        self.betas.append(beta)
        st["theta"] = st["theta"] + beta
        return np.zeros(P.m), np.zeros(P.n), 0.0, 0.0


def _bb_setup():
    lp = W.planted_dense(4, 9, seed=3)
    P = O.Problem(lp.A, lp.b, lp.c)
    prm = O.Params(bb_beta=True)
    return P, O.Projection(P, O.make_linsys(P, prm)), prm


@pytest.mark.parametrize("script,beta,spent,used", [
    ([1.0], 1.0, 2, [1.0, 1.0]),                                  # beta_hat == beta: keep it
    ([1.06], 1.03, 2, [1.0, 1.0]),                                # |beta_hat - beta| <= 0.1: average
    ([3.0, 3.04], 3.02, 4, [1.0, 1.0, 3.0, 3.0]),                 # redo with 3, then average
    ([3.0, 5.0, 7.0, 9.0, 11.0, 13.0], 11.0, 12,                  # five redos, then stop with the
     [1.0, 1.0, 3.0, 3.0, 5.0, 5.0, 7.0, 7.0, 9.0, 9.0, 11.0, 11.0]),   # beta that made the state
])
def test_bb_select_branches(monkeypatch, script, beta, spent, used):
    """Sec. 4.3 heuristic selection (reading B5): keep, average, redo from the same start,
    and the bound on redo rounds; each round restarts from the outer step's start point."""
    P, proj, prm = _bb_setup()
    fake = _ScriptedBB(monkeypatch, script)
    st0 = O.initial_state(P)
    b, st, n = O.bb_select(P, proj, st0, 1.0, 1.0, prm)
    assert b == pytest.approx(beta, rel=1e-15) and n == spent
    assert fake.betas == used
    # the returned state is the last round's: two updates from st0 with that round's beta
    assert st["theta"] == pytest.approx(st0["theta"] + 2 * used[-1], rel=1e-15)
    assert st0["theta"] == 1.0


def test_bb_select_respects_the_update_budget(monkeypatch):
    """A budget of 5 updates allows two rounds (4 updates): the second round's beta is kept
    and no third round starts."""
    P, proj, prm = _bb_setup()
    fake = _ScriptedBB(monkeypatch, [3.0, 5.0, 7.0])
    b, st, n = O.bb_select(P, proj, O.initial_state(P), 1.0, 1.0, prm, budget=5)
    assert (b, n) == (3.0, 4) and fake.betas == [1.0, 1.0, 3.0, 3.0]


def test_bb_beta_solve_never_passes_the_cap():
    lp = W.planted_dense(20, 60, seed=23)
    for cap in (2, 3, 7, 40):
        r = O.solve(lp.A, lp.b, lp.c, O.Params(bb_beta=True, max_admm_iters=cap))
        assert r.admm_iters <= cap


def test_bb_beta_solve_reaches_the_planted_optimum():
    lp = W.planted_dense(20, 60, seed=23)
    r = O.solve(lp.A, lp.b, lp.c, O.Params(bb_beta=True))
    assert r.status == O.OPTIMAL
    p_star = lp.c @ lp.x0
    assert abs(r.obj - p_star) <= 1e-5 * max(1.0, abs(p_star))
    assert len(r.raw["betas"]) == r.outer_iters        # one selection per outer iteration k >= 1
    assert all(b > 0 for b in r.raw["betas"])


# --- Sec. 5: the adaptive decrease ratio (reading B11) -------------------------------

def test_gamma_for_endpoints_and_log_linear_midpoint():
    """The ratio is gamma far from the optimum (residual >= 1e-1), gamma_max at the target
    (residual <= eps), the mean of the two at the geometric mean of 1e-1 and eps, never
    outside [gamma, gamma_max], and gamma itself when the rule is off."""
    prm = O.Params(gamma=0.1, gamma_max=0.5, eps=1e-6)
    assert O.gamma_for(prm, 10.0) == 0.1
    assert O.gamma_for(prm, 1e-1) == 0.1
    assert O.gamma_for(prm, 1e-6) == pytest.approx(0.5, abs=1e-15)
    assert O.gamma_for(prm, 1e-12) == 0.5
    assert O.gamma_for(prm, 0.0) == 0.5
    assert O.gamma_for(prm, math.sqrt(1e-1 * 1e-6)) == pytest.approx(0.3, rel=1e-12)
    rhos = np.logspace(1, -9, 61)
    g = [O.gamma_for(prm, r) for r in rhos]
    assert all(0.1 <= v <= 0.5 for v in g)
    assert all(b >= a for a, b in zip(g, g[1:]))        # smaller residual, larger ratio
    assert O.gamma_for(O.Params(gamma=0.2), 1e-5) == 0.2


def _rel_kkt(A, b, c, st):
    """Sec. 4.1 relative residuals of the candidate (x, y, s) / tau, in plain numpy."""
    tau = st["tau"]
    x, y, s = st["x"] / tau, st["y"] / tau, st["s"] / tau
    pres = np.linalg.norm(A @ x - b) / (1 + np.linalg.norm(b))
    dres = np.linalg.norm(A.T @ y + s - c) / (1 + np.linalg.norm(c))
    gap = abs(c @ x - b @ y) / (1 + abs(c @ x) + abs(b @ y))
    return max(pres, dres, gap)


def test_adaptive_gamma_follows_the_residual_of_the_iterate():
    """Every decrease mu <- g mu takes g from the residual of the iterate it leaves: the
    recorded ratios multiply to mu_final / mu0, each lies in [gamma, gamma_max], and each
    decrease that follows an ADMM update matches the ratio of that update's iterate
    (its residuals recomputed here from Sec. 4.1's definitions)."""
    lp = W.planted_dense(8, 20, seed=5)
    prm = O.Params(gamma=0.1, gamma_max=0.4)
    last = {}

    def on_iter(k, mu, st):
        last[mu] = {key: (v.copy() if isinstance(v, np.ndarray) else v) for key, v in st.items()}

    r = O.solve(lp.A, lp.b, lp.c, prm, on_iter=on_iter)
    gam = r.raw["gammas"]
    assert r.status == O.OPTIMAL and len(gam) == r.outer_iters > 0
    assert math.prod(gam) * prm.beta == pytest.approx(r.mu, rel=1e-12)
    assert all(0.1 <= g <= 0.4 for g in gam)
    assert gam[-1] > 0.1                                  # the rule moved the ratio
    mu, checked = prm.beta, 0
    for g in gam:
        if mu in last:
            assert g == pytest.approx(O.gamma_for(prm, _rel_kkt(lp.A, lp.b, lp.c, last[mu])), rel=1e-9)
            checked += 1
        mu *= g
    assert checked >= len(gam) - 1


def test_adaptive_gamma_off_and_flat_reproduce_the_fixed_ratio():
    """gamma_max = gamma gives the fixed-ratio iteration exactly, and the adaptive run
    reaches the planted optimum (Theorem 3.1 holds for any ratio in (0, 1))."""
    lp = W.planted_dense(8, 20, seed=5)
    a = O.solve(lp.A, lp.b, lp.c, O.Params(gamma=0.2))
    b = O.solve(lp.A, lp.b, lp.c, O.Params(gamma=0.2, gamma_max=0.2))
    assert a.admm_iters == b.admm_iters and np.array_equal(a.x, b.x) and np.array_equal(a.y, b.y)
    c = O.solve(lp.A, lp.b, lp.c, O.Params(gamma=0.1, gamma_max=0.5))
    assert c.status == O.OPTIMAL
    assert abs(c.obj - lp.p_star) <= 1e-5 * max(1.0, abs(lp.p_star))
