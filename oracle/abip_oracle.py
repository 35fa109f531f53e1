"""Plain FP64 CPU oracle for ABIP (Lin, Ma, Ye & Zhang, "An ADMM-Based Interior-Point
Method for Large-Scale Linear Programming", arXiv 1805.12344).

TEST INFRASTRUCTURE ONLY.  This module is the correctness reference for the CUDA
library.  It is imported only by tests/, by ``__graft_entry__.smoke()`` and by the
CPU-baseline / reference legs of ``bench.py``; the product path never calls it and
shares no code with it.

Everything is float64 numpy.  Library primitives used as single steps: dense and
sparse matrix-vector products, ``numpy.linalg.cholesky`` and triangular solves.
The algorithm follows the paper's order and notation:

* HSD embedding with x0 = e, s0 = e, y0 = 0 (Sec. 3.1, the matrix Q and Eq.
  bar-b-c-z-re):  u = (y, x, tau, theta),  v = (r, s, kappa, xi),  r = 0, xi = -n-1.
* Algorithm 2 (Sec. 3.2): inner ADMM loop at fixed mu with the projection of Eq.
  Simple-Update:Affine, the closed-form barrier steps Eqs. Simple-Update:Barrier-Y/X/
  tau/theta, the dual step Eq. Simple-Update:Dual, the inner stop Eq. inner-stop, and
  mu <- gamma mu between inner loops.
* Over-relaxation (Sec. 4.2) with alpha.
* Termination and infeasibility certificates (Sec. 4.1).
* Projection by block elimination and Sherman-Morrison-Woodbury (Sec. 4.4),
  generalised from the printed 3-block form to the 4-block Q (a rank-2 Schur
  complement; reading A1), with M^{-1} applied through G = I + A A^T by a dense
  Cholesky factor or by Jacobi-preconditioned CG (Sec. 4.4, last paragraph).
* The warm-start rule used in the paper's experiments (Sec. 5, the scaling
  heuristic that keeps the larger of x_j, s_j), or the sqrt(gamma) rescale of
  Eq. update-next-iterate.

Readings of silent or ambiguous points (labels shared with the CUDA library's notes):
A1 4-block Q; A2 fixed gamma; A3 beta = mu0 = 1; A4 heuristic warm start for
(x,s),(tau,kappa) and sqrt(gamma) for y, theta, ties keep x; A6 dgap normaliser uses
the tau-scaled candidate; A8 certificate signs and test order; A9 two-root stable
prox; A10 CG stop rule; A13 MAX_ITER status; B5 Barzilai-Borwein beta (Sec. 4.3,
opt-in): continue from the trial iterates, at most 5 redo rounds and never past the
update cap, keeping the beta that produced the state when the rounds run out; B6 the
curvature pairs with the printed signs; B7 the selection starts at the second outer
iteration; B11 the adaptive decrease ratio (opt-in).

Parity status: every function here is pinned by tests in tests/test_oracle_*.py
except the exact iteration trajectory of `solve` (iteration counts, the iterates
themselves), which no closed form fixes: "parity unpinned" beyond the pins listed
there (objective, status, certificates, Thm 3.1 identities, fixed-point limit).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

try:  # scipy is a convenience for triangular solves and CSR products
    import scipy.linalg as _sla
    import scipy.sparse as _sp
except ImportError:  # pragma: no cover
    _sla = None
    _sp = None

# status codes (shared numbering with the C ABI, defined independently there)
OPTIMAL = 1
PRIMAL_INFEASIBLE = 2
DUAL_INFEASIBLE = 3
MAX_ITER = 4

MAX_OUTER = 4000   # gamma**MAX_OUTER underflows every double: a guard, never reached in practice

STATUS_NAMES = {OPTIMAL: "optimal", PRIMAL_INFEASIBLE: "primal_infeasible",
                DUAL_INFEASIBLE: "dual_infeasible", MAX_ITER: "max_iter"}


@dataclass
class Params:
    beta: float = 1.0            # barrier weight; mu0 = beta (Algorithm 2, first step; reading A3)
    gamma: float = 0.1           # mu decrease ratio (Algorithm 2; reading A2)
    alpha: float = 1.8           # over-relaxation (Sec. 4.2; value from Sec. 5)
    eps: float = 1e-6            # all five tolerances of Sec. 4.1
    max_admm_iters: int = 1_000_000   # Sec. 5 cap
    linsys: int = 0              # 0 dense Cholesky of G, 1 Jacobi-PCG on G
    cg_tol: float = 1e-13        # reading A10: ||r|| <= cg_tol * max(1, ||rhs||)
    cg_max_iter: int = 10000
    cg_warm: int = 2             # PCG start (reading A10): 0 the previous z_y; 1 the linear
                                 # extrapolation 2 z_k - z_{k-1}; 2 the quadratic one
                                 # 3 z_k - 3 z_{k-1} + z_{k-2}
    warmstart: int = 0           # 0 keep-larger heuristic (Sec. 5), 1 sqrt(gamma) (Eq. update-next-iterate)
    stop_rule: int = 0           # 0 Sec. 4.1 tests, 1 stop once mu < eps (outer-count check of Thm 3.6)
    bb_beta: bool = False        # Sec. 4.3: Barzilai-Borwein choice of beta at each outer iteration
    eps_cor: float = 0.2         # Sec. 4.3 curvature-quality threshold (value from Sec. 5)
    eps_penalty: float = 0.1     # Sec. 4.3 heuristic threshold (value from Sec. 5)
    bb_max_redo: int = 5         # reading B5: the paper does not bound the "redo" loop
    gamma_max: float = 0.0       # Sec. 5 adaptive decrease ratio (reading B11): 0 keeps gamma fixed;
                                 # else gamma_for() raises gamma from `gamma` toward gamma_max as the
                                 # relative KKT residual falls from 1e-1 to eps


@dataclass
class Result:
    status: int
    x: np.ndarray
    y: np.ndarray
    s: np.ndarray
    tau: float
    kappa: float
    theta: float
    mu: float
    admm_iters: int
    outer_iters: int
    cg_iters: int
    pres: float                  # relative primal residual ||Ax/tau - b|| / (1 + ||b||)
    dres: float                  # relative dual residual
    dgap: float                  # relative gap
    obj: float                   # c^T x / tau
    raw: dict = field(default_factory=dict)   # unscaled final state (y, x, s, tau, kappa, theta)
    trace: list = field(default_factory=list)


# ---------------------------------------------------------------------------
# Embedding (Sec. 3.1)
# ---------------------------------------------------------------------------

class Problem:
    """Data of the HSD embedding for  min c^T x, A x = b, x >= 0  with x0 = e, s0 = e, y0 = 0."""

    def __init__(self, A, b, c):
        self.sparse = _sp is not None and _sp.issparse(A)
        self.A = A.tocsr().astype(np.float64) if self.sparse else np.asarray(A, dtype=np.float64)
        self.AT = self.A.T.tocsr() if self.sparse else self.A.T
        self.b = np.asarray(b, dtype=np.float64)
        self.c = np.asarray(c, dtype=np.float64)
        self.m, self.n = self.A.shape
        e = np.ones(self.n)
        # Eq. bar-b-c-z-re: bbar = b - A e, cbar = c - e, zbar = c^T e + 1
        self.bbar = self.b - self.Amul(e)
        self.cbar = self.c - 1.0
        self.zbar = float(self.c.sum()) + 1.0
        self.xi = -float(self.n) - 1.0          # xi = -(x0)^T s0 - 1 = -n - 1

    def Amul(self, v):
        return self.A @ v

    def ATmul(self, v):
        return self.AT @ v


def apply_Q(P: Problem, y, x, tau, theta):
    """Q u for u = (y, x, tau, theta) with Q the skew-symmetric matrix of Sec. 3.1.

    Rows (block order y, x, tau, theta):
        [ 0    A    -b    bbar ] [y    ]
        [-A^T  0     c   -cbar ] [x    ]
        [ b^T -c^T   0    zbar ] [tau  ]
        [-bbar^T cbar^T -zbar 0] [theta]
    """
    qy = P.Amul(x) - P.b * tau + P.bbar * theta
    qx = -P.ATmul(y) + P.c * tau - P.cbar * theta
    qt = P.b @ y - P.c @ x + P.zbar * theta
    qth = -(P.bbar @ y) + P.cbar @ x - P.zbar * tau
    return qy, qx, float(qt), float(qth)


def residual_Qu_v(P: Problem, y, x, tau, theta, r, s, kappa, xi):
    """The vector Q u - v (the left side of the inner stop, Eq. inner-stop)."""
    qy, qx, qt, qth = apply_Q(P, y, x, tau, theta)
    return qy - r, qx - s, qt - kappa, qth - xi


def dense_Q(P: Problem) -> np.ndarray:
    """Q as an explicit dense matrix (small problems only), assembled column by column
    from `apply_Q` applied to unit vectors."""
    N = P.m + P.n + 2
    Q = np.zeros((N, N))
    for k in range(N):
        u = np.zeros(N)
        u[k] = 1.0
        qy, qx, qt, qth = apply_Q(P, u[:P.m], u[P.m:P.m + P.n], u[P.m + P.n], u[P.m + P.n + 1])
        Q[:, k] = np.concatenate([qy, qx, [qt, qth]])
    return Q


# ---------------------------------------------------------------------------
# Barrier step (Eqs. Simple-Update:Barrier-X / -tau and Simple-Update:Dual)
# ---------------------------------------------------------------------------

def barrier_prox(omega, cmu):
    """Minimiser of  -cmu*log(x) + 0.5*(x - omega)^2  and the matching dual value.

    The minimiser is the positive root of x^2 - omega*x - cmu = 0, that is
    x = (omega + sqrt(omega^2 + 4 cmu)) / 2 (Eq. Simple-Update:Barrier-X); the dual
    step (Eq. Simple-Update:Dual) then gives s_new = x - omega, the other root's
    magnitude, so x * s_new = cmu.  Each root is evaluated in the form that adds
    quantities of equal sign (reading A9):  for omega >= 0 the large root is
    (omega + D)/2 and the small one 2 cmu / (omega + D); for omega < 0 the roles swap.
    Returns (x_new, s_new).
    """
    omega = np.asarray(omega, dtype=np.float64)
    D = np.sqrt(omega * omega + 4.0 * cmu)
    pos = omega >= 0
    with np.errstate(divide="ignore", invalid="ignore"):
        big_x = 0.5 * (omega + D)
        small_s = 2.0 * cmu / (omega + D)
        small_x = 2.0 * cmu / (D - omega)
        big_s = 0.5 * (D - omega)
    x = np.where(pos, big_x, small_x)
    s = np.where(pos, small_s, big_s)
    return x, s


# ---------------------------------------------------------------------------
# Linear systems with G = I + A A^T (Sec. 4.4)
# ---------------------------------------------------------------------------

class DenseCholesky:
    """G = I + A A^T formed once and factored G = L L^T (Sec. 4.4, dense A)."""

    def __init__(self, P: Problem):
        Ad = P.A.toarray() if P.sparse else P.A
        self.G = np.eye(P.m) + Ad @ Ad.T
        self.L = np.linalg.cholesky(self.G)
        self.iters = 0

    def solve(self, q, z0=None):
        if _sla is not None:
            w = _sla.solve_triangular(self.L, q, lower=True)
            return _sla.solve_triangular(self.L.T, w, lower=False)
        return np.linalg.solve(self.G, q)


class JacobiPCG:
    """Conjugate gradients on G = I + A A^T with the Jacobi preconditioner
    diag(G)_i = 1 + sum_j A_ij^2, warm-started from the previous solution.

    Each iteration multiplies once by A^T and once by A (Sec. 4.4).  The stop rule is
    ||r||_2 <= tol * max(1, ||q||_2) (reading A10); exceeding `max_iter` raises.
    """

    def __init__(self, P: Problem, tol: float, max_iter: int):
        self.P = P
        if P.sparse:
            sq = np.asarray(P.A.multiply(P.A).sum(axis=1)).ravel()
        else:
            sq = (P.A * P.A).sum(axis=1)
        self.dinv = 1.0 / (1.0 + sq)
        self.tol = tol
        self.max_iter = max_iter
        self.iters = 0

    def G(self, p):
        return p + self.P.Amul(self.P.ATmul(p))

    def solve(self, q, z0=None):
        z = np.zeros_like(q) if z0 is None else z0.copy()
        r = q - self.G(z)
        zr = self.dinv * r
        p = zr.copy()
        rz = r @ zr
        bound = self.tol * max(1.0, float(np.linalg.norm(q)))
        k = 0
        while np.linalg.norm(r) > bound:
            if k >= self.max_iter:
                raise RuntimeError("PCG did not converge")
            Gp = self.G(p)
            a = rz / (p @ Gp)
            z += a * p
            r -= a * Gp
            zr = self.dinv * r
            rz_new = r @ zr
            p = zr + (rz_new / rz) * p
            rz = rz_new
            k += 1
        self.iters += k
        return z


def solve_M(P: Problem, lin, a, d, z0=None):
    """Solve M [zy; zx] = [a; d] with M = [[I, A], [-A^T, I]] (Sec. 4.4).

    From the second block row zx = d + A^T zy; substituting in the first gives
    (I + A A^T) zy = a - A d.
    """
    zy = lin.solve(a - P.Amul(d), z0)
    zx = d + P.ATmul(zy)
    return zy, zx


class Projection:
    """The projection of Eq. Simple-Update:Affine, u_tilde = (I + Q)^{-1} w, by block
    elimination (Sec. 4.4 and its Remark on caching M^{-1} h).

    Partition I + Q = [[M, H], [-H^T, I_2 + S]] with H = [h1 h2], h1 = [-b; c],
    h2 = [bbar; -cbar], S = [[0, zbar], [-zbar, 0]] (reading A1: the (tau, theta)
    block of the 4-block Q).  With Gm = M^{-1} H cached and K = I_2 + S + H^T Gm,
        z = M^{-1} w_yx,   t = K^{-1} (w_{tau,theta} + H^T z),   u_yx = z - Gm t,
        (u_tau, u_theta) = t.
    """

    def __init__(self, P: Problem, lin):
        self.P = P
        self.lin = lin
        self.h1y, self.h1x = -P.b, P.c.copy()
        self.h2y, self.h2x = P.bbar.copy(), -P.cbar
        self.g1y, self.g1x = solve_M(P, lin, self.h1y, self.h1x)
        self.g2y, self.g2x = solve_M(P, lin, self.h2y, self.h2x)
        HtG = np.array([[self.h1y @ self.g1y + self.h1x @ self.g1x, self.h1y @ self.g2y + self.h1x @ self.g2x],
                        [self.h2y @ self.g1y + self.h2x @ self.g1x, self.h2y @ self.g2y + self.h2x @ self.g2x]])
        S = np.array([[0.0, P.zbar], [-P.zbar, 0.0]])
        self.K = np.eye(2) + S + HtG
        self.zy_prev = np.zeros(P.m)
        self.zy_prev2 = np.zeros(P.m)
        self.zy_prev3 = np.zeros(P.m)
        self.solves = 0
        self.cg_warm = 0

    def start_point(self):
        """Initial guess of the iterative M-solve (reading A10): the previous z_y; with
        cg_warm = 1 (and two previous solves) the linear extrapolation 2 z_k - z_{k-1};
        with cg_warm = 2 (and three) the quadratic one 3 z_k - 3 z_{k-1} + z_{k-2}."""
        if self.cg_warm == 2 and self.solves >= 3:
            return 3.0 * self.zy_prev - 3.0 * self.zy_prev2 + self.zy_prev3
        if self.cg_warm >= 1 and self.solves >= 2:
            return 2.0 * self.zy_prev - self.zy_prev2
        return self.zy_prev

    def __call__(self, wy, wx, wt, wth):
        zy, zx = solve_M(self.P, self.lin, wy, wx, self.start_point())
        self.zy_prev3 = self.zy_prev2
        self.zy_prev2 = self.zy_prev
        self.zy_prev = zy
        self.solves += 1
        Hz = np.array([self.h1y @ zy + self.h1x @ zx, self.h2y @ zy + self.h2x @ zx])
        t = np.linalg.solve(self.K, np.array([wt, wth]) + Hz)
        uy = zy - self.g1y * t[0] - self.g2y * t[1]
        ux = zx - self.g1x * t[0] - self.g2x * t[1]
        return uy, ux, float(t[0]), float(t[1])


def dense_projection(P: Problem, w: np.ndarray) -> np.ndarray:
    """(I + Q)^{-1} w by a dense solve (small sizes; used only to check `Projection`)."""
    Q = dense_Q(P)
    return np.linalg.solve(np.eye(Q.shape[0]) + Q, w)


# ---------------------------------------------------------------------------
# Termination (Sec. 4.1)
# ---------------------------------------------------------------------------

@dataclass
class Check:
    status: int                   # 0 = continue
    pres: float
    dres: float
    dgap: float
    pres_abs: float
    dres_abs: float
    gap_abs: float
    bty: float
    ctx: float


def termination(P: Problem, y, x, s, tau, eps, nb, nc) -> Check:
    """Sec. 4.1.  Candidate (x/tau, y/tau, s/tau); optimal when
        ||A x/tau - b|| <= eps (1 + ||b||),  ||(A^T y + s)/tau - c|| <= eps (1 + ||c||),
        |c^T x/tau - b^T y/tau| <= eps (1 + |c^T x/tau| + |b^T y/tau|)      (reading A6);
    else primal-infeasible when b^T y > 0 and ||A^T y + s|| <= eps b^T y / ||b||, else
    dual-infeasible when c^T x < 0 and ||A x|| <= eps (-c^T x) / ||c|| (reading A8)."""
    Ax = P.Amul(x)
    ATy_s = P.ATmul(y) + s
    ctx = float(P.c @ x)
    bty = float(P.b @ y)
    pres_abs = float(np.linalg.norm(Ax / tau - P.b))
    dres_abs = float(np.linalg.norm(ATy_s / tau - P.c))
    gap_abs = abs(ctx / tau - bty / tau)
    pres = pres_abs / (1.0 + nb)
    dres = dres_abs / (1.0 + nc)
    dgap = gap_abs / (1.0 + abs(ctx / tau) + abs(bty / tau))
    status = 0
    if pres <= eps and dres <= eps and dgap <= eps:
        status = OPTIMAL
    elif bty > 0 and float(np.linalg.norm(ATy_s)) <= eps * bty / nb:
        status = PRIMAL_INFEASIBLE
    elif ctx < 0 and float(np.linalg.norm(Ax)) <= eps * (-ctx) / nc:
        status = DUAL_INFEASIBLE
    return Check(status, pres, dres, dgap, pres_abs, dres_abs, gap_abs, bty, ctx)


# ---------------------------------------------------------------------------
# Algorithm 2 with over-relaxation
# ---------------------------------------------------------------------------

def make_linsys(P: Problem, prm: Params):
    if prm.linsys == 0:
        return DenseCholesky(P)
    return JacobiPCG(P, prm.cg_tol, prm.cg_max_iter)


def admm_step(P: Problem, proj: Projection, st: dict, mu: float, prm: Params, beta: Optional[float] = None):
    """One inner iteration of Algorithm 2 with over-relaxation (Sec. 4.2):
    projection, relaxation, barrier step for u, dual step for v.  beta: the outer
    iteration's beta (Sec. 4.3), prm.beta when None.  Returns the projection u_tilde
    as (y, x, tau, theta)."""
    y, x, s = st["y"], st["x"], st["s"]
    tau, kappa, theta = st["tau"], st["kappa"], st["theta"]
    r = np.zeros(P.m)
    xi = P.xi
    # Eq. Simple-Update:Affine with w = u + v
    uy, ux, ut, uth = proj(y + r, x + s, tau + kappa, theta + xi)
    a = prm.alpha
    # Sec. 4.2: replace u_tilde by alpha u_tilde + (1 - alpha) u_i
    yh = a * uy + (1 - a) * y
    xh = a * ux + (1 - a) * x
    th = a * ut + (1 - a) * tau
    thh = a * uth + (1 - a) * theta
    cmu = mu / (prm.beta if beta is None else beta)
    # Eqs. Simple-Update:Barrier-Y/X/tau/theta and Simple-Update:Dual
    x_new, s_new = barrier_prox(xh - s, cmu)
    tau_new, kappa_new = barrier_prox(np.array([th - kappa]), cmu)
    st["y"] = yh
    st["x"] = x_new
    st["s"] = s_new
    st["tau"] = float(tau_new[0])
    st["kappa"] = float(kappa_new[0])
    st["theta"] = thh
    return uy, ux, float(ut), float(uth)


# ---------------------------------------------------------------------------
# Barzilai-Borwein choice of beta (Sec. 4.3)
# ---------------------------------------------------------------------------

def _u_vec(st: dict) -> np.ndarray:
    return np.concatenate([st["y"], st["x"], [st["tau"], st["theta"]]])


def _v_vec(P: Problem, st: dict) -> np.ndarray:
    """v = (r, s, kappa, xi) with r = 0 and xi = -n-1 (Algorithm 2)."""
    return np.concatenate([np.zeros(P.m), st["s"], [st["kappa"], P.xi]])


def _hybrid(sd: float, mg: float) -> float:
    """The hybrid spectral step: the minimum-gradient step when 2 MG > SD, else SD - MG/2."""
    return mg if 2.0 * mg > sd else sd - mg / 2.0


def bb_estimate(dv_hat: np.ndarray, du_tilde: np.ndarray, du: np.ndarray, beta: float, eps_cor: float) -> float:
    """beta_hat of Sec. 4.3 from the curvature pairs (dv_hat, du_tilde) and (dv_hat, du):
    steepest-descent and minimum-gradient spectral steps, their hybrid, the correlation
    safeguards, and the geometric mean when both estimates are reliable."""
    vv = float(dv_hat @ dv_hat)
    nv = np.sqrt(vv)

    def pair(d):
        vd, dd = float(dv_hat @ d), float(d @ d)
        if vd == 0.0 or dd == 0.0 or nv == 0.0:
            return 0.0, -1.0
        return _hybrid(vv / vd, vd / dd), vd / (nv * np.sqrt(dd))

    phi, phi_cor = pair(du_tilde)
    psi, psi_cor = pair(du)
    if phi_cor > eps_cor and psi_cor > eps_cor:
        return float(np.sqrt(phi * psi))
    if phi_cor > eps_cor:
        return float(phi)
    if psi_cor > eps_cor:
        return float(psi)
    return float(beta)


def bb_select(P: Problem, proj: Projection, st0: dict, mu: float, beta: float, prm: Params,
              budget: Optional[int] = None):
    """Sec. 4.3 at the start of an outer iteration: two ADMM updates from st0 with beta give
    the curvature pairs; then the heuristic selection (reading B5).  A redo starts again
    from st0 with the new beta; rounds stop after prm.bb_max_redo redos, or before a round
    would take the updates spent past `budget`.  Returns (beta for this outer iteration,
    state to continue from, ADMM updates spent); when the rounds stop without a selection
    the beta returned is the one that produced the returned state."""
    a = prm.alpha
    spent = 0
    st = st0
    used = beta
    for _ in range(prm.bb_max_redo + 1):
        if budget is not None and spent + 2 > budget:
            break
        st = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in st0.items()}
        u0, v0 = _u_vec(st), _v_vec(P, st)
        ut1 = np.concatenate(list(map(np.atleast_1d, admm_step(P, proj, st, mu, prm, beta))))
        u1, v1 = _u_vec(st), _v_vec(P, st)
        ut2 = np.concatenate(list(map(np.atleast_1d, admm_step(P, proj, st, mu, prm, beta))))
        u2 = _u_vec(st)
        spent += 2
        used = beta
        vh1 = v0 - a * ut1 - (1 - a) * u0 + a * u1
        vh2 = v1 - a * ut2 - (1 - a) * u1 + a * u2
        beta_hat = bb_estimate(vh2 - vh1, a * (ut2 - ut1) + (1 - a) * (u1 - u0), -(u2 - u1), beta, prm.eps_cor)
        if beta_hat == beta:                       # no reliable curvature: keep beta, go on
            return beta, st, spent
        if abs(beta_hat - beta) <= prm.eps_penalty:
            return 0.5 * (beta + beta_hat), st, spent
        beta = beta_hat                            # redo from the same initial point
    return used, st, spent


GAMMA_FAR = 1e-1   # reading B11: residual at and above which the decrease ratio is prm.gamma


def gamma_for(prm: Params, rho: float) -> float:
    """The decrease ratio of the next mu <- gamma mu.  Sec. 5 increases gamma as the iterate
    approaches the optimal solution without a formula (reading B11): with gamma_max > 0,
    gamma moves from prm.gamma to gamma_max linearly in log10 of the relative KKT residual
    rho = max(pres, dres, dgap) of the current iterate, from rho >= 1e-1 to rho <= eps."""
    if prm.gamma_max <= 0.0:
        return prm.gamma
    rho = rho if rho > 1e-300 else 1e-300      # also a NaN residual: the largest ratio
    t = np.log10(GAMMA_FAR / rho) / np.log10(GAMMA_FAR / prm.eps)
    t = min(1.0, max(0.0, float(t)))
    return prm.gamma + (prm.gamma_max - prm.gamma) * t


def warm_start(st: dict, gamma: float, rule: int):
    """Rescale after mu <- gamma mu.  rule 0 (Sec. 5): for each j keep the larger of
    x_j, s_j and multiply the other by gamma (ties keep x), the same for (tau, kappa),
    and y, theta by sqrt(gamma) (reading A4).  rule 1: Eq. update-next-iterate, every
    component by sqrt(gamma)."""
    if rule == 1:
        g = np.sqrt(gamma)
        for k in ("y", "x", "s"):
            st[k] = g * st[k]
        for k in ("tau", "kappa", "theta"):
            st[k] = g * st[k]
        return
    x, s = st["x"], st["s"]
    keep_x = x >= s
    st["x"] = np.where(keep_x, x, gamma * x)
    st["s"] = np.where(keep_x, gamma * s, s)
    if st["tau"] >= st["kappa"]:
        st["kappa"] = gamma * st["kappa"]
    else:
        st["tau"] = gamma * st["tau"]
    g = np.sqrt(gamma)
    st["y"] = g * st["y"]
    st["theta"] = g * st["theta"]


def inner_residual_sq(P: Problem, st: dict) -> float:
    """||Q u - v||^2 of Eq. inner-stop, with r = 0 and xi = -n - 1."""
    ry, rx, rt, rth = residual_Qu_v(P, st["y"], st["x"], st["tau"], st["theta"],
                                    np.zeros(P.m), st["s"], st["kappa"], P.xi)
    return float(ry @ ry + rx @ rx + rt * rt + rth * rth)


def initial_state(P: Problem) -> dict:
    """Algorithm 2 start: r = y = 0, x = s = e, tau = kappa = theta = 1 (xi = -n-1)."""
    return dict(y=np.zeros(P.m), x=np.ones(P.n), s=np.ones(P.n), tau=1.0, kappa=1.0, theta=1.0)


def stacked(st: dict) -> np.ndarray:
    """(y, x, tau, theta, s, kappa) as one vector (the iterate compared in parity tests)."""
    return np.concatenate([st["y"], st["x"], [st["tau"], st["theta"]], st["s"], [st["kappa"]]])


def solve(A, b, c, prm: Optional[Params] = None, trace_iters: int = 0,
          on_iter: Optional[Callable] = None) -> Result:
    """ABIP, Algorithm 2 with Sec. 4 details, in FP64.

    trace_iters: record `stacked(state)` after each of the first `trace_iters` ADMM
    updates.  on_iter(k, mu, state): optional callback after every update.
    """
    prm = prm or Params()
    if prm.gamma_max != 0.0 and not (prm.gamma <= prm.gamma_max < 1.0):
        raise ValueError("gamma_max must be 0 (off) or in [gamma, 1)")
    P = Problem(A, b, c)
    lin = make_linsys(P, prm)
    proj = Projection(P, lin)
    proj.cg_warm = prm.cg_warm
    nb = float(np.linalg.norm(P.b))
    nc = float(np.linalg.norm(P.c))
    st = initial_state(P)
    mu = prm.beta                      # mu0 = beta
    beta_k = prm.beta
    betas = []
    gammas = []                        # the ratio of every mu <- gamma mu (reading B11)
    total = 0
    outer = 0
    trace = []
    chk = None
    status = 0
    while status == 0:
        # reading B7: from the second outer iteration on (the first starts at the exact
        # central point of mu0 = beta, where the ADMM map does not move and the curvature
        # pairs would be rounding noise)
        if prm.bb_beta and outer >= 1 and total + 2 <= prm.max_admm_iters:
            beta_k, st, spent = bb_select(P, proj, st, mu, beta_k, prm, budget=prm.max_admm_iters - total)
            total += spent
            betas.append(beta_k)
            if total >= prm.max_admm_iters:      # the trial updates used the last of the cap
                status = MAX_ITER
                break
        # inner loop at fixed mu (Algorithm 2)
        while True:
            if inner_residual_sq(P, st) <= mu:
                break
            admm_step(P, proj, st, mu, prm, beta_k)
            total += 1
            if total <= trace_iters:
                trace.append(stacked(st))
            if on_iter is not None:
                on_iter(total, mu, st)
            if prm.stop_rule == 0:
                chk = termination(P, st["y"], st["x"], st["s"], st["tau"], prm.eps, nb, nc)
                if chk.status != 0:
                    status = chk.status
                    break
            if total >= prm.max_admm_iters:
                status = MAX_ITER
                break
        if status != 0:
            break
        g = prm.gamma
        if prm.gamma_max > 0.0:     # reading B11: from the residuals of the current state
            cur = termination(P, st["y"], st["x"], st["s"], st["tau"], prm.eps, nb, nc)
            g = gamma_for(prm, max(cur.pres, cur.dres, cur.dgap))
        gammas.append(g)
        mu *= g
        outer += 1
        if prm.stop_rule == 1 and mu < prm.eps:
            status = OPTIMAL
            break
        if outer >= MAX_OUTER:          # mu has underflowed; stop as unsolved
            status = MAX_ITER
            break
        warm_start(st, g, prm.warmstart)
    if chk is None:
        chk = termination(P, st["y"], st["x"], st["s"], st["tau"], prm.eps, nb, nc)
    tau = st["tau"]
    x, y, s = st["x"], st["y"], st["s"]
    if status == PRIMAL_INFEASIBLE:
        xo, yo, so = x.copy(), y / chk.bty, s / chk.bty           # Sec. 4.1 certificate y / b^T y
    elif status == DUAL_INFEASIBLE:
        xo, yo, so = -x / chk.ctx, y.copy(), s.copy()             # certificate -x / c^T x
    else:
        xo, yo, so = x / tau, y / tau, s / tau
    return Result(status=status, x=xo, y=yo, s=so, tau=tau, kappa=st["kappa"], theta=st["theta"],
                  mu=mu, admm_iters=total, outer_iters=outer, cg_iters=getattr(lin, "iters", 0),
                  pres=chk.pres, dres=chk.dres, dgap=chk.dgap, obj=chk.ctx / tau,
                  raw=dict(y=y.copy(), x=x.copy(), s=s.copy(), tau=tau, kappa=st["kappa"], theta=st["theta"],
                           betas=betas, gammas=gammas),
                  trace=trace)


def run_iterations(A, b, c, k: int, prm: Optional[Params] = None) -> np.ndarray:
    """The stacked state after exactly k ADMM updates of Algorithm 2 (no final test)."""
    prm = prm or Params()
    P = Problem(A, b, c)
    proj = Projection(P, make_linsys(P, prm))
    proj.cg_warm = prm.cg_warm
    st = initial_state(P)
    mu = prm.beta
    done = 0
    while done < k:
        if inner_residual_sq(P, st) <= mu:
            mu *= prm.gamma
            warm_start(st, prm.gamma, prm.warmstart)
            continue
        admm_step(P, proj, st, mu, prm)
        done += 1
    return stacked(st)


# ---------------------------------------------------------------------------
# Algorithm 1 with explicit multipliers (debug mode for Theorem 3.1)
# ---------------------------------------------------------------------------

def algorithm1(A, b, c, mu: float, iters: int, beta: float = 1.0, alpha: float = 1.0,
               start: Optional[dict] = None):
    """Algorithm 1 (Eqs. admm-typical-1..3) at one fixed mu with explicit scaled
    multipliers p (for u~ = u) and q (for v~ = v), initialised as Theorem 3.1 asks:
    p0 = v0, q0 = u0.  The projection onto {Q u = v} of a point (a, g) is computed
    generically as u = (I + Q^T Q)^{-1} (a + Q^T g), v = Q u (dense, small sizes).
    With alpha != 1 the projected pair is relaxed, (u~, v~) <- alpha (u~, v~) +
    (1 - alpha)(u, v) (Sec. 4.2), before the barrier and multiplier steps.
    Returns the list of (u, v, p, q) after each iteration (vectors in block order).
    """
    P = Problem(A, b, c)
    m, n = P.m, P.n
    Q = dense_Q(P)
    N = m + n + 2
    IQQ = np.eye(N) + Q.T @ Q
    st = initial_state(P) if start is None else start
    u = np.concatenate([st["y"], st["x"], [st["tau"], st["theta"]]])
    v = np.concatenate([np.zeros(m), st["s"], [st["kappa"], P.xi]])
    p = v.copy()
    q = u.copy()
    cmu = mu / beta
    sl_y, sl_x, i_t, i_th = slice(0, m), slice(m, m + n), m + n, m + n + 1
    out = []
    for _ in range(iters):
        a_pt, g_pt = u + p, v + q
        ut = np.linalg.solve(IQQ, a_pt + Q.T @ g_pt)
        vt = Q @ ut
        ut = alpha * ut + (1 - alpha) * u
        vt = alpha * vt + (1 - alpha) * v
        # barrier step (Eq. admm-typical-2), separable per coordinate:
        #   argmin B(u, v, mu) + beta/2 ||(u, v) - (ut - p, vt - q)||^2
        au, av = ut - p, vt - q
        un = np.empty(N)
        vn = np.empty(N)
        un[sl_y] = au[sl_y]                                   # y free
        un[sl_x] = barrier_prox(au[sl_x], cmu)[0]             # -mu log x
        un[i_t] = barrier_prox(np.array([au[i_t]]), cmu)[0][0]
        un[i_th] = au[i_th] - (n + 1)                         # beta (n+1) theta + beta/2 (theta - a)^2
        vn[sl_y] = 0.0                                        # indicator r = 0
        vn[sl_x] = barrier_prox(av[sl_x], cmu)[0]             # -mu log s
        vn[i_t] = barrier_prox(np.array([av[i_t]]), cmu)[0][0]
        vn[i_th] = -(n + 1.0)                                 # indicator xi = -n-1
        # multiplier step (Eq. admm-typical-3)
        p = p - ut + un
        q = q - vt + vn
        u, v = un, vn
        out.append((u.copy(), v.copy(), p.copy(), q.copy()))
    return out


# ---------------------------------------------------------------------------
# Central path point (Remark after Algorithm 2, system HSD-log-kkt)
# ---------------------------------------------------------------------------

def central_point(A, b, c, mu: float, beta: float = 1.0, start: Optional[dict] = None,
                  tol: float = 1e-13, max_iter: int = 100) -> dict:
    """The unique solution of system HSD-log-kkt at mu by damped Newton's method.

    Unknowns (y, x, tau, theta, s, kappa); equations Q u - v = 0 with r = 0 and
    xi = -n-1, x o s = mu/beta e, tau kappa = mu/beta.  (theta = mu/beta then follows.)
    Dense Jacobian: small and medium sizes only.
    """
    P = Problem(A, b, c)
    m, n = P.m, P.n
    Ad = P.A.toarray() if P.sparse else P.A
    cmu = mu / beta
    st = initial_state(P) if start is None else {k: (np.array(v, dtype=float) if np.ndim(v) else float(v))
                                                    for k, v in start.items()}
    z = np.concatenate([st["y"], st["x"], [st["tau"], st["theta"]], st["s"], [st["kappa"]]])
    iy, ix = slice(0, m), slice(m, m + n)
    it, ith = m + n, m + n + 1
    isl = slice(m + n + 2, m + 2 * n + 2)
    ik = m + 2 * n + 2
    N = m + 2 * n + 3

    def F(z):
        y, x, tau, theta, s, kap = z[iy], z[ix], z[it], z[ith], z[isl], z[ik]
        ry, rx, rt, rth = residual_Qu_v(P, y, x, tau, theta, np.zeros(m), s, kap, P.xi)
        return np.concatenate([ry, rx, [rt, rth], x * s - cmu, [tau * kap - cmu]])

    J = np.zeros((N, N))
    Q = dense_Q(P)
    J[:m + n + 2, :m + n + 2] = Q
    J[m:m + n, isl] = -np.eye(n)          # -s in the x rows
    J[m + n, ik] = -1.0                   # -kappa in the tau row
    for k in range(max_iter):
        fz = F(z)
        if np.linalg.norm(fz) <= tol * max(1.0, np.linalg.norm(z)):
            break
        Jk = J.copy()
        Jk[m + n + 2:m + 2 * n + 2, ix] = np.diag(z[isl])
        Jk[m + n + 2:m + 2 * n + 2, isl] = np.diag(z[ix])
        Jk[N - 1, it] = z[ik]
        Jk[N - 1, ik] = z[it]
        dz = np.linalg.solve(Jk, -fz)
        step = 1.0
        pos = np.concatenate([np.arange(m, m + n + 1), np.arange(m + n + 2, N)])
        neg = dz[pos] < 0
        if neg.any():
            step = min(1.0, 0.99 * float(np.min(-z[pos][neg] / dz[pos][neg])))
        z = z + step * dz
    return dict(y=z[iy].copy(), x=z[ix].copy(), tau=float(z[it]), theta=float(z[ith]),
                s=z[isl].copy(), kappa=float(z[ik]), residual=float(np.linalg.norm(F(z))))


# ---------------------------------------------------------------------------
# Differentiation of the central point (system HSD-log-kkt) with respect to (A, b, c)
# ---------------------------------------------------------------------------

def kkt_residual(P: Problem, z: np.ndarray, cmu: float) -> np.ndarray:
    """F(z) of system HSD-log-kkt for z = (y, x, tau, theta, s, kappa): Q u - v with r = 0
    and xi = -n-1, then x o s - cmu e and tau kappa - cmu."""
    m, n = P.m, P.n
    y, x = z[:m], z[m:m + n]
    tau, theta = z[m + n], z[m + n + 1]
    s, kap = z[m + n + 2:m + 2 * n + 2], z[m + 2 * n + 2]
    ry, rx, rt, rth = residual_Qu_v(P, y, x, tau, theta, np.zeros(m), s, kap, P.xi)
    return np.concatenate([ry, rx, [rt, rth], x * s - cmu, [tau * kap - cmu]])


def kkt_jacobian(P: Problem, z: np.ndarray) -> np.ndarray:
    """dF/dz of `kkt_residual` (dense): Q in the (y, x, tau, theta) columns, -I for s in
    the x rows, -1 for kappa in the tau row, diag(s), diag(x) and (kappa, tau) below."""
    m, n = P.m, P.n
    N = m + 2 * n + 3
    J = np.zeros((N, N))
    J[:m + n + 2, :m + n + 2] = dense_Q(P)
    J[m:m + n, m + n + 2:m + 2 * n + 2] = -np.eye(n)
    J[m + n, N - 1] = -1.0
    x, s = z[m:m + n], z[m + n + 2:m + 2 * n + 2]
    J[m + n + 2:m + 2 * n + 2, m:m + n] = np.diag(s)
    J[m + n + 2:m + 2 * n + 2, m + n + 2:m + 2 * n + 2] = np.diag(x)
    J[N - 1, m + n] = z[N - 1]
    J[N - 1, N - 1] = z[m + n]
    return J


def central_point_grad(A, b, c, mu: float, dl_dxstar: Callable, beta: float = 1.0,
                       start: Optional[dict] = None) -> dict:
    """Gradient of L(x*) with x* = x / tau at the central point of system HSD-log-kkt
    (the barrier-smoothed solution at mu) with respect to A, b and c, by implicit
    differentiation: solve J^T lam = dL/dz at the central point, then
    dL/dp = -lam^T dF/dp.  F is affine in (A, b, c) for fixed z, including through
    bbar = b - A e, cbar = c - e, zbar = c^T e + 1 (Eq. bar-b-c-z-re), which gives
      dL/dA_ij = -(lam1_i (x_j - theta) - lam2_j y_i + lam4 y_i)
      dL/db_i  = -(lam1_i (theta - tau) + (lam3 - lam4) y_i)
      dL/dc_j  = -(lam2_j (tau - theta) + lam3 (theta - x_j) + lam4 (x_j - tau))
    with lam = (lam1 (m), lam2 (n), lam3, lam4, lam5 (n), lam6) in the order of F's rows.
    dl_dxstar(xstar) returns dL/dx*.  Dense: small and medium sizes."""
    P = Problem(A, b, c)
    m, n = P.m, P.n
    cp = central_point(A, b, c, mu, beta, start=start)
    z = np.concatenate([cp["y"], cp["x"], [cp["tau"], cp["theta"]], cp["s"], [cp["kappa"]]])
    y, x, tau, theta = cp["y"], cp["x"], cp["tau"], cp["theta"]
    xstar = x / tau
    g = np.asarray(dl_dxstar(xstar), dtype=np.float64)
    dz = np.zeros_like(z)
    dz[m:m + n] = g / tau
    dz[m + n] = -(g @ x) / tau ** 2
    lam = np.linalg.solve(kkt_jacobian(P, z).T, dz)
    l1, l2, l3, l4 = lam[:m], lam[m:m + n], lam[m + n], lam[m + n + 1]
    dA = -(np.outer(l1, x - theta) - np.outer(y, l2) + l4 * np.outer(y, np.ones(n)))
    db = -(l1 * (theta - tau) + (l3 - l4) * y)
    dc = -(l2 * (tau - theta) + l3 * (theta - x) + l4 * (x - tau))
    return dict(xstar=xstar, dA=dA, db=db, dc=dc, lam=lam, point=cp, residual=cp["residual"])
