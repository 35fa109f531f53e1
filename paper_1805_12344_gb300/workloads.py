"""Seeded synthetic LP generators shared by the oracle tests, the CUDA tests and the benchmark.

This module builds problem data only: it contains none of ABIP's arithmetic.
Every generator draws from ``numpy.random.Generator(PCG64(seed))`` and returns
host arrays in float64 (sparse values are drawn in float32 and upcast exactly).

The planted recipe (a primal-dual optimal pair chosen first, then b = A x0 and
c = A^T y0 + s0) makes the LP optimum known exactly:  p* = c^T x0 = b^T y0,
because x0 >= 0, s0 >= 0 and x0 o s0 = 0 (weak duality is tight; Sec. 2, the
primal-dual pair (P)/(D)).

Seeds follow ``SEED_BASE + 1000 * workload_id + instance``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

SEED_BASE = 1805012344

# workload ids used for the seed formula
DENSE_PLANTED = 0     # dense 50 x 120 planted LP and its 10 x 20 infeasible twin
SPARSE_PLANTED = 1    # [R I] CSR LP, 8 nonzeros per column of R
BASIS_PURSUIT = 2
BATCH_UNEVEN = 3
L1_SVM = 4
GRID_FLOW = 8         # planted min-cost flow LPs on a 2-D grid (the sparse direct projection's workload)
TINY = 9              # tiny random LPs for brute-force basis enumeration


def seed_for(workload: int, instance: int = 0) -> int:
    return SEED_BASE + 1000 * workload + instance


@dataclass
class CSR:
    """Compressed sparse row matrix: int64 row pointers, int32 column indices."""
    m: int
    n: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_dense(self) -> np.ndarray:
        out = np.zeros((self.m, self.n), dtype=np.float64)
        rows = np.repeat(np.arange(self.m), np.diff(self.row_ptr))
        out[rows, self.col_idx] = self.val
        return out

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val.astype(np.float64), self.col_idx, self.row_ptr),
                             shape=(self.m, self.n))


@dataclass
class LP:
    """Standard-form LP  min c^T x  s.t.  A x = b,  x >= 0  (A dense float64 or CSR)."""
    A: object
    b: np.ndarray
    c: np.ndarray
    x0: Optional[np.ndarray] = None      # planted primal optimum (if any)
    y0: Optional[np.ndarray] = None      # planted dual optimum (if any)
    s0: Optional[np.ndarray] = None
    expect: str = "optimal"              # "optimal" | "primal_infeasible" | "dual_infeasible" | "unknown"
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return self.A.m if isinstance(self.A, CSR) else self.A.shape[0]

    @property
    def n(self) -> int:
        return self.A.n if isinstance(self.A, CSR) else self.A.shape[1]

    @property
    def p_star(self) -> Optional[float]:
        if self.x0 is None:
            return None
        return float(self.c @ self.x0)

    def dense_A(self) -> np.ndarray:
        return self.A.to_dense() if isinstance(self.A, CSR) else self.A


def _planted_pair(rng: np.random.Generator, n: int, m: int, support_frac: float = 0.3):
    """x0: `support_frac` of entries U[0.5,2], rest 0; s0: U[0.5,2] off x0's support; y0 ~ N(0,1)."""
    k = int(round(support_frac * n))
    perm = rng.permutation(n)
    x0 = np.zeros(n)
    s0 = np.zeros(n)
    x0[perm[:k]] = rng.uniform(0.5, 2.0, k)
    s0[perm[k:]] = rng.uniform(0.5, 2.0, n - k)
    y0 = rng.standard_normal(m)
    return x0, y0, s0


def planted_dense(m: int = 50, n: int = 120, seed: Optional[int] = None) -> LP:
    """Dense planted LP: A iid N(0,1) float64; b = A x0, c = A^T y0 + s0."""
    rng = np.random.default_rng(seed_for(DENSE_PLANTED) if seed is None else seed)
    A = rng.standard_normal((m, n))
    x0, y0, s0 = _planted_pair(rng, n, m)
    return LP(A=A, b=A @ x0, c=A.T @ y0 + s0, x0=x0, y0=y0, s0=s0, expect="optimal",
              meta=dict(kind="planted_dense", m=m, n=n))


def infeasible_twin(m: int = 10, n: int = 20, seed: Optional[int] = None) -> LP:
    """Planted dense LP whose row 1 is replaced by |N(0,1)| with b_1 = -1.

    A_1 x = -1 has no solution with x >= 0; y = -e_1 is a Farkas certificate
    (A^T y <= 0 and b^T y = 1 > 0).
    """
    rng = np.random.default_rng(seed_for(DENSE_PLANTED, 1) if seed is None else seed)
    A = rng.standard_normal((m, n))
    x0, y0, s0 = _planted_pair(rng, n, m)
    b = A @ x0
    c = A.T @ y0 + s0
    A[0, :] = np.abs(rng.standard_normal(n))
    b[0] = -1.0
    return LP(A=A, b=b, c=c, expect="primal_infeasible", meta=dict(kind="infeasible_twin", m=m, n=n))


def dual_infeasible(m: int = 10, n: int = 20, seed: Optional[int] = None) -> LP:
    """Planted dense LP plus one extra all-zero column with cost -1 (unbounded primal).

    x = x0 + t e_new stays feasible for all t >= 0 while the objective falls without bound;
    e_new is a dual-infeasibility certificate (A e_new = 0, c^T e_new = -1 < 0).
    """
    rng = np.random.default_rng(seed_for(DENSE_PLANTED, 2) if seed is None else seed)
    A = rng.standard_normal((m, n))
    x0, y0, s0 = _planted_pair(rng, n, m)
    b = A @ x0
    c = A.T @ y0 + s0
    A = np.hstack([A, np.zeros((m, 1))])
    c = np.concatenate([c, [-1.0]])
    return LP(A=A, b=b, c=c, expect="dual_infeasible", meta=dict(kind="dual_infeasible", m=m, n=n + 1))


def planted_sparse(m: int = 100000, n_r: Optional[int] = None, per_col: int = 8,
                   seed: Optional[int] = None) -> LP:
    """Sparse planted LP  A = [R  I_m]  in CSR.

    R is m x n_r (default n_r = 3m) with `per_col` nonzeros per column at distinct
    uniform random rows, values N(0,1) drawn in float32; the identity block is the
    slack block, so n = n_r + m.  The planted pair spans all n columns.
    """
    if n_r is None:
        n_r = 3 * m
    rng = np.random.default_rng(seed_for(SPARSE_PLANTED) if seed is None else seed)
    per_col = min(per_col, m)
    # distinct rows per column: draw uniformly, redraw any column that repeats a row
    if per_col == m:
        rows = np.tile(np.arange(m), n_r).reshape(n_r, m)
    else:
        rows = rng.integers(0, m, size=(n_r, per_col))
        while True:
            srt = np.sort(rows, axis=1)
            bad = np.nonzero((srt[:, 1:] == srt[:, :-1]).any(axis=1))[0]
            if bad.size == 0:
                break
            rows[bad] = rng.integers(0, m, size=(bad.size, per_col))
    vals = rng.standard_normal((n_r, per_col), dtype=np.float32)
    n = n_r + m
    # assemble CSR of [R I]: entries (row, col, val)
    r_all = np.concatenate([rows.ravel(), np.arange(m)])
    c_all = np.concatenate([np.repeat(np.arange(n_r), per_col), n_r + np.arange(m)])
    v_all = np.concatenate([vals.ravel(), np.ones(m, np.float32)])
    order = np.lexsort((c_all, r_all))
    r_all, c_all, v_all = r_all[order], c_all[order], v_all[order]
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(r_all, minlength=m), out=row_ptr[1:])
    A = CSR(m=m, n=n, row_ptr=row_ptr, col_idx=c_all.astype(np.int32), val=v_all.astype(np.float32))
    x0, y0, s0 = _planted_pair(rng, n, m)
    Asp = A.to_scipy()
    b = Asp @ x0
    c = Asp.T @ y0 + s0
    return LP(A=A, b=b, c=c, x0=x0, y0=y0, s0=s0, expect="optimal",
              meta=dict(kind="planted_sparse", m=m, n=n, nnz=A.nnz, per_col=per_col))


def grid_flow(side: int = 48, seed: Optional[int] = None) -> LP:
    """Planted min-cost flow LP on a side x side grid with 4-neighbour links, CSR.

    One column per directed arc (both directions of every grid link, n = 4 side (side - 1)),
    one row per node except the last (m = side^2 - 1): A_{v,a} = +1 if arc a leaves node v,
    -1 if it enters it.  The node-arc incidence matrix of a connected graph has rank
    nodes - 1, so dropping one node's row leaves A with full row rank (the standing
    assumption of Sec. 2).  I + A A^T is I plus twice the grid's graph Laplacian with that
    row and column removed: its condition number grows like side^2, so Jacobi-PCG needs
    many iterations per projection, while the factor of the quasi-definite system stays
    sparse under a minimum-degree order.  The planted pair follows _planted_pair (b = A x0,
    c = A^T y0 + s0), so the optimum is known."""
    rng = np.random.default_rng(seed_for(GRID_FLOW) if seed is None else seed)
    nodes = side * side
    links = [(r * side + q, r * side + q + 1) for r in range(side) for q in range(side - 1)]
    links += [(r * side + q, (r + 1) * side + q) for r in range(side - 1) for q in range(side)]
    tails, heads = [], []
    for u, v in links:
        tails += [u, v]
        heads += [v, u]
    tails = np.asarray(tails)
    heads = np.asarray(heads)
    n = tails.size
    keep = nodes - 1                       # rows 0 .. nodes-2; the last node's row is dropped
    rows = np.concatenate([tails, heads])
    cols = np.concatenate([np.arange(n), np.arange(n)])
    vals = np.concatenate([np.ones(n, np.float32), -np.ones(n, np.float32)])
    sel = rows < keep
    rows, cols, vals = rows[sel], cols[sel], vals[sel]
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    row_ptr = np.zeros(keep + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=keep), out=row_ptr[1:])
    A = CSR(m=keep, n=n, row_ptr=row_ptr, col_idx=cols.astype(np.int32), val=vals.astype(np.float32))
    x0, y0, s0 = _planted_pair(rng, n, keep)
    Asp = A.to_scipy()
    return LP(A=A, b=Asp @ x0, c=Asp.T @ y0 + s0, x0=x0, y0=y0, s0=s0, expect="optimal",
              meta=dict(kind="grid_flow", side=side, m=keep, n=n, nnz=A.nnz))


RANDOM_UDV = 5        # the random dense LPs of the paper's experiments (Sec. 5.1)


def _sprandn(rng: np.random.Generator, rows: int, cols: int, density: float) -> np.ndarray:
    """Dense array holding a sparse random matrix: round(density * rows * cols) positions
    chosen uniformly without repetition, values N(0, 1), zeros elsewhere."""
    M = np.zeros(rows * cols)
    k = int(round(density * rows * cols))
    M[rng.choice(rows * cols, k, replace=False)] = rng.standard_normal(k)
    return M.reshape(rows, cols)


def random_udv(m: int = 500, n: int = 5000, seed: Optional[int] = None) -> LP:
    """The random dense LP of Sec. 5.1 (Tables 1 and 2): A = U^T D V with D = diag(N(0,1)^m),
    U (m x m) and V (m x n) sparse random with density 0.2 and N(0,1) values.  The planted
    x has 60 % of its entries 0, 10 % |N(0,1)| * 10 and the other 30 % |N(0,1)| / 10; s is
    |N(0,1)| on x's zero set and 0 elsewhere (x o s = 0); y ~ N(0,1); b = A x, c = A^T y + s.
    The paper calls x and s Gaussian; their magnitudes are used here so that x, s >= 0
    (the LP is in standard form).  The optimal value is c^T x = b^T y."""
    rng = np.random.default_rng(seed_for(RANDOM_UDV) if seed is None else seed)
    U = _sprandn(rng, m, m, 0.2)
    D = rng.standard_normal(m)
    V = _sprandn(rng, m, n, 0.2)
    A = U.T @ (D[:, None] * V)
    perm = rng.permutation(n)
    n0, n1 = int(round(0.6 * n)), int(round(0.1 * n))
    x0 = np.abs(rng.standard_normal(n))
    x0[perm[:n0]] = 0.0
    x0[perm[n0:n0 + n1]] *= 10.0
    x0[perm[n0 + n1:]] /= 10.0
    s0 = np.zeros(n)
    s0[perm[:n0]] = np.abs(rng.standard_normal(n0))
    y0 = rng.standard_normal(m)
    return LP(A=A, b=A @ x0, c=A.T @ y0 + s0, x0=x0, y0=y0, s0=s0, expect="optimal",
              meta=dict(kind="random_udv", m=m, n=n))


def tiny_random(m: int, n: int, seed: int) -> LP:
    """Tiny unplanted LP with random signs: may be optimal, infeasible or unbounded."""
    rng = np.random.default_rng(seed)
    A = np.round(rng.standard_normal((m, n)) * 4.0) / 4.0
    b = np.round(rng.standard_normal(m) * 4.0) / 4.0
    c = np.round(rng.standard_normal(n) * 4.0) / 4.0
    return LP(A=A, b=b, c=c, expect="unknown", meta=dict(kind="tiny_random", m=m, n=n))


def tiny_planted(m: int, n: int, seed: int) -> LP:
    """Tiny planted LP (same recipe as `planted_dense`) for brute-force checks."""
    lp = planted_dense(m, n, seed=seed)
    lp.meta["kind"] = "tiny_planted"
    return lp


def csr_transpose(A: CSR) -> CSR:
    """CSR of A^T (the column-major view of A), values and pattern unchanged."""
    counts = np.bincount(A.col_idx, minlength=A.n)
    row_ptr = np.zeros(A.n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    rows = np.repeat(np.arange(A.m, dtype=np.int64), np.diff(A.row_ptr))
    order = np.lexsort((rows, A.col_idx))
    return CSR(m=A.n, n=A.m, row_ptr=row_ptr, col_idx=rows[order].astype(np.int32), val=A.val[order])


def dense_to_csr(A: np.ndarray, dtype=np.float64) -> CSR:
    m, n = A.shape
    mask = A != 0
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(mask.sum(axis=1), out=row_ptr[1:])
    rows, cols = np.nonzero(mask)
    return CSR(m=m, n=n, row_ptr=row_ptr, col_idx=cols.astype(np.int32), val=A[rows, cols].astype(dtype))


def planted_dense_f32(m: int, n: int, seed: int) -> LP:
    """Dense planted LP whose A is iid N(0,1) drawn in float32 (exactly representable in
    both precisions); b and c are formed in float64 from the exact values."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n), dtype=np.float32).astype(np.float64)
    x0, y0, s0 = _planted_pair(rng, n, m)
    return LP(A=A, b=A @ x0, c=A.T @ y0 + s0, x0=x0, y0=y0, s0=s0, expect="optimal",
              meta=dict(kind="planted_dense_f32", m=m, n=n))


def batch_uneven(count: int = 4096, infeasible_frac: float = 0.1, m_lo: int = 16, m_hi: int = 256,
                 seed: int | None = None) -> list:
    """Batch of independent dense planted LPs of uneven size: m ~ U{m_lo..m_hi},
    n = round(m * U[2, 4]); a seeded choice of round(infeasible_frac * count) instances
    gets the infeasible-twin treatment (row 1 of A <- |N(0,1)|, b_1 = -1)."""
    rng = np.random.default_rng(seed_for(BATCH_UNEVEN) if seed is None else seed)
    ms = rng.integers(m_lo, m_hi + 1, size=count)
    ratio = rng.uniform(2.0, 4.0, size=count)
    bad = set(rng.permutation(count)[:int(round(infeasible_frac * count))].tolist())
    out = []
    for k in range(count):
        m = int(ms[k])
        n = int(round(m * ratio[k]))
        lp = planted_dense_f32(m, n, seed=seed_for(BATCH_UNEVEN, 100000 + k) if seed is None else seed + 1 + k)
        if k in bad:
            r2 = np.random.default_rng((seed_for(BATCH_UNEVEN, 200000 + k) if seed is None else seed + 10**6 + k))
            lp.A[0, :] = np.abs(r2.standard_normal(n, dtype=np.float32)).astype(np.float64)
            lp.b = lp.b.copy()
            lp.b[0] = -1.0
            lp.x0 = lp.y0 = lp.s0 = None
            lp.expect = "primal_infeasible"
        lp.meta.update(batch_index=k)
        out.append(lp)
    return out


def l1_svm(d: int = 64, N: int = 512, C: float = 1.0, seed: int | None = None) -> LP:
    """L1-regularised SVM  min ||w||_1 + C sum(xi)  s.t.  y_i (w^T a_i + b0) >= 1 - xi_i,
    xi >= 0, in standard form.  Variables x = [w+ (d), w- (d), b+, b-, xi (N), t (N)],
    n = 2d + 2 + 2N; row i reads  y_i a_i^T (w+ - w-) + y_i (b+ - b-) + xi_i - t_i = 1.
    Labels: N/2 of each sign in a seeded order; a_i ~ N(0.5 y_i e, I).  meta["x_target"]
    is an N(0,1) vector of length n (the target of the differentiation loss)."""
    rng = np.random.default_rng(seed_for(L1_SVM) if seed is None else seed)
    labels = np.concatenate([np.ones(N // 2), -np.ones(N - N // 2)])
    labels = labels[rng.permutation(N)]
    feats = rng.standard_normal((N, d)) + 0.5 * labels[:, None]
    n = 2 * d + 2 + 2 * N
    A = np.zeros((N, n))
    ya = labels[:, None] * feats
    A[:, :d] = ya
    A[:, d:2 * d] = -ya
    A[:, 2 * d] = labels
    A[:, 2 * d + 1] = -labels
    A[np.arange(N), 2 * d + 2 + np.arange(N)] = 1.0
    A[np.arange(N), 2 * d + 2 + N + np.arange(N)] = -1.0
    b = np.ones(N)
    c = np.concatenate([np.ones(2 * d), [0.0, 0.0], C * np.ones(N), np.zeros(N)])
    x_target = rng.standard_normal(n)
    return LP(A=A, b=b, c=c, expect="optimal",
              meta=dict(kind="l1_svm", m=N, n=n, d=d, C=C, x_target=x_target))


def bf16_exact(a: np.ndarray) -> np.ndarray:
    """Round float values to the nearest bfloat16 (ties to even) and return them as float64:
    numbers exactly representable in bfloat16, float32 and float64 alike."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


@dataclass
class SharedBatch:
    """Independent LPs  min c_k^T x  s.t.  A x = b_k,  x >= 0  sharing one dense A."""
    A: np.ndarray
    bs: list
    cs: list
    meta: dict = field(default_factory=dict)


def basis_pursuit(m: int = 2048, n_d: int = 8192, batch: int = 64, density: float = 0.05,
                  seed: Optional[int] = None, bf16: bool = False) -> SharedBatch:
    """Basis pursuit  min ||x||_1  s.t.  D x = b_k  as the standard-form LP with x = x+ - x-:
    A = [D, -D] (m x 2 n_d), c = e, b_k = D x_true_k (in float64 from the exact D).  D iid
    N(0, 1/m) in float32 (with bf16=True rounded further to bfloat16-representable values,
    a case the tensor-core path stores in one bfloat16 term); x_true_k has
    round(density * n_d) nonzeros N(0, 1).  meta["x_true"]: the planted sparse vectors
    (x_true is feasible, so the optimum is at most ||x_true||_1, with equality when l1
    recovery succeeds)."""
    rng = np.random.default_rng(seed_for(BASIS_PURSUIT) if seed is None else seed)
    D = (rng.standard_normal((m, n_d)) / np.sqrt(m)).astype(np.float32).astype(np.float64)
    if bf16:
        D = bf16_exact(D)
    A = np.concatenate([D, -D], axis=1)
    k = int(round(density * n_d))
    xs, bs = [], []
    for _ in range(batch):
        xt = np.zeros(n_d)
        idx = rng.choice(n_d, k, replace=False)
        xt[idx] = rng.standard_normal(k)
        xs.append(xt)
        bs.append(D @ xt)
    cs = [np.ones(2 * n_d) for _ in range(batch)]
    return SharedBatch(A=A, bs=bs, cs=cs, meta=dict(kind="basis_pursuit", m=m, n=2 * n_d, n_d=n_d,
                                                    density=density, x_true=xs, bf16=bf16))


# --- general-form LPs for the presolve (Sec. 4.5) and the SICE LPs (Sec. 5.2) ------------

GENERAL = 6           # general-form LPs with bounds
SICE = 7              # sparse inverse covariance estimation subproblems


@dataclass
class GeneralLP:
    """min c^T x  s.t.  A x = b,  l <= x <= w  (l_j may be -inf, w_j +inf), dense A.
    With a planted optimum (x0, y0, z0): z0 = c - A^T y0 has z0_j >= 0 where x0_j = l_j < w_j,
    <= 0 where x0_j = w_j > l_j, 0 where l_j < x0_j < w_j (any sign where l_j = w_j), so
    p_star = c^T x0 (the KKT conditions of the bounded LP)."""
    A: np.ndarray
    b: np.ndarray
    c: np.ndarray
    l: np.ndarray
    w: np.ndarray
    x0: Optional[np.ndarray] = None
    y0: Optional[np.ndarray] = None
    z0: Optional[np.ndarray] = None
    p_star: Optional[float] = None
    meta: dict = field(default_factory=dict)


def general_lp(m: int = 24, n: int = 60, density: float = 0.3, seed: Optional[int] = None,
               extras: bool = True) -> GeneralLP:
    """A general-form LP with every kind of bound and, with `extras`, the structures each
    reduction of Sec. 4.5 removes: two empty rows (P1), two empty columns (P2), two fixed
    variables (P4), free variables (P5), two singleton rows (P6), and three rows on two
    otherwise unused columns (a structurally over-determined block, P7).
    Column kinds of the m x n core (N(0,1) entries at `density`): 35 % [l, inf),
    25 % [l, w], 10 % (-inf, w], 10 % free, 20 % [l, inf) held at l; bounds l ~ U(-2, 1),
    w = l + U(0.5, 3).  Each bounded variable sits at a bound (nonzero z0 of the matching
    sign) or strictly inside (z0 = 0); y0 ~ N(0, 1)."""
    rng = np.random.default_rng(seed_for(GENERAL) if seed is None else seed)
    A = _sprandn(rng, m, n, density)
    kind = rng.choice(5, size=n, p=[0.35, 0.25, 0.10, 0.10, 0.20])
    l = np.full(n, -np.inf)
    w = np.full(n, np.inf)
    x0 = np.zeros(n)
    z0 = np.zeros(n)
    lo = rng.uniform(-2.0, 1.0, n)
    width = rng.uniform(0.5, 3.0, n)
    for j in range(n):
        k = kind[j]
        if k in (0, 4):                        # [l, inf)
            l[j] = lo[j]
            if k == 4 or rng.random() < 0.4:
                x0[j], z0[j] = l[j], rng.uniform(0.5, 2.0)
            else:
                x0[j] = l[j] + rng.uniform(0.5, 2.0)
        elif k == 1:                           # [l, w]
            l[j], w[j] = lo[j], lo[j] + width[j]
            r = rng.random()
            if r < 1 / 3:
                x0[j], z0[j] = l[j], rng.uniform(0.5, 2.0)
            elif r < 2 / 3:
                x0[j], z0[j] = w[j], -rng.uniform(0.5, 2.0)
            else:
                x0[j] = l[j] + width[j] * rng.uniform(0.2, 0.8)
        elif k == 2:                           # (-inf, w]
            w[j] = lo[j] + width[j]
            if rng.random() < 0.5:
                x0[j], z0[j] = w[j], -rng.uniform(0.5, 2.0)
            else:
                x0[j] = w[j] - rng.uniform(0.5, 2.0)
        else:                                  # free
            x0[j] = rng.standard_normal()
    y0 = rng.standard_normal(m)
    if extras:
        # fixed variables (P4): two interior columns of the core get l = w = x0
        inner = [j for j in range(n) if z0[j] == 0.0 and np.isfinite(l[j])][:2]
        for j in inner:
            l[j] = w[j] = x0[j]
            z0[j] = rng.standard_normal()
        # empty columns (P2): c > 0 at a finite lower bound, c < 0 at a finite upper bound
        Ae = np.zeros((m, 2))
        le = np.array([rng.uniform(-1, 1), -np.inf])
        we = np.array([np.inf, rng.uniform(-1, 1)])
        xe = np.array([le[0], we[1]])
        ze = np.array([rng.uniform(0.5, 2.0), -rng.uniform(0.5, 2.0)])
        # over-determined block (P7): two columns used only by three rows
        xb = rng.uniform(0.5, 2.0, 2)
        A = np.hstack([A, Ae, np.zeros((m, 2))])
        l = np.concatenate([l, le, [0.0, 0.0]])
        w = np.concatenate([w, we, [np.inf, np.inf]])
        x0 = np.concatenate([x0, xe, xb])
        z0 = np.concatenate([z0, ze, [0.0, 0.0]])
        N = A.shape[1]
        blk = np.zeros((3, N))
        blk[:, N - 2:] = [[1.0, 1.0], [1.0, -1.0], [1.0, 2.0]]
        # singleton rows (P6) on two interior core columns, empty rows (P1)
        sing = np.zeros((2, N))
        cols = [j for j in range(n) if z0[j] == 0.0 and np.isfinite(l[j]) and l[j] < w[j]][:2]
        for r, j in enumerate(cols):
            sing[r, j] = rng.uniform(0.5, 2.0) * rng.choice([-1.0, 1.0])
        A = np.vstack([A[:m // 2], np.zeros((1, N)), sing, A[m // 2:], blk, np.zeros((1, N))])
        y0 = rng.standard_normal(A.shape[0])
    b = A @ x0
    c = A.T @ y0 + z0
    return GeneralLP(A=A, b=b, c=c, l=l, w=w, x0=x0, y0=y0, z0=z0, p_star=float(c @ x0),
                     meta=dict(kind="general", m=A.shape[0], n=A.shape[1], extras=extras))


def sice(d: int = 50, samples: Optional[int] = None, seed: Optional[int] = None):
    """Sample covariance Sigma (d x d) of `samples` (default 2d) draws of a zero-mean Gaussian
    whose precision matrix is tridiagonal (1 on the diagonal, -0.4 beside it), and the
    tolerance lam = 1.5 sqrt(log d / samples) of Sec. 5.2."""
    rng = np.random.default_rng(seed_for(SICE) if seed is None else seed)
    N = 2 * d if samples is None else samples
    Om = np.eye(d) - 0.4 * (np.eye(d, k=1) + np.eye(d, k=-1))
    L = np.linalg.cholesky(np.linalg.inv(Om))
    X = rng.standard_normal((N, d)) @ L.T
    X -= X.mean(axis=0)
    Sigma = X.T @ X / N
    lam = 1.5 * np.sqrt(np.log(d) / N)
    return Sigma, float(lam)


def sice_general_lp(Sigma: np.ndarray, lam: float, j: int) -> GeneralLP:
    """Column j of SICE (Sec. 5.2): min ||beta||_1 s.t. ||Sigma beta - e_j||_inf <= lam, as the
    general LP  min e^T beta+ + e^T beta-  s.t.  Sigma beta+ - Sigma beta- - r = e_j,
    beta+/- >= 0, -lam <= r <= lam  (no planted optimum)."""
    d = Sigma.shape[0]
    A = np.hstack([Sigma, -Sigma, -np.eye(d)])
    b = np.zeros(d)
    b[j] = 1.0
    c = np.concatenate([np.ones(2 * d), np.zeros(d)])
    l = np.concatenate([np.zeros(2 * d), np.full(d, -lam)])
    w = np.concatenate([np.full(2 * d, np.inf), np.full(d, lam)])
    return GeneralLP(A=A, b=b, c=c, l=l, w=w, meta=dict(kind="sice", d=d, j=j, lam=lam))
