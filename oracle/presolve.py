"""Presolve, reformulation to standard form, scaling and postsolve (Sec. 4.5 and the Remark
closing it): the plain reference for the library's host presolve.

TEST INFRASTRUCTURE: only the tests import this module (the library never does).

Input: the general LP of Sec. 4.5,

    min c^T x   s.t.  A x = b,  l <= x <= w      (l_j may be -inf, w_j may be +inf).

Steps, in this order (readings P-A .. P-F state what the paper leaves open):

1. Reductions P1-P6, in passes until a pass changes nothing.  Each pass scans the
   columns in index order for P3 (l_j > w_j: infeasible) and P4 (l_j = w_j: fixed),
   then the rows in index order for P1 (no entry in an active column) and P6 (exactly one
   entry a_ik in an active column: x_k = b_i / a_ik, infeasible if outside [l_k, w_k]
   by more than the tolerance), then the columns for P2 (no entry in an active row: x_j at
   the bound that minimises c_j x_j; c_j != 0 toward an infinite bound is dual infeasible
   (reading P-A: P2 with c_j = 0 takes the finite bound nearest 0, or 0 if free).
   A fixed variable leaves the problem: b_r -= a_rj x_j for its rows, the objective
   constant gains c_j x_j.  An empty row with |b_i| <= tol (1 + ||b||_inf) is dropped,
   else infeasible (reading P-B: the tolerance).
2. P7: the rows that the Dulmage-Mendelsohn decomposition of the remaining pattern puts
   in its over-determined part (the rows reachable from a row left unmatched by a maximum
   matching, along alternating paths) have entries only in the matched columns of that
   part, so they are linearly dependent; among them, in index order, a row whose values
   are (to tolerance) a combination of the rows kept before it is dropped when b agrees
   with the same combination, else the LP is infeasible (reading P-C: which rows of the
   dependent part go, and the tolerance).
3. Reformulation (Sec. 4.5's last step), per remaining column in index order: l finite:
   x = l + xbar; if w is finite too, a new row xbar_j + t_j = w_j - l_j with a new column
   t_j >= 0 (rows appended after the equality rows, columns after the structural ones).
   l = -inf, w finite: x = w - xbar (the column and its cost change sign; reading P-D,
   the paper assumes l > -inf after presolve).  Free (P5): x = x+ - x-, two columns.
4. Scaling (the Remark; reading P-E, a Ruiz equilibration): `ruiz` passes of
   D_i <- D_i / sqrt(max_j |a_ij|), E_j <- E_j / sqrt(max_i |a_ij|) on the current scaled
   matrix, then Ahat = D A E, bhat = D b, chat = E c.  A solution (xh, yh, sh) of the
   scaled LP maps back as x = E xh, y = D yh, s = E^-1 sh.
5. Postsolve: undo 4 and 3, restore the removed columns at their fixed values, and the
   duals: y = 0 on dropped rows (P1, P7), and for the singleton rows, in the reverse of
   their removal order, y_i = (c_k - sum_{r != i} a_rk y_r) / a_ik, which makes the
   reduced cost of the variable it fixed zero (reading P-F).  Reduced costs z = c - A^T y.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import maximum_bipartite_matching

OPTIMAL_SO_FAR = 0          # reductions done; the standard-form LP is to be solved
OPTIMAL_BY_REDUCTION = 1    # every row removed: the reductions solved the LP (postsolve of empty x, y)
PRIMAL_INFEASIBLE = 2       # the status codes of the solver (abip_oracle)
DUAL_INFEASIBLE = 3


@dataclass
class Presolved:
    status: int
    A: Optional[sp.csr_matrix] = None       # standard form, scaled
    b: Optional[np.ndarray] = None
    c: Optional[np.ndarray] = None
    obj_offset: float = 0.0                  # add to c^T x of the standard form
    # postsolve records
    m0: int = 0
    n0: int = 0
    A0: Optional[sp.csc_matrix] = None
    c0: Optional[np.ndarray] = None
    fixed: dict = field(default_factory=dict)        # column -> value (P2, P4, P6)
    singleton: list = field(default_factory=list)    # (row, column) in removal order
    rows: Optional[np.ndarray] = None                # original index of each equality row kept
    cols: list = field(default_factory=list)         # per kept column: (original j, kind, bound)
    D: Optional[np.ndarray] = None
    E: Optional[np.ndarray] = None
    removed: dict = field(default_factory=dict)      # counts per rule
    why: str = ""


def _active_entries(Acsr, i, col_on):
    lo, hi = Acsr.indptr[i], Acsr.indptr[i + 1]
    js = Acsr.indices[lo:hi]
    vs = Acsr.data[lo:hi]
    keep = col_on[js] & (vs != 0.0)
    return js[keep], vs[keep]


def _dm_overdetermined(S: sp.csr_matrix):
    """Rows and columns of the over-determined part of the Dulmage-Mendelsohn decomposition
    of the pattern of S: from every row unmatched by a maximum matching, alternate row ->
    any column of the row -> the row matched to that column."""
    m, n = S.shape
    if m == 0:
        return np.zeros(0, dtype=bool), np.zeros(0, dtype=bool)
    pat = sp.csr_matrix((np.ones(S.nnz), S.indices, S.indptr), shape=S.shape)
    col_of_row = maximum_bipartite_matching(pat, perm_type="column")    # -1: unmatched
    row_of_col = np.full(n, -1)
    for i, j in enumerate(col_of_row):
        if j >= 0:
            row_of_col[j] = i
    r_seen = np.zeros(m, dtype=bool)
    c_seen = np.zeros(n, dtype=bool)
    stack = [i for i in range(m) if col_of_row[i] < 0]
    for i in stack:
        r_seen[i] = True
    while stack:
        i = stack.pop()
        for j in pat.indices[pat.indptr[i]:pat.indptr[i + 1]]:
            if not c_seen[j]:
                c_seen[j] = True
                r = row_of_col[j]
                if r >= 0 and not r_seen[r]:
                    r_seen[r] = True
                    stack.append(r)
    return r_seen, c_seen


def presolve(A, b, c, l, w, tol: float = 1e-9, ruiz: int = 10) -> Presolved:
    A0 = sp.csr_matrix(A, dtype=np.float64)
    A0.eliminate_zeros()
    A0.sort_indices()
    m0, n0 = A0.shape
    b = np.array(b, dtype=np.float64)
    c0 = np.array(c, dtype=np.float64)
    l = np.array(l, dtype=np.float64)
    w = np.array(w, dtype=np.float64)
    Acsc = A0.tocsc()
    row_on = np.ones(m0, dtype=bool)
    col_on = np.ones(n0, dtype=bool)
    P = Presolved(status=OPTIMAL_SO_FAR, m0=m0, n0=n0, A0=Acsc, c0=c0,
                  removed=dict(P1=0, P2=0, P4=0, P6=0, P7=0, P5=0))
    bscale = 1.0 + (np.abs(b).max() if m0 else 0.0)
    offset = 0.0

    def fix(j, v):
        nonlocal offset
        col_on[j] = False
        P.fixed[j] = v
        offset += c0[j] * v
        lo, hi = Acsc.indptr[j], Acsc.indptr[j + 1]
        for r, a in zip(Acsc.indices[lo:hi], Acsc.data[lo:hi]):
            if row_on[r]:
                b[r] -= a * v

    def fail(status, why):
        P.status, P.why = status, why
        return P

    changed = True
    while changed:
        changed = False
        for j in range(n0):                                   # P3, P4
            if not col_on[j]:
                continue
            if l[j] > w[j]:
                return fail(PRIMAL_INFEASIBLE, f"P3: l > w at column {j}")
            if l[j] == w[j]:
                fix(j, l[j])
                P.removed["P4"] += 1
                changed = True
        for i in range(m0):                                   # P1, P6
            if not row_on[i]:
                continue
            js, vs = _active_entries(A0, i, col_on)
            if js.size == 0:
                if abs(b[i]) > tol * bscale:
                    return fail(PRIMAL_INFEASIBLE, f"P1: empty row {i} with b = {b[i]:g}")
                row_on[i] = False
                P.removed["P1"] += 1
                changed = True
            elif js.size == 1:
                k, a = int(js[0]), float(vs[0])
                v = b[i] / a
                slack = tol * max(1.0, abs(v))
                if v < l[k] - slack or v > w[k] + slack:
                    return fail(PRIMAL_INFEASIBLE, f"P6: row {i} fixes column {k} outside its bounds")
                v = min(max(v, l[k]), w[k])
                row_on[i] = False
                P.singleton.append((i, k))
                fix(k, v)
                P.removed["P6"] += 1
                changed = True
        for j in range(n0):                                   # P2
            if not col_on[j]:
                continue
            lo, hi = Acsc.indptr[j], Acsc.indptr[j + 1]
            if np.any(row_on[Acsc.indices[lo:hi]] & (Acsc.data[lo:hi] != 0.0)):
                continue
            if c0[j] > 0:
                if not np.isfinite(l[j]):
                    return fail(DUAL_INFEASIBLE, f"P2: empty column {j} unbounded below")
                v = l[j]
            elif c0[j] < 0:
                if not np.isfinite(w[j]):
                    return fail(DUAL_INFEASIBLE, f"P2: empty column {j} unbounded below")
                v = w[j]
            else:
                v = min(max(0.0, l[j]), w[j])
            fix(j, v)
            P.removed["P2"] += 1
            changed = True

    # P7 on the remaining rows and columns
    rows = np.nonzero(row_on)[0]
    cols = np.nonzero(col_on)[0]
    S = A0[rows][:, cols].tocsr()
    S.eliminate_zeros()
    r_over, _ = _dm_overdetermined(S)
    if r_over.any():
        kept = []
        for t in np.nonzero(r_over)[0]:
            row = S.getrow(t).toarray().ravel()
            if kept:
                K = np.array([S.getrow(u).toarray().ravel() for u in kept])
                alpha, *_ = np.linalg.lstsq(K.T, row, rcond=None)
                resid = np.linalg.norm(K.T @ alpha - row)
            else:
                alpha, resid = np.zeros(0), np.linalg.norm(row)
            if resid > tol * max(1.0, np.linalg.norm(row)):
                kept.append(t)
                continue
            bt = b[rows[kept]] @ alpha
            if abs(b[rows[t]] - bt) > tol * bscale:
                return fail(PRIMAL_INFEASIBLE, f"P7: dependent row {rows[t]} with inconsistent b")
            row_on[rows[t]] = False
            P.removed["P7"] += 1
        rows = np.nonzero(row_on)[0]

    # reformulation to standard form
    Ak = A0[rows][:, cols].tocsc()
    bk = b[rows].copy()
    m = rows.size
    col_blocks, cost, kinds = [], [], []
    up_rows, up_rhs = [], []               # (standard column index, w - l)
    for t, j in enumerate(cols):
        a = Ak.getcol(t)
        if np.isfinite(l[j]):
            bk -= a.toarray().ravel() * l[j]
            offset += c0[j] * l[j]
            kinds.append((int(j), "lo", float(l[j])))
            col_blocks.append(a)
            cost.append(c0[j])
            if np.isfinite(w[j]):
                up_rows.append((len(col_blocks) - 1, w[j] - l[j]))
        elif np.isfinite(w[j]):
            bk -= a.toarray().ravel() * w[j]
            offset += c0[j] * w[j]
            kinds.append((int(j), "up", float(w[j])))
            col_blocks.append(-a)
            cost.append(-c0[j])
        else:
            kinds.append((int(j), "free", 0.0))
            col_blocks.append(a)
            col_blocks.append(-a)
            cost += [c0[j], -c0[j]]
            P.removed["P5"] += 1
    nstruct = len(col_blocks)
    nu = len(up_rows)
    Astruct = sp.hstack(col_blocks, format="csr") if col_blocks else sp.csr_matrix((m, 0))
    if nu:
        Eu = sp.csr_matrix((np.ones(nu), ([r for r in range(nu)], [k for k, _ in up_rows])), shape=(nu, nstruct))
        top = sp.hstack([Astruct, sp.csr_matrix((m, nu))])
        bot = sp.hstack([Eu, sp.identity(nu, format="csr")])
        Astd = sp.vstack([top, bot], format="csr")
        bstd = np.concatenate([bk, [r for _, r in up_rows]])
        cstd = np.concatenate([cost, np.zeros(nu)])
    else:
        Astd = Astruct.tocsr()
        bstd = bk
        cstd = np.array(cost, dtype=np.float64)

    # Ruiz equilibration
    ms, ns = Astd.shape
    D = np.ones(ms)
    E = np.ones(ns)
    S = Astd.copy()
    for _ in range(ruiz):
        ra = np.asarray(abs(S).max(axis=1).todense()).ravel() if ns else np.zeros(ms)
        ca = np.asarray(abs(S).max(axis=0).todense()).ravel() if ms else np.zeros(ns)
        dr = np.where(ra > 0, 1.0 / np.sqrt(np.where(ra > 0, ra, 1.0)), 1.0)
        dc = np.where(ca > 0, 1.0 / np.sqrt(np.where(ca > 0, ca, 1.0)), 1.0)
        D *= dr
        E *= dc
        S = sp.diags(dr) @ S @ sp.diags(dc)
    Ahat = (sp.diags(D) @ Astd @ sp.diags(E)).tocsr()
    Ahat.sort_indices()
    P.A, P.b, P.c = Ahat, D * bstd, E * cstd
    P.obj_offset = offset
    P.rows, P.cols, P.D, P.E = rows, kinds, D, E
    if ms == 0:          # the reductions removed every row (and so every column): solved
        P.status = OPTIMAL_BY_REDUCTION
    return P


def postsolve(P: Presolved, x, y, s):
    """(x, y, z, objective) of the original LP from a solution (x, y, s) of the standard-form
    LP `P.A, P.b, P.c`.  z = c - A^T y are the original reduced costs."""
    xs = P.E * np.asarray(x, dtype=np.float64)
    ys = P.D * np.asarray(y, dtype=np.float64)
    xo = np.zeros(P.n0)
    for j, v in P.fixed.items():
        xo[j] = v
    t = 0
    for j, kind, bound in P.cols:
        if kind == "lo":
            xo[j] = bound + xs[t]
            t += 1
        elif kind == "up":
            xo[j] = bound - xs[t]
            t += 1
        else:
            xo[j] = xs[t] - xs[t + 1]
            t += 2
    yo = np.zeros(P.m0)
    yo[P.rows] = ys[:P.rows.size]
    A = P.A0
    for i, k in reversed(P.singleton):
        lo, hi = A.indptr[k], A.indptr[k + 1]
        acc = P.c0[k]
        aik = 0.0
        for r, a in zip(A.indices[lo:hi], A.data[lo:hi]):
            if r == i:
                aik = a
            else:
                acc -= a * yo[r]
        yo[i] = acc / aik
    z = P.c0 - A.T @ yo
    return xo, yo, z, float(P.c0 @ xo)
