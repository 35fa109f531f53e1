"""Brute-force basis enumeration for tiny standard-form LPs (test infrastructure only).

A pin for the ABIP oracle that shares nothing with it: for  min c^T x, A x = b,
x >= 0  with A of full row rank (Sec. 2, problem (P)/(D)), every basic solution
comes from an m-column subset B with A_B nonsingular:  x_B = A_B^{-1} b, x_N = 0.
It is primal feasible when x_B >= 0 and dual feasible when the reduced costs
c - A^T y, y = A_B^{-T} c_B, are >= 0.  By the fundamental theorem of LP:
  * a basis that is primal and dual feasible is optimal, p* = c_B^T x_B;
  * primal feasible with no such basis  ->  unbounded (dual infeasible);
  * no primal-feasible basis  ->  primal infeasible.
Only for m <= 6 and n <= 14 or so (C(n, m) subsets).
"""
from __future__ import annotations

import itertools

import numpy as np


def enumerate_lp(A, b, c, tol: float = 1e-9):
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    m, n = A.shape
    if np.linalg.matrix_rank(A) < m:
        raise ValueError("A must have full row rank")
    any_primal = False
    best = None
    best_x = []
    for B in itertools.combinations(range(n), m):
        AB = A[:, B]
        if abs(np.linalg.det(AB)) < 1e-10:
            continue
        xB = np.linalg.solve(AB, b)
        if np.min(xB) < -tol:
            continue
        any_primal = True
        y = np.linalg.solve(AB.T, c[list(B)])
        red = c - A.T @ y
        if np.min(red) < -tol:
            continue
        x = np.zeros(n)
        x[list(B)] = xB
        obj = float(c @ x)
        if best is None or obj < best - 1e-12:
            best = obj
        best_x.append(x)
    if not any_primal:
        return dict(status="primal_infeasible")
    if best is None:
        return dict(status="dual_infeasible")
    return dict(status="optimal", p_star=best, optimal_vertices=best_x)
