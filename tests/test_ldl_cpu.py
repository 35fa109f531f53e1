"""Host side of the sparse direct projection (Sec. 4.4, the quasi-definite system), no GPU.

abip_ldl_analyze orders K = [I A^T; A -I] by minimum degree and returns the pattern size of
its LDL^T factor.  Integer work, so it is checked bit-exactly against a brute-force
symbolic elimination written here; the reformulation of the projection's system as a
quasi-definite one is checked against the oracle's projection with a plain dense LDL^T.
"""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1805_12344_gb300 import abip, workloads as W  # noqa: E402
from oracle import abip_oracle as O  # noqa: E402


def _have_lib():
    try:
        abip.lib()
        return True
    except Exception:
        return False


needs_lib = pytest.mark.skipif(not _have_lib(), reason="libabip not built")


def _graph(A_dense):
    """Adjacency (boolean) of K's graph: x_j -- yhat_i for every nonzero A_ij."""
    m, n = A_dense.shape
    N = m + n
    G = np.zeros((N, N), dtype=bool)
    rows, cols = np.nonzero(A_dense)
    G[cols, n + rows] = True
    G[n + rows, cols] = True
    return G


def _eliminate(G, perm):
    """Symbolic elimination in the order perm: per pivot its degree in the elimination
    graph, the least degree among the remaining nodes (smallest node on ties), and the
    pattern size of its column of L."""
    G = G.copy()
    N = G.shape[0]
    alive = np.ones(N, dtype=bool)
    degs, mins, counts = [], [], []
    for v in perm:
        deg = (G & alive[None, :]).sum(axis=1)
        deg_alive = np.where(alive, deg, N + 1)
        mins.append((int(deg_alive.min()), int(np.argmin(deg_alive))))
        nb = np.nonzero(G[v] & alive)[0]
        nb = nb[nb != v]
        degs.append(len(nb))
        counts.append(len(nb))
        G[np.ix_(nb, nb)] = True
        np.fill_diagonal(G, False)
        alive[v] = False
    return np.array(degs), mins, np.array(counts)


def _cases():
    out = []
    for k, (m, n) in enumerate([(3, 5), (5, 9), (8, 14)]):
        rng = np.random.default_rng(100 + k)
        A = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.35)
        A[np.arange(m), rng.choice(n, m, replace=False)] = 1.0   # no empty row
        out.append(("random%d" % k, A))
    out.append(("grid4", W.grid_flow(4).A.to_dense()))
    out.append(("grid6", W.grid_flow(6).A.to_dense()))
    out.append(("sparse_planted", W.planted_sparse(m=20, per_col=3, seed=7).A.to_dense()))
    out.append(("dense", np.random.default_rng(3).standard_normal((6, 10))))
    return out


@needs_lib
@pytest.mark.parametrize("name,A", _cases(), ids=[c[0] for c in _cases()])
def test_ldl_analyze_matches_brute_force_elimination(name, A):
    m, n = A.shape
    perm, counts, nnz = abip.abip_ldl_analyze(A)
    assert sorted(perm.tolist()) == list(range(m + n))
    G = _graph(A)
    degs, mins, bf_counts = _eliminate(G, perm)
    # the pattern of each column of L is the pivot's neighbourhood when it is eliminated
    np.testing.assert_array_equal(counts, bf_counts)
    assert nnz == int(counts.sum())
    # minimum degree with ties to the smaller node, until the rest is a complete graph
    # (then node order): every pivot has the least degree among the remaining nodes
    for p, v in enumerate(perm):
        least, first = mins[p]
        assert degs[p] == least, (p, v)
        remaining = m + n - p
        if least < remaining - 1:
            assert v == first, (p, v, first)
        else:
            assert list(perm[p:]) == sorted(perm[p:])
            break


@needs_lib
def test_ldl_analyze_is_deterministic_and_accepts_csr():
    lp = W.grid_flow(8)
    p1, c1, z1 = abip.abip_ldl_analyze(lp.A)
    p2, c2, z2 = abip.abip_ldl_analyze(lp.A.to_dense())
    np.testing.assert_array_equal(p1, p2)
    np.testing.assert_array_equal(c1, c2)
    assert z1 == z2
    # a 2-D grid keeps the factor far from dense under minimum degree
    N = lp.m + lp.n
    assert z1 < 0.1 * N * (N - 1) / 2


@needs_lib
def test_ldl_analyze_refuses_device_matrices_and_bad_input():
    import ctypes as C
    lib = abip.lib()
    A = np.ones((2, 3))
    M, keep = abip._matrix(A)
    M.on_device = 1
    assert lib.abip_ldl_analyze(C.byref(M), None, None, None) == abip.ABIP_E_INVALID_ARG
    assert lib.abip_ldl_analyze(None, None, None, None) == abip.ABIP_E_INVALID_ARG
    M2, keep2 = abip._matrix(np.ones((3, 2)))
    assert lib.abip_ldl_analyze(C.byref(M2), None, None, None) == abip.ABIP_E_DIM


@needs_lib
def test_direct_projection_refuses_reduced_precision():
    lp = W.grid_flow(4)
    for prec in (abip.ABIP_PREC_MIXED, abip.ABIP_PREC_MIXED_BF16):
        with pytest.raises(abip.AbipError) as e:
            abip.abip_setup(lp.A, lp.b, lp.c, abip.default_params(linsys=abip.ABIP_LINSYS_SPARSE_LDL, precision=prec))
        assert e.value.code == abip.ABIP_E_INVALID_ARG
        assert "FP64" in str(e.value)


@needs_lib
@pytest.mark.parametrize("name,A", _cases()[:5], ids=[c[0] for c in _cases()[:5]])
def test_quasi_definite_ldl_reproduces_the_projection(name, A):
    """With yhat = -y, M [y; x] = r is K [x; yhat] = [r_x; r_y].  A plain dense LDL^T of
    P K P^T (P from the library's order) exists with D > 0 on x nodes and D < 0 on row
    nodes, and its solution equals the oracle's M-solve."""
    m, n = A.shape
    N = m + n
    perm, _, _ = abip.abip_ldl_analyze(A)
    K = np.zeros((N, N))
    K[:n, :n] = np.eye(n)
    K[n:, n:] = -np.eye(m)
    K[:n, n:] = A.T
    K[n:, :n] = A
    Kp = K[np.ix_(perm, perm)]
    L = np.eye(N)
    D = np.zeros(N)
    for j in range(N):
        D[j] = Kp[j, j] - np.sum(L[j, :j] ** 2 * D[:j])
        for i in range(j + 1, N):
            L[i, j] = (Kp[i, j] - np.sum(L[i, :j] * L[j, :j] * D[:j])) / D[j]
    np.testing.assert_allclose(L @ np.diag(D) @ L.T, Kp, atol=1e-10)
    assert np.all((D > 0) == (perm < n))
    rng = np.random.default_rng(5)
    ry, rx = rng.standard_normal(m), rng.standard_normal(n)
    rhs = np.concatenate([rx, ry])[perm]
    z = np.linalg.solve(L, rhs)
    w = np.linalg.solve(L.T, z / D)
    sol = np.empty(N)
    sol[perm] = w
    x, y = sol[:n], -sol[n:]
    P = O.Problem(A, np.zeros(m), np.zeros(n))
    zy, zx = O.solve_M(P, O.DenseCholesky(P), ry, rx)
    np.testing.assert_allclose(y, zy, atol=1e-10)
    np.testing.assert_allclose(x, zx, atol=1e-10)


@pytest.mark.parametrize("side", [2, 3, 5])
def test_grid_flow_structure_and_planted_pair(side):
    """Node-arc incidence with one row dropped: every arc column holds +1 at its tail and
    -1 at its head (one of them absent when it touches the dropped node), A has full row
    rank (Sec. 2's assumption), and the planted pair is optimal by construction:
    x0, s0 >= 0, x0 o s0 = 0, b = A x0, c = A^T y0 + s0."""
    lp = W.grid_flow(side)
    A = lp.A.to_dense()
    nodes = side * side
    assert lp.m == nodes - 1 and lp.n == 4 * side * (side - 1)
    assert set(np.unique(A)) <= {-1.0, 0.0, 1.0}
    sums = A.sum(axis=0)
    dropped = np.abs(A).sum(axis=0) == 1          # arcs touching the dropped node
    assert np.all(sums[~dropped] == 0) and np.all(np.abs(sums[dropped]) == 1)
    assert np.linalg.matrix_rank(A) == lp.m
    assert np.all(lp.x0 >= 0) and np.all(lp.s0 >= 0) and np.all(lp.x0 * lp.s0 == 0)
    np.testing.assert_allclose(A @ lp.x0, lp.b, atol=1e-12)
    np.testing.assert_allclose(A.T @ lp.y0 + lp.s0, lp.c, atol=1e-12)


def test_oracle_reaches_the_grid_flow_optimum():
    """The oracle (exact projection) solves the 3 x 3 grid flow LP to the planted optimum."""
    lp = W.grid_flow(3)
    r = O.solve(lp.A.to_dense(), lp.b, lp.c, O.Params(linsys=0))
    assert r.status == O.OPTIMAL
    assert abs(r.obj - lp.p_star) <= 1e-5 * max(1.0, abs(lp.p_star))
