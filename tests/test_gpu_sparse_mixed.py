"""GPU parity of the sparse (Jacobi-PCG) path in mixed precision: the persistent kernel
that keeps the iterate and its products in FP64 and runs every product and the PCG
correction solves in FP32 (precision = ABIP_PREC_MIXED on a CSR A), through the C ABI,
against the FP64 oracle.

Bars, stated per test:
* end to end: identical status; relative primal and dual residuals and gap <= 1e-6 (as
  the kernel reports them, and recomputed on the host in FP64 from the returned
  candidate); objective within 1e-5 relative of the oracle's and of the planted optimum;
* first updates: the stacked state after 20 updates within 1e-6 relative of the oracle's.
  The products of changes carry FP32 rounding of about 6e-8 times the size of each change
  (unit roundoff times the row norm of A), and each correction solve stops at the PCG
  tolerance, so early iterates agree to about 1e-7 relative, not to the 1e-10 of the
  FP64 path.
"""
import numpy as np
import pytest

from oracle import abip_oracle as O
from paper_1805_12344_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OBJ_TOL = 1e-5
RES_TOL = 1e-6
EARLY_TOL = 1e-6


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


def _host_residuals(A, b, c, x, y, s):
    """Sec. 4.1 relative residuals of the returned candidate, in FP64 on the host."""
    Ax = A @ x
    ATy = A.T @ y
    pres = np.linalg.norm(Ax - b) / (1 + np.linalg.norm(b))
    dres = np.linalg.norm(ATy + s - c) / (1 + np.linalg.norm(c))
    ctx, bty = c @ x, b @ y
    gap = abs(ctx - bty) / (1 + abs(ctx) + abs(bty))
    return pres, dres, gap


def _mixed(abip, A, b, c, **kw):
    return abip.Solver(A, b, c, precision=abip.ABIP_PREC_MIXED, **kw)


def _check_optimal(info, x, y, s, lp, ref_obj):
    assert info["status"] == O.OPTIMAL
    assert max(info["pres"], info["dres"], info["dgap"]) <= RES_TOL
    A = lp.A.to_scipy() if isinstance(lp.A, W.CSR) else lp.A
    pres, dres, gap = _host_residuals(A, lp.b, lp.c, x, y, s)
    # the kernel decides on residuals of A's FP32 values; 1 % slack for the host's rounding
    assert max(pres, dres, gap) <= RES_TOL * 1.01, (pres, dres, gap)
    assert np.all(x >= 0) and np.all(s >= 0)
    if ref_obj is not None:
        assert abs(info["obj"] - ref_obj) <= OBJ_TOL * max(1.0, abs(ref_obj))
    if lp.p_star is not None:
        assert abs(info["obj"] - lp.p_star) <= OBJ_TOL * max(1.0, abs(lp.p_star))


def test_mixed_sparse_first_updates(abip):
    """20 updates on the 300 x 1200 sparse LP (slices of several widths, a ragged last
    slice) against the oracle's iterate."""
    lp = W.planted_sparse(300, seed=W.seed_for(W.SPARSE_PLANTED, 20))
    ref = O.solve(lp.A.to_scipy(), lp.b, lp.c, O.Params(linsys=1, cg_tol=1e-13, max_admm_iters=20),
                  trace_iters=20)
    s = _mixed(abip, lp.A, lp.b, lp.c, cg_tol=1e-10, max_admm_iters=20)
    info, *_ = s.solve()
    assert info["admm_iters"] == 20
    rel = _rel(s.stacked_state(), ref.trace[-1])
    assert rel <= EARLY_TOL, rel


@pytest.mark.parametrize("m,seed", [(80, 10), (300, 30)])
def test_mixed_sparse_end_to_end(abip, oracle_memo, m, seed):
    lp = W.planted_sparse(m, seed=W.seed_for(W.SPARSE_PLANTED, seed))
    ref = oracle_memo(("sparse", m, seed),
                      lambda: O.solve(lp.A.to_scipy(), lp.b, lp.c, O.Params(linsys=1, cg_tol=1e-10)))
    assert ref.status == O.OPTIMAL
    s = _mixed(abip, lp.A, lp.b, lp.c, cg_tol=1e-10)
    info, x, y, sv = s.solve()
    _check_optimal(info, x, y, sv, lp, ref.obj)
    assert info["fp32_iters"] == info["admm_iters"]
    # the FP64 path on the same LP reaches the same optimum
    f = abip.Solver(lp.A, lp.b, lp.c, cg_tol=1e-10)
    i64, *_ = f.solve()
    assert i64["status"] == O.OPTIMAL
    assert abs(i64["obj"] - info["obj"]) <= OBJ_TOL * max(1.0, abs(ref.obj))


def test_mixed_sparse_m2000(abip):
    """2000 x 8000 (nnz 50000): beyond what the oracle finishes in a test (its update count
    grows with m); the planted pair fixes the optimum and the status (a planted LP with
    a strictly complementary pair is solvable, Sec. 2), and the host recomputes the
    residuals of the returned candidate in FP64."""
    lp = W.planted_sparse(2000, seed=W.seed_for(W.SPARSE_PLANTED, 40))
    s = _mixed(abip, lp.A, lp.b, lp.c, cg_tol=1e-10)
    info, x, y, sv = s.solve()
    _check_optimal(info, x, y, sv, lp, None)


def test_mixed_dense_as_csr_end_to_end(abip):
    """The 50 x 120 dense planted LP through the CSR path (FP64 values rounded to FP32:
    the kernel solves the LP of the rounded A, whose optimum differs by ~1e-7 relative)."""
    lp = W.planted_dense()
    ref = O.solve(lp.A, lp.b, lp.c, O.Params(linsys=1, cg_tol=1e-10))
    s = _mixed(abip, W.dense_to_csr(lp.A), lp.b, lp.c, cg_tol=1e-10)
    info, x, y, sv = s.solve()
    assert info["status"] == ref.status == O.OPTIMAL
    assert max(info["pres"], info["dres"], info["dgap"]) <= RES_TOL
    assert abs(info["obj"] - ref.obj) <= OBJ_TOL * max(1.0, abs(ref.obj))


@pytest.mark.parametrize("make", [W.infeasible_twin, W.dual_infeasible])
def test_mixed_sparse_infeasible_status(abip, make):
    lp = make()
    A32 = lp.A.astype(np.float32).astype(np.float64)
    ref = O.solve(A32, lp.b, lp.c, O.Params(linsys=1))
    s = _mixed(abip, W.dense_to_csr(A32, np.float32), lp.b, lp.c)
    info, x, y, sv = s.solve()
    assert info["status"] == ref.status == {"primal_infeasible": 2, "dual_infeasible": 3}[lp.expect]
    assert info["kappa"] > 0 and info["tau"] < 1e-6 * info["kappa"]
    if info["status"] == O.PRIMAL_INFEASIBLE:
        assert abs(lp.b @ y - 1.0) < 1e-9
        assert np.linalg.norm(A32.T @ y + sv) <= 1e-6 / np.linalg.norm(lp.b) * 1.01
    else:
        assert abs(lp.c @ x + 1.0) < 1e-9
        assert np.linalg.norm(A32 @ x) <= 1e-6 / np.linalg.norm(lp.c) * 1.01


def test_mixed_sparse_set_state_resumes(abip):
    """abip_set_state on the mixed sparse path: a run resumed from the state after 40
    updates ends at the same optimum as an uninterrupted one."""
    lp = W.planted_sparse(80, seed=W.seed_for(W.SPARSE_PLANTED, 10))
    a = _mixed(abip, lp.A, lp.b, lp.c, cg_tol=1e-10, max_admm_iters=40)
    a.solve()
    st = a.state()
    b = _mixed(abip, lp.A, lp.b, lp.c, cg_tol=1e-10)
    b.set_state(st)
    info, x, y, sv = b.solve()
    _check_optimal(info, x, y, sv, lp, None)
