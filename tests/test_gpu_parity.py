"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Bars (stated per test): FP64 iterates within 1e-10 relative for the first 20 ADMM
updates; at the end identical status, relative residuals <= 1e-6, objective within
1e-5 relative of the oracle's.
"""
import numpy as np
import pytest

from oracle import abip_oracle as O
from paper_1805_12344_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ITER_TOL = 1e-10
OBJ_TOL = 1e-5


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


def _first_iterates_gpu(abip, A, b, c, K, **prm):
    out = []
    for k in range(1, K + 1):
        s = abip.Solver(A, b, c, max_admm_iters=k, **prm)
        info, *_ = s.solve()
        assert info["admm_iters"] == k
        out.append(s.stacked_state())
        s.close()
    return out


def _check_end(info, ref, lp=None):
    assert info["status"] == ref.status
    if ref.status == O.OPTIMAL:
        assert max(info["pres"], info["dres"], info["dgap"]) <= 1e-6
        assert abs(info["obj"] - ref.obj) <= OBJ_TOL * max(1.0, abs(ref.obj))
        if lp is not None and lp.p_star is not None:
            assert abs(info["obj"] - lp.p_star) <= OBJ_TOL * max(1.0, abs(lp.p_star))


# --- dense Cholesky path (one CTA per LP) -----------------------------------

def test_dense_first_20_iterates(abip):
    lp = W.planted_dense()
    ref = O.solve(lp.A, lp.b, lp.c, O.Params(max_admm_iters=20), trace_iters=20)
    got = _first_iterates_gpu(abip, lp.A, lp.b, lp.c, 20)
    for k in range(20):
        assert _rel(got[k], ref.trace[k]) <= ITER_TOL, (k, _rel(got[k], ref.trace[k]))


def test_dense_planted_end_to_end(abip):
    lp = W.planted_dense()
    ref = O.solve(lp.A, lp.b, lp.c)
    s = abip.Solver(lp.A, lp.b, lp.c)
    info, x, y, sv = s.solve()
    _check_end(info, ref, lp)
    # returned candidate: independent FP64 residuals on the host
    assert np.linalg.norm(lp.A @ x - lp.b) <= 1e-6 * (1 + np.linalg.norm(lp.b)) * 1.01
    assert np.linalg.norm(lp.A.T @ y + sv - lp.c) <= 1e-6 * (1 + np.linalg.norm(lp.c)) * 1.01
    assert np.all(x >= 0) and np.all(sv >= 0)


@pytest.mark.parametrize("make", [W.infeasible_twin, W.dual_infeasible])
def test_dense_infeasible_status(abip, make):
    lp = make()
    ref = O.solve(lp.A, lp.b, lp.c)
    s = abip.Solver(lp.A, lp.b, lp.c)
    info, x, y, sv = s.solve()
    assert info["status"] == ref.status == {"primal_infeasible": 2, "dual_infeasible": 3}[lp.expect]
    assert info["kappa"] > 0 and info["tau"] < 1e-6 * info["kappa"]
    if info["status"] == 2:
        assert abs(lp.b @ y - 1.0) < 1e-9
        assert np.linalg.norm(lp.A.T @ y + sv) <= 1e-6 / np.linalg.norm(lp.b) * 1.01
    else:
        assert abs(lp.c @ x + 1.0) < 1e-9
        assert np.linalg.norm(lp.A @ x) <= 1e-6 / np.linalg.norm(lp.c) * 1.01


@pytest.mark.parametrize("m,n", [(1, 3), (7, 7), (33, 70), (64, 200)])
def test_dense_shapes_and_ragged_tiles(abip, m, n):
    """m = 1, m = n, and sizes that are not multiples of the 32-row triangular-solve block."""
    lp = W.planted_dense(m, n, seed=W.seed_for(W.DENSE_PLANTED, 200 + m))
    ref = O.solve(lp.A, lp.b, lp.c, O.Params(max_admm_iters=20), trace_iters=20)
    s = abip.Solver(lp.A, lp.b, lp.c, max_admm_iters=20)
    s.solve()
    assert _rel(s.stacked_state(), ref.trace[-1]) <= ITER_TOL


def test_sqrt_gamma_warm_start_and_outer_count(abip):
    lp = W.planted_dense(8, 20, seed=5)
    ref = O.solve(lp.A, lp.b, lp.c, O.Params(warmstart=1, max_admm_iters=200), trace_iters=200)
    s = abip.Solver(lp.A, lp.b, lp.c, warmstart=1, max_admm_iters=200)
    s.solve()
    assert _rel(s.stacked_state(), ref.trace[-1]) <= 1e-9
    r2 = O.solve(lp.A, lp.b, lp.c, O.Params(gamma=0.5, eps=1e-3, stop_rule=1))
    s2 = abip.Solver(lp.A, lp.b, lp.c, gamma=0.5, eps=1e-3, stop_rule=1)
    info, *_ = s2.solve()
    assert info["outer_iters"] == r2.outer_iters == 10


# --- CSR / Jacobi-PCG path (persistent grid kernel) --------------------------

def test_pcg_first_20_iterates_dense_as_csr(abip):
    lp = W.planted_dense()
    A = W.dense_to_csr(lp.A)
    prm = O.Params(linsys=1, cg_tol=1e-13, max_admm_iters=20)
    ref = O.solve(lp.A, lp.b, lp.c, prm, trace_iters=20)
    got = _first_iterates_gpu(abip, A, lp.b, lp.c, 20, cg_tol=1e-13)
    for k in range(20):
        assert _rel(got[k], ref.trace[k]) <= ITER_TOL, (k, _rel(got[k], ref.trace[k]))


def test_pcg_first_20_iterates_sparse(abip):
    lp = W.planted_sparse(300, seed=W.seed_for(W.SPARSE_PLANTED, 20))
    prm = O.Params(linsys=1, cg_tol=1e-13, max_admm_iters=20)
    ref = O.solve(lp.A.to_scipy(), lp.b, lp.c, prm, trace_iters=20)
    s = abip.Solver(lp.A, lp.b, lp.c, cg_tol=1e-13, max_admm_iters=20)
    s.solve()
    assert _rel(s.stacked_state(), ref.trace[-1]) <= ITER_TOL


def test_pcg_planted_end_to_end(abip):
    lp = W.planted_dense()
    A = W.dense_to_csr(lp.A)
    ref = O.solve(lp.A, lp.b, lp.c, O.Params(linsys=1, cg_tol=1e-10))
    s = abip.Solver(A, lp.b, lp.c, cg_tol=1e-10)
    info, x, y, sv = s.solve()
    _check_end(info, ref, lp)


def test_pcg_sparse_end_to_end(abip, oracle_memo):
    lp = W.planted_sparse(80, seed=W.seed_for(W.SPARSE_PLANTED, 10))
    ref = oracle_memo(("sparse", 80, 10), lambda: O.solve(lp.A.to_scipy(), lp.b, lp.c, O.Params(linsys=1, cg_tol=1e-10)))
    s = abip.Solver(lp.A, lp.b, lp.c, cg_tol=1e-10)
    info, x, y, sv = s.solve()
    _check_end(info, ref, lp)


def test_pcg_infeasible_status(abip):
    lp = W.infeasible_twin()
    ref = O.solve(lp.A, lp.b, lp.c, O.Params(linsys=1))
    s = abip.Solver(W.dense_to_csr(lp.A), lp.b, lp.c)
    info, *_ = s.solve()
    assert info["status"] == ref.status == O.PRIMAL_INFEASIBLE


def test_device_outputs_match_host_outputs(abip):
    lp = W.planted_dense(20, 45, seed=9)
    s = abip.Solver(W.dense_to_csr(lp.A), lp.b, lp.c)
    info, x, y, sv = s.solve()
    info2, xd, yd, sd = s.solve(device_out=True)
    assert info2["admm_iters"] == info["admm_iters"]
    assert np.array_equal(xd.cpu().numpy(), x) and np.array_equal(yd.cpu().numpy(), y)


# --- batched dense path ------------------------------------------------------

def test_batch_uneven_matches_single(abip):
    lps = [W.planted_dense(m, n, seed=W.seed_for(W.BATCH_UNEVEN, k)) for k, (m, n) in
           enumerate([(5, 12), (17, 40), (33, 99), (9, 9 * 3), (40, 150)])]
    lps.append(W.infeasible_twin(12, 25, seed=W.seed_for(W.BATCH_UNEVEN, 99)))
    infos, xs, ys, ss = abip.abip_solve_batch([l.A for l in lps], [l.b for l in lps], [l.c for l in lps])
    for lp, info, x in zip(lps, infos, xs):
        ref = O.solve(lp.A, lp.b, lp.c)
        _check_end(info, ref)


def test_batch_mixed_precision_matches_oracle(abip):
    """FP32 iterates with FP64 termination decisions: same status as the FP64 oracle and
    final relative residuals within 1e-6 (recomputed in FP64 on the device), objective
    within 1e-5."""
    lps = W.batch_uneven(count=10, infeasible_frac=0.3, m_lo=16, m_hi=48, seed=W.seed_for(W.BATCH_UNEVEN, 7))
    prm = abip.default_params(precision=abip.ABIP_PREC_MIXED)
    infos, xs, ys, ss = abip.abip_solve_batch([l.A for l in lps], [l.b for l in lps], [l.c for l in lps], prm)
    for lp, info, x in zip(lps, infos, xs):
        ref = O.solve(lp.A, lp.b, lp.c)
        assert info["status"] == ref.status, (lp.meta, info["status"], ref.status)
        if ref.status == O.OPTIMAL:
            assert max(info["pres"], info["dres"], info["dgap"]) <= 1e-6
            assert abs(info["obj"] - ref.obj) <= OBJ_TOL * max(1.0, abs(ref.obj))
            # independent FP64 residual of the returned candidate on the host
            assert np.linalg.norm(lp.A @ x - lp.b) <= 2e-6 * (1 + np.linalg.norm(lp.b))


def test_batch_fp64_and_mixed_agree_with_single(abip):
    lp = W.planted_dense_f32(40, 110, seed=W.seed_for(W.BATCH_UNEVEN, 11))
    s = abip.Solver(lp.A, lp.b, lp.c, precision=abip.ABIP_PREC_MIXED)
    info, *_ = s.solve()
    ref = O.solve(lp.A, lp.b, lp.c)
    assert info["status"] == ref.status == O.OPTIMAL
    assert abs(info["obj"] - ref.obj) <= OBJ_TOL * max(1.0, abs(ref.obj))


def test_set_state_resumes_the_iteration(abip):
    """get_state after k updates, set_state on a fresh handle and k more updates give the
    state after 2k updates (dense path: the projection has no PCG warm start)."""
    lp = W.planted_dense()
    a = abip.Solver(lp.A, lp.b, lp.c, max_admm_iters=30)
    a.solve()
    s30 = a.state()
    b = abip.Solver(lp.A, lp.b, lp.c, max_admm_iters=60)
    b.solve()
    c = abip.Solver(lp.A, lp.b, lp.c, max_admm_iters=30)
    c.set_state(s30)
    c.solve()
    assert _rel(c.state(), b.state()) <= 1e-13
    ref = O.solve(lp.A, lp.b, lp.c, O.Params(max_admm_iters=60), trace_iters=60)
    assert _rel(c.stacked_state(), ref.trace[-1]) <= ITER_TOL
    bad = s30.copy()
    bad[lp.m] = -1.0                       # x_0 < 0 is rejected
    with pytest.raises(abip.AbipError):
        c.set_state(bad)
