"""GPU parity of the sparse direct projection (linsys = ABIP_LINSYS_SPARSE_LDL, Sec. 4.4):
the LDL^T factor of the quasi-definite system, formed and applied on the GPU, against the
FP64 oracle with its exact projection (dense Cholesky of G = I + A A^T).

Bars: FP64 iterates within 1e-10 relative for the first 20 ADMM updates; at the end
identical status, relative residuals <= 1e-6, objective within 1e-5 relative of the
oracle's and of the planted optimum.
"""
import numpy as np
import pytest

from oracle import abip_oracle as O
from paper_1805_12344_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ITER_TOL = 1e-10
OBJ_TOL = 1e-5
LDL = 2


@pytest.fixture(scope="module")
def abip():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1805_12344_gb300 import build, abip as _abip
    build.build()
    _abip.lib()
    assert _abip.ABIP_LINSYS_SPARSE_LDL == LDL
    return _abip


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _check_end(info, ref, lp=None):
    assert info["status"] == ref.status
    assert info["cg_iters"] == 0                       # no PCG on this path
    if ref.status == O.OPTIMAL:
        assert max(info["pres"], info["dres"], info["dgap"]) <= 1e-6
        assert abs(info["obj"] - ref.obj) <= OBJ_TOL * max(1.0, abs(ref.obj))
        if lp is not None and lp.p_star is not None:
            assert abs(info["obj"] - lp.p_star) <= OBJ_TOL * max(1.0, abs(lp.p_star))


def test_ldl_first_20_iterates_grid_flow(abip):
    """Every one of the first 20 iterates (one solve per count, so setup, factorisation
    and every sweep epoch run each time) on the 6 x 6 grid flow LP."""
    lp = W.grid_flow(6)
    A = lp.A.to_scipy()
    ref = O.solve(A, lp.b, lp.c, O.Params(linsys=0, max_admm_iters=20), trace_iters=20)
    for k in range(1, 21):
        s = abip.Solver(lp.A, lp.b, lp.c, linsys=LDL, max_admm_iters=k)
        info, *_ = s.solve()
        assert info["admm_iters"] == k
        got = s.stacked_state()
        s.close()
        assert _rel(got, ref.trace[k - 1]) <= ITER_TOL, (k, _rel(got, ref.trace[k - 1]))


def test_ldl_iterates_random_sparse(abip):
    """Random sparse [R I] (heavy fill under any order) and a second solve on the same
    handle, which must continue the flag epochs of the first."""
    lp = W.planted_sparse(300, seed=W.seed_for(W.SPARSE_PLANTED, 20))
    ref = O.solve(lp.A.to_scipy(), lp.b, lp.c, O.Params(linsys=0, max_admm_iters=20), trace_iters=20)
    s = abip.Solver(lp.A, lp.b, lp.c, linsys=LDL, max_admm_iters=20)
    s.solve()
    first = s.stacked_state()
    assert _rel(first, ref.trace[-1]) <= ITER_TOL
    s.solve()
    assert _rel(s.stacked_state(), first) <= 1e-13


def test_ldl_grid_flow_end_to_end(abip, oracle_memo):
    lp = W.grid_flow(6)
    ref = oracle_memo(("grid_flow", 6), lambda: O.solve(lp.A.to_scipy(), lp.b, lp.c, O.Params(linsys=0)))
    s = abip.Solver(lp.A, lp.b, lp.c, linsys=LDL)
    info, x, y, sv = s.solve()
    _check_end(info, ref, lp)
    Ad = lp.A.to_dense()
    assert np.linalg.norm(Ad @ x - lp.b) <= 1e-6 * (1 + np.linalg.norm(lp.b)) * 1.01
    assert np.linalg.norm(Ad.T @ y + sv - lp.c) <= 1e-6 * (1 + np.linalg.norm(lp.c)) * 1.01
    assert np.all(x >= 0) and np.all(sv >= 0)


def test_ldl_dense_input_end_to_end(abip):
    """A dense A read as CSR: K's graph is complete bipartite, so the ordering soon reaches
    its complete-graph tail."""
    lp = W.planted_dense()
    ref = O.solve(lp.A, lp.b, lp.c)
    s = abip.Solver(lp.A, lp.b, lp.c, linsys=LDL)
    info, *_ = s.solve()
    _check_end(info, ref, lp)


@pytest.mark.parametrize("make", [W.infeasible_twin, W.dual_infeasible])
def test_ldl_infeasible_status(abip, make):
    lp = make()
    ref = O.solve(lp.A, lp.b, lp.c)
    s = abip.Solver(W.dense_to_csr(lp.A), lp.b, lp.c, linsys=LDL)
    info, *_ = s.solve()
    assert info["status"] == ref.status


def test_ldl_wait_limit_returns_timeout(abip):
    """A 1 ns wait limit: the barrier and flag waits give up, the kernel returns, and the
    call reports ABIP_E_TIMEOUT; the context stays usable."""
    lp = W.grid_flow(6)
    with pytest.raises(abip.AbipError) as e:
        abip.Solver(lp.A, lp.b, lp.c, linsys=LDL, barrier_limit_ns=1).solve()
    assert e.value.code == abip.ABIP_E_TIMEOUT
    s = abip.Solver(lp.A, lp.b, lp.c, linsys=LDL, max_admm_iters=5)
    info, *_ = s.solve()
    assert info["admm_iters"] == 5
