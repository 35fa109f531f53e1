"""GPU parity of the Barzilai-Borwein choice of beta (Sec. 4.3; reading B5) on the dense
Cholesky path in FP64 (abip_params.bb_beta = 1) against the oracle's bb_select.

The selection runs from the second outer iteration on (reading B7).  The LPs cover every
branch with genuine curvature (each decision clears its threshold by 0.02 or more, so
rounding cannot flip it): basis pursuit 32 x 128 (estimates far from beta: five redos,
then the beta that made the state), an L1-SVM with 16 samples (two redos, then the
average), the infeasible twin (a redo, then keep), the 20 x 60 planted LP (keep).  Bars:
the raw state after a capped number of updates (trial updates included) within 1e-10
relative, the last beta within 1e-10 relative; end to end the same status, objective
within 1e-5 relative.
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


MOVING = ["basis_pursuit32x128", "svm16", "twin10x20"]


def _lps():
    sb = W.basis_pursuit(32, 128, batch=1, seed=7)
    d = W.planted_dense(20, 60, seed=23)
    t = W.infeasible_twin()
    sv = W.l1_svm(d=4, N=16, seed=3)
    return {"dense20x60": (d.A, d.b, d.c), "basis_pursuit32x128": (sb.A, sb.bs[0], sb.cs[0]),
            "twin10x20": (t.A, t.b, t.c), "svm16": (sv.A, sv.b, sv.c)}


def _stacked_raw(r):
    raw = r.raw
    return np.concatenate([raw["y"], raw["x"], [raw["tau"], raw["theta"]], raw["s"], [raw["kappa"]]])


@pytest.mark.parametrize("name", MOVING + ["dense20x60"])
@pytest.mark.parametrize("cap", [1, 2, 3, 57, 400, 1500])
def test_bb_state_after_capped_updates(abip, name, cap):
    A, b, c = _lps()[name]
    ref = O.solve(A, b, c, O.Params(bb_beta=True, max_admm_iters=cap))
    s = abip.Solver(A, b, c, bb_beta=1, max_admm_iters=cap)
    info, *_ = s.solve()
    assert info["admm_iters"] == ref.admm_iters
    assert info["status"] == ref.status
    got = s.stacked_state()
    rel = np.linalg.norm(got - _stacked_raw(ref)) / np.linalg.norm(_stacked_raw(ref))
    assert rel <= ITER_TOL, rel
    last = ref.raw["betas"][-1] if ref.raw["betas"] else 1.0   # cap 1: no room for a selection
    assert abs(info["beta"] - last) <= ITER_TOL * last


@pytest.mark.parametrize("name", MOVING)
def test_bb_end_to_end(abip, name):
    A, b, c = _lps()[name]
    ref = O.solve(A, b, c, O.Params(bb_beta=True))
    assert ref.raw["betas"][-1] != 1.0
    s = abip.Solver(A, b, c, bb_beta=1)
    info, x, y, sv = s.solve()
    assert info["status"] == ref.status
    assert abs(info["admm_iters"] - ref.admm_iters) <= 0.005 * ref.admm_iters + 2
    assert abs(info["beta"] - ref.raw["betas"][-1]) <= 1e-8 * ref.raw["betas"][-1]
    if ref.status == O.OPTIMAL:
        assert max(info["pres"], info["dres"], info["dgap"]) <= 1e-6
        assert abs(info["obj"] - ref.obj) <= OBJ_TOL * max(1.0, abs(ref.obj))


def test_bb_batch_matches_single(abip):
    """abip_solve_batch with bb_beta: every instance selects its own beta."""
    lps = _lps()
    names = list(lps)
    prm = abip.default_params(bb_beta=1)
    infos, xs, ys, ss = abip.abip_solve_batch([lps[k][0] for k in names], [lps[k][1] for k in names],
                                              [lps[k][2] for k in names], prm)
    for k, name in enumerate(names):
        single, *_ = abip.Solver(*lps[name], bb_beta=1).solve()
        assert infos[k]["status"] == single["status"]
        assert infos[k]["admm_iters"] == single["admm_iters"]
        assert infos[k]["beta"] == single["beta"]


def test_bb_refused_where_not_provided(abip):
    d = W.planted_dense(20, 60, seed=23)
    with pytest.raises(abip.AbipError) as e:
        abip.Solver(d.A, d.b, d.c, bb_beta=1, precision=abip.ABIP_PREC_MIXED)
    assert e.value.code == abip.ABIP_E_UNSUPPORTED
    with pytest.raises(abip.AbipError) as e:
        abip.Solver(W.dense_to_csr(d.A), d.b, d.c, bb_beta=1)
    assert e.value.code == abip.ABIP_E_UNSUPPORTED
