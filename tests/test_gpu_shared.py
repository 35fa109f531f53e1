"""GPU parity of the shared-A batch path (abip_solve_batch_shared) against the FP64 oracle.

Bars as for the other paths: FP64 iterates within 1e-10 relative for the first 20
ADMM updates; at the end identical status, relative residuals <= 1e-6 and the
objective within 1e-5 relative of the oracle's.
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


def _raw(info, x, y, s):
    """(y, x, tau, theta, s, kappa) from the outputs of an unfinished solve (scaled by 1/tau)."""
    tau = info["tau"]
    return np.concatenate([y * tau, x * tau, [tau, info["theta"]], s * tau, [info["kappa"]]])


def _shared_planted(m, n, count, seed):
    """One A (row 0 positive, last column zero) with planted feasible instances, plus one
    primal-infeasible (b_0 = -1) and one dual-infeasible (cost -1 on the zero column)."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n))
    A[0] = np.abs(A[0]) + 0.1
    A[:, -1] = 0.0
    bs, cs, expect = [], [], []
    for _ in range(count):
        k = max(1, int(0.3 * (n - 1)))
        perm = rng.permutation(n - 1)
        x0 = np.zeros(n)
        s0 = np.zeros(n)
        x0[perm[:k]] = rng.uniform(0.5, 2.0, k)
        s0[perm[k:]] = rng.uniform(0.5, 2.0, n - 1 - k)
        s0[-1] = 1.0
        y0 = rng.standard_normal(m)
        bs.append(A @ x0)
        cs.append(A.T @ y0 + s0)
        expect.append(O.OPTIMAL)
    b = bs[0].copy()
    b[0] = -1.0
    bs.append(b)
    cs.append(cs[0].copy())
    expect.append(O.PRIMAL_INFEASIBLE)
    c = cs[1].copy()
    c[-1] = -1.0
    bs.append(bs[1].copy())
    cs.append(c)
    expect.append(O.DUAL_INFEASIBLE)
    return A, bs, cs, expect


def test_shared_first_20_iterates(abip):
    sb = W.basis_pursuit(24, 64, batch=3, seed=3)
    refs = [O.solve(sb.A, b, c, O.Params(max_admm_iters=20), trace_iters=20) for b, c in zip(sb.bs, sb.cs)]
    for k in range(1, 21):
        prm = abip.default_params(max_admm_iters=k)
        infos, xs, ys, ss = abip.abip_solve_batch_shared(sb.A, sb.bs, sb.cs, prm)
        for i in range(3):
            assert infos[i]["admm_iters"] == k
            got = _raw(infos[i], xs[i], ys[i], ss[i])
            assert _rel(got, refs[i].trace[k - 1]) <= ITER_TOL, (k, i, _rel(got, refs[i].trace[k - 1]))


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_shared_basis_pursuit_end_to_end(abip, precision):
    sb = W.basis_pursuit(32, 128, batch=4, seed=5)
    prec = abip.ABIP_PREC_MIXED if precision == "mixed" else abip.ABIP_PREC_F64
    infos, xs, ys, ss = abip.abip_solve_batch_shared(sb.A, sb.bs, sb.cs, abip.default_params(precision=prec))
    for k in range(4):
        ref = O.solve(sb.A, sb.bs[k], sb.cs[k])
        f = infos[k]
        assert f["status"] == ref.status == O.OPTIMAL
        assert max(f["pres"], f["dres"], f["dgap"]) <= 1e-6
        assert abs(f["obj"] - ref.obj) <= OBJ_TOL * max(1.0, abs(ref.obj))
        # independent FP64 residuals of the returned candidate
        assert np.linalg.norm(sb.A @ xs[k] - sb.bs[k]) <= 1e-6 * (1 + np.linalg.norm(sb.bs[k])) * 1.01
        # l1 recovery of the planted sparse vector (objective bound ||x_true||_1)
        xt = sb.meta["x_true"][k]
        assert f["obj"] <= np.abs(xt).sum() * (1 + 1e-5)


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_shared_statuses(abip, precision):
    A, bs, cs, expect = _shared_planted(12, 30, 4, seed=8)
    prec = abip.ABIP_PREC_MIXED if precision == "mixed" else abip.ABIP_PREC_F64
    infos, xs, ys, ss = abip.abip_solve_batch_shared(A, bs, cs, abip.default_params(precision=prec))
    for k, want in enumerate(expect):
        ref = O.solve(A, bs[k], cs[k])
        assert ref.status == want
        assert infos[k]["status"] == want, (k, infos[k]["status_name"])
        if want == O.OPTIMAL:
            assert abs(infos[k]["obj"] - ref.obj) <= OBJ_TOL * max(1.0, abs(ref.obj))


def test_shared_matches_per_instance_batch(abip):
    """Same instances through the per-CTA dense batch: same algorithm, same update counts."""
    A, bs, cs, _ = _shared_planted(10, 26, 3, seed=4)
    prm = abip.default_params()
    i1, x1, _, _ = abip.abip_solve_batch_shared(A, bs, cs, prm)
    i2, x2, _, _ = abip.abip_solve_batch([A] * len(bs), bs, cs, prm)
    for k in range(len(bs)):
        assert i1[k]["status"] == i2[k]["status"]
        assert i1[k]["admm_iters"] == i2[k]["admm_iters"]
        assert _rel(x1[k], x2[k]) <= 1e-8


def test_shared_chunks_past_64(abip):
    A, bs, cs, expect = _shared_planted(5, 12, 64, seed=6)
    infos, xs, _, _ = abip.abip_solve_batch_shared(A, bs, cs, abip.default_params())
    assert len(infos) == 66
    for k, want in enumerate(expect):
        assert infos[k]["status"] == want
    for k in (0, 33, 63):
        ref = O.solve(A, bs[k], cs[k])
        assert abs(infos[k]["obj"] - ref.obj) <= OBJ_TOL * max(1.0, abs(ref.obj))


@pytest.mark.parametrize("m,nd,bf16", [(128, 256, False), (256, 1024, False), (128, 256, True)])
def test_shared_tensor_cores_end_to_end(abip, m, nd, bf16):
    """ABIP_PREC_MIXED_BF16: the products with A run on tcgen05, the changes split in three
    bfloat16 terms and A in three (float32 D, as the basis-pursuit workload draws it) or in
    one (D rounded to bfloat16); same bars as the other paths, plus the l1 bound
    ||x_true||_1 (x_true is feasible).  The oracle solves three of the sixteen instances."""
    sb = W.basis_pursuit(m, nd, batch=16, seed=9 + m, bf16=bf16)
    prm = abip.default_params(precision=abip.ABIP_PREC_MIXED_BF16)
    infos, xs, ys, ss = abip.abip_solve_batch_shared(sb.A, sb.bs, sb.cs, prm)
    for k in range(16):
        f = infos[k]
        assert f["status"] == O.OPTIMAL, (k, f["status_name"])
        assert max(f["pres"], f["dres"], f["dgap"]) <= 1e-6
        assert np.linalg.norm(sb.A @ xs[k] - sb.bs[k]) <= 1e-6 * (1 + np.linalg.norm(sb.bs[k])) * 1.01
        assert np.linalg.norm(sb.A.T @ ys[k] + ss[k] - sb.cs[k]) <= 1e-6 * (1 + np.linalg.norm(sb.cs[k])) * 1.01
        assert f["obj"] <= np.abs(sb.meta["x_true"][k]).sum() * (1 + 1e-5)
    for k in (0, 7, 15):
        ref = O.solve(sb.A, sb.bs[k], sb.cs[k])
        assert ref.status == O.OPTIMAL
        assert abs(infos[k]["obj"] - ref.obj) <= OBJ_TOL * max(1.0, abs(ref.obj))


def test_shared_tensor_cores_refuse_A_beyond_fp32(abip):
    """The tensor-core path holds A as bfloat16 terms of its FP32 value: an entry beyond
    the FP32 range cannot be represented and is refused."""
    A, bs, cs, _ = _shared_planted(128, 256, 16, seed=3)
    A = A.copy()
    A[5, 7] = 1e39
    with pytest.raises(abip.AbipError) as e:
        abip.abip_solve_batch_shared(A, bs, cs, abip.default_params(precision=abip.ABIP_PREC_MIXED_BF16))
    assert e.value.code == abip.ABIP_E_INVALID_ARG


def test_shared_tensor_cores_general_A_matches_fp32_products(abip):
    """A general float64 A (not exact in FP32): the tensor-core path (A in three bfloat16
    terms of its FP32 rounding) and the FP32 SIMT path reach the same statuses and optima."""
    A, bs, cs, expect = _shared_planted(128, 256, 14, seed=4)   # 16 instances: the tensor-core shape
    assert len(bs) == 16
    p1 = abip.default_params(precision=abip.ABIP_PREC_MIXED_BF16)
    p2 = abip.default_params(precision=abip.ABIP_PREC_MIXED)
    i1, *_ = abip.abip_solve_batch_shared(A, bs, cs, p1)
    i2, *_ = abip.abip_solve_batch_shared(A, bs, cs, p2)
    for k in range(16):
        assert i1[k]["status"] == i2[k]["status"] == expect[k]
        if expect[k] == O.OPTIMAL:
            assert abs(i1[k]["obj"] - i2[k]["obj"]) <= OBJ_TOL * max(1.0, abs(i2[k]["obj"]))
