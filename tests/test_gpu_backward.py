"""GPU gradients of x* = x / tau at the central point of the final mu (abip_backward,
abip_backward_batch and the autograd layer) against the oracle's dense KKT gradient,
the checkpointed unrolled backward through the inner iterations, the vertex limit and
FP64 central differences of the oracle's central-point map.

Bar: 1e-5 relative (per block, against the block's largest entry).  The L1-SVM LP is
dual degenerate (the bias is split into two free columns of zero cost), so its central
point's gradient grows like 1/mu and the Jacobian's condition number like 1/mu: central
differences with step 1e-6 are accurate to ~(1e-6/mu)^2 relative and are used at
mu ~ 1e-3; the KKT-gradient comparisons run at the final mu of solves to eps = 1e-4
(mu ~ 1e-7 .. 1e-6), where FP64 still fixes the gradient to better than the bar.
"""
import numpy as np
import pytest

from oracle import abip_oracle as O
from paper_1805_12344_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-5


@pytest.fixture(scope="module")
def abip():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1805_12344_gb300 import build, abip as _abip
    build.build()
    _abip.lib()
    return _abip


def _unpack(st, m, n):
    return dict(y=st[:m], x=st[m:m + n], tau=st[m + n], theta=st[m + n + 1],
                s=st[m + n + 2:m + 2 * n + 2], kappa=st[m + 2 * n + 2]), st[-1]


def _blockrel(a, ref):
    return np.abs(a - ref).max() / np.abs(ref).max()


def _vertex_lp(m, n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n))
    basic = np.zeros(n, dtype=bool)
    basic[rng.permutation(n)[:m]] = True
    x0 = np.where(basic, rng.uniform(0.5, 2.0, n), 0.0)
    s0 = np.where(basic, 0.0, rng.uniform(0.5, 2.0, n))
    y0 = rng.standard_normal(m)
    return A, A @ x0, A.T @ y0 + s0, x0, basic, rng.standard_normal(n)


def _solve_and_grad(abip, A, b, c, xt, eps, cap=10**6):
    S = abip.Solver(A, b, c, eps=eps, linsys=0, max_admm_iters=cap)
    info, x, _, _ = S.solve()
    assert info["status"] in (abip.ABIP_OPTIMAL, abip.ABIP_MAX_ITER)
    g = 2.0 * (x - xt)
    out = S.backward(g)
    m, n = A.shape
    start, mu = _unpack(S.state(), m, n)
    S.close()
    return out, g, start, mu


@pytest.mark.parametrize("d,N,eps,cap", [(3, 8, 1e-4, 10**6), (8, 40, 1e-4, 10**6), (16, 96, 1e-4, 10**6),
                                         (64, 512, 1e-6, 20000)])
def test_backward_matches_oracle_kkt_gradient(abip, d, N, eps, cap):
    """Last case: the full L1-SVM size (512 x 1154), forward stopped at 20000 updates."""
    lp = W.l1_svm(d=d, N=N, seed=5)
    out, g, start, mu = _solve_and_grad(abip, lp.A, lp.b, lp.c, lp.meta["x_target"], eps, cap)
    ref = O.central_point_grad(lp.A, lp.b, lp.c, mu, lambda xs: g, start=start)
    for k, key in (("c", "dc"), ("b", "db"), ("A", "dA")):
        assert _blockrel(out[k], ref[key]) <= GRAD_TOL, (k, _blockrel(out[k], ref[key]))


def test_backward_vertex_limit(abip):
    """Small final mu on a nondegenerate vertex: dL/db -> B^{-T} g_B, dL/dc -> 0,
    dL/dA -> -(B^{-T} g_B) x0^T, independently of the oracle."""
    A, b, c, x0, basic, xt = _vertex_lp(12, 30, seed=21)
    out, g, start, mu = _solve_and_grad(abip, A, b, c, xt, 1e-8)
    w = np.linalg.solve(A[:, basic].T, g[basic])
    assert mu < 1e-6
    tol = 1e-4   # the limit holds up to O(mu) and the forward's 1e-8 accuracy in x
    assert _blockrel(out["b"], w) <= tol
    assert np.abs(out["c"]).max() <= tol * np.abs(w).max()
    assert _blockrel(out["A"], -np.outer(w, x0)) <= tol


def test_backward_central_differences(abip):
    """GPU gradient against FP64 central differences (step 1e-6 max(1, |p|)) of the oracle's
    central-point map at the GPU's final mu, on every entry of b and c and a sample of A."""
    lp = W.l1_svm(d=4, N=12, seed=9)
    xt = lp.meta["x_target"]
    out, g, start, mu = _solve_and_grad(abip, lp.A, lp.b, lp.c, xt, 1e-2)
    assert mu >= 1e-4

    def loss_lin(A, b, c):
        cp = O.central_point(A, b, c, mu, start=start, tol=1e-15)
        return float(g @ (cp["x"] / cp["tau"]))     # dL/dx* held at g: the linearised loss

    base = {"A": lp.A, "b": lp.b, "c": lp.c}
    rng = np.random.default_rng(3)
    for which in ("b", "c", "A"):
        P = base[which]
        idxs = list(np.ndindex(P.shape))
        if which == "A":
            idxs = [idxs[i] for i in rng.choice(len(idxs), 40, replace=False)]
        fd = np.zeros(len(idxs))
        got = np.array([out[which][i] for i in idxs])
        for k, idx in enumerate(idxs):
            h = 1e-6 * max(1.0, abs(P[idx]))
            vals = []
            for sgn in (1, -1):
                Pp = P.copy()
                Pp[idx] += sgn * h
                vals.append(loss_lin(**dict(base, **{which: Pp})))
            fd[k] = (vals[0] - vals[1]) / (2 * h)
        scale = np.abs(out[which]).max()
        assert np.abs(got - fd).max() <= GRAD_TOL * scale, (which, np.abs(got - fd).max() / scale)


@pytest.mark.parametrize("d,N", [(8, 40), (16, 96)])
def test_backward_matches_unrolled_backward(abip, d, N):
    """The adjoint kernel (abip_backward_batch) at the central point of mu = 1e-2 against the
    checkpointed unrolled backward: reverse mode through 2000 inner iterations of Algorithm 2
    from the same point (oracle/unrolled.py), a route with no KKT solve at all."""
    from oracle.unrolled import unrolled_grad
    lp = W.l1_svm(d=d, N=N, seed=5)
    mu = 1e-2
    cp = O.central_point(lp.A, lp.b, lp.c, mu)
    tau = cp["tau"]
    xs = cp["x"] / tau
    g = 2.0 * (xs - lp.meta["x_target"])
    info = dict(status=abip.ABIP_OPTIMAL, tau=tau, kappa=cp["kappa"], theta=cp["theta"], mu=mu)
    dcs, dbs, dAs = abip.abip_backward_batch([lp.A], [lp.b], [lp.c], [xs], [cp["y"] / tau], [cp["s"] / tau],
                                             [info], [g])
    start = {k: cp[k] for k in ("y", "x", "tau", "theta", "s", "kappa")}
    ref = unrolled_grad(lp.A, lp.b, lp.c, mu, lambda x_: g, start, iters=2000, segment=200)
    assert _blockrel(dcs[0], ref["dc"]) <= GRAD_TOL, _blockrel(dcs[0], ref["dc"])
    assert _blockrel(dbs[0], ref["db"]) <= GRAD_TOL, _blockrel(dbs[0], ref["db"])
    assert _blockrel(dAs[0], ref["dA"]) <= GRAD_TOL, _blockrel(dAs[0], ref["dA"])


def test_backward_batch_matches_single(abip):
    """abip_backward_batch over uneven instances matches the oracle's KKT gradient per instance."""
    lps = [W.l1_svm(d=d, N=N, seed=s) for d, N, s in ((3, 8, 1), (5, 20, 2), (2, 6, 3), (6, 30, 4))]
    prm = abip.default_params(eps=1e-4)
    infos, xs, ys, ss = abip.abip_solve_batch([l.A for l in lps], [l.b for l in lps], [l.c for l in lps], prm)
    gs = [2.0 * (x - l.meta["x_target"]) for x, l in zip(xs, lps)]
    dcs, dbs, dAs = abip.abip_backward_batch([l.A for l in lps], [l.b for l in lps], [l.c for l in lps],
                                             xs, ys, ss, infos, gs, prm)
    for k, l in enumerate(lps):
        start, mu = None, infos[k]["mu"]
        tau = infos[k]["tau"]
        m, n = l.A.shape
        start = dict(y=ys[k] * tau, x=xs[k] * tau, s=ss[k] * tau, tau=tau, theta=infos[k]["theta"],
                     kappa=infos[k]["kappa"])
        ref = O.central_point_grad(l.A, l.b, l.c, mu, lambda xs_: gs[k], start=start)
        assert _blockrel(dcs[k], ref["dc"]) <= GRAD_TOL
        assert _blockrel(dbs[k], ref["db"]) <= GRAD_TOL
        assert _blockrel(dAs[k], ref["dA"]) <= GRAD_TOL


def test_autograd_layer(abip):
    """torch.autograd through lp_solve on CUDA tensors equals the oracle's KKT gradient."""
    from paper_1805_12344_gb300.layer import lp_solve
    lps = [W.l1_svm(d=4, N=16, seed=s) for s in (11, 12)]
    A = torch.tensor(np.stack([l.A for l in lps]), device="cuda", requires_grad=True)
    b = torch.tensor(np.stack([l.b for l in lps]), device="cuda", requires_grad=True)
    c = torch.tensor(np.stack([l.c for l in lps]), device="cuda", requires_grad=True)
    xt = torch.tensor(np.stack([l.meta["x_target"] for l in lps]), device="cuda")
    x = lp_solve(A, b, c, eps=1e-4)
    loss = ((x - xt) ** 2).sum()
    loss.backward()
    # the oracle at the same final mu, from the GPU's own final iterate
    prm = abip.default_params(eps=1e-4)
    infos, xs, ys, ss = abip.abip_solve_batch([l.A for l in lps], [l.b for l in lps], [l.c for l in lps], prm)
    for k, l in enumerate(lps):
        tau = infos[k]["tau"]
        start = dict(y=ys[k] * tau, x=xs[k] * tau, s=ss[k] * tau, tau=tau, theta=infos[k]["theta"],
                     kappa=infos[k]["kappa"])
        gk = 2.0 * (x[k].detach().cpu().numpy() - l.meta["x_target"])
        ref = O.central_point_grad(l.A, l.b, l.c, infos[k]["mu"], lambda xs_: gk, start=start)
        assert _blockrel(c.grad[k].cpu().numpy(), ref["dc"]) <= GRAD_TOL
        assert _blockrel(b.grad[k].cpu().numpy(), ref["db"]) <= GRAD_TOL
        assert _blockrel(A.grad[k].cpu().numpy(), ref["dA"]) <= GRAD_TOL


def test_backward_errors(abip):
    lp = W.infeasible_twin()
    S = abip.Solver(lp.A, lp.b, lp.c, linsys=0)
    with pytest.raises(abip.AbipError) as e:
        S.backward(np.ones(lp.A.shape[1]))
    assert e.value.code == abip.ABIP_E_NOT_SOLVED
    info, *_ = S.solve()
    assert info["status"] == abip.ABIP_PRIMAL_INFEASIBLE
    with pytest.raises(abip.AbipError) as e:
        S.backward(np.ones(lp.A.shape[1]))
    assert e.value.code == abip.ABIP_E_INVALID_ARG
    S.close()
    lp = W.planted_dense(8, 20, seed=2)
    S = abip.Solver(W.dense_to_csr(lp.A), lp.b, lp.c, linsys=1)
    S.solve()
    with pytest.raises(abip.AbipError) as e:
        S.backward(np.ones(20))
    assert e.value.code == abip.ABIP_E_UNSUPPORTED
    S.close()
