"""The checkpointed unrolled backward (oracle/unrolled.py) against the implicit-
differentiation gradient of the central point (oracle.central_point_grad): two routes to
the same derivative that share no arithmetic -- reverse mode through thousands of inner
iterations of Algorithm 2 with a dense (I + Q)^{-1}, against one transposed solve with the
Jacobian of system HSD-log-kkt at its Newton-polished root (Sec. 3.2, Theorem 3.1).
"""
import numpy as np
import pytest

from oracle import abip_oracle as O
from paper_1805_12344_gb300 import workloads as W

torch = pytest.importorskip("torch")
from oracle.unrolled import unrolled_grad  # noqa: E402


def _rel(a, ref):
    return np.abs(a - ref).max() / np.abs(ref).max()


def _case(lp, mu, seed=1):
    xt = lp.meta.get("x_target")
    if xt is None:
        xt = np.random.default_rng(seed).standard_normal(lp.A.shape[1])
    f = lambda xs: 2.0 * (xs - xt)
    ref = O.central_point_grad(lp.A, lp.b, lp.c, mu, f)
    start = {k: ref["point"][k] for k in ("y", "x", "tau", "theta", "s", "kappa")}
    return f, ref, start


@pytest.mark.parametrize("name,lp", [("l1_svm_3x8", W.l1_svm(d=3, N=8, seed=5)),
                                     ("planted_6x14", W.planted_dense(6, 14, seed=7))])
def test_unrolled_gradient_matches_the_implicit_gradient(name, lp):
    """At mu = 1e-2, 2000 iterations from the central point put the unrolled gradient within
    1e-9 of the implicit one on every entry block (the gap falls geometrically with the
    contraction factor of the iteration; measured ~5e-13)."""
    mu = 1e-2
    f, ref, start = _case(lp, mu)
    u = unrolled_grad(lp.A, lp.b, lp.c, mu, f, start, iters=2000, segment=100)
    assert u["change"] <= 1e-12                  # the start is the fixed point of the iteration
    assert np.allclose(u["xstar"], ref["xstar"], rtol=0, atol=1e-12 * np.abs(ref["xstar"]).max())
    for key in ("dA", "db", "dc"):
        assert _rel(u[key], ref[key]) <= 1e-9, (name, key, _rel(u[key], ref[key]))


def test_unrolled_gap_shrinks_geometrically_with_depth():
    """At mu = 1e-3 the iteration contracts more slowly: the gap to the implicit gradient
    falls by a roughly constant factor per added block of iterations."""
    lp = W.l1_svm(d=3, N=8, seed=5)
    mu = 1e-3
    f, ref, start = _case(lp, mu)
    gaps = [_rel(unrolled_grad(lp.A, lp.b, lp.c, mu, f, start, iters=K)["dc"], ref["dc"]) for K in (1000, 2000, 3000)]
    assert gaps[0] > gaps[1] > gaps[2]
    r1, r2 = gaps[1] / gaps[0], gaps[2] / gaps[1]
    assert r1 < 0.5 and r2 < 0.5 and 0.3 < r2 / r1 < 3.0, gaps


def test_checkpoint_segments_do_not_change_the_gradient():
    """Recomputing segments in the backward pass gives the gradient of the uncheckpointed
    run (one segment) to rounding."""
    lp = W.planted_dense(6, 14, seed=7)
    f, ref, start = _case(lp, 1e-2)
    a = unrolled_grad(lp.A, lp.b, lp.c, 1e-2, f, start, iters=300, segment=300)
    b = unrolled_grad(lp.A, lp.b, lp.c, 1e-2, f, start, iters=300, segment=37)
    for key in ("dA", "db", "dc"):
        assert _rel(b[key], a[key]) <= 1e-13


def test_unrolled_from_a_displaced_start_converges_to_the_same_gradient():
    """The limit does not depend on the start: from the central point at 2 mu (so the first
    iterations move the iterate), the gradient after enough iterations is the implicit one."""
    lp = W.l1_svm(d=3, N=8, seed=5)
    mu = 1e-2
    f, ref, _ = _case(lp, mu)
    far = O.central_point(lp.A, lp.b, lp.c, 2 * mu)
    start = {k: far[k] for k in ("y", "x", "tau", "theta", "s", "kappa")}
    u = unrolled_grad(lp.A, lp.b, lp.c, mu, f, start, iters=3000, segment=250)
    for key in ("dA", "db", "dc"):
        assert _rel(u[key], ref[key]) <= 1e-8, (key, _rel(u[key], ref[key]))
