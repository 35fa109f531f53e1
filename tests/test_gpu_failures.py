"""Failure detection on the GPU without a GPU fault: every failure here is made on the
host (a parameter, an input magnitude) or is a device-side wait given a short limit that
returns an error status; the CUDA context stays usable afterwards.

* PCG cap: cg_max_iter = 1 cannot meet the PCG tolerance -> ABIP_E_NUMERICAL.
* Grid-barrier limit: barrier_limit_ns = 1 makes the first barrier wait of the persistent
  kernel run past its limit; every CTA leaves the kernel -> ABIP_E_TIMEOUT.
* Non-finite reduction: finite inputs whose sums overflow FP64 -> ABIP_E_NUMERICAL.
"""
import pytest

from paper_1805_12344_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abip():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1805_12344_gb300 import build, abip as _abip
    build.build()
    _abip.lib()
    return _abip


def _sparse():
    return W.planted_sparse(300, seed=W.seed_for(W.SPARSE_PLANTED, 20))


def _still_works(abip):
    lp = W.planted_dense(12, 30, seed=W.seed_for(W.DENSE_PLANTED, 100))
    info, *_ = abip.Solver(W.dense_to_csr(lp.A), lp.b, lp.c).solve()
    assert info["status"] == abip.ABIP_OPTIMAL


@pytest.mark.parametrize("precision", [0, 1])
def test_pcg_cap_reports_numerical(abip, precision):
    lp = _sparse()
    with pytest.raises(abip.AbipError) as ex:
        abip.Solver(lp.A, lp.b, lp.c, cg_max_iter=1, cg_tol=1e-13, precision=precision).solve()
    assert ex.value.code == abip.ABIP_E_NUMERICAL
    assert "PCG" in str(ex.value)
    _still_works(abip)


@pytest.mark.parametrize("precision", [0, 1])
def test_barrier_limit_reports_timeout(abip, precision):
    lp = _sparse()
    with pytest.raises(abip.AbipError) as ex:
        abip.Solver(lp.A, lp.b, lp.c, barrier_limit_ns=1, precision=precision).solve()
    assert ex.value.code == abip.ABIP_E_TIMEOUT
    assert "barrier" in str(ex.value)
    _still_works(abip)


@pytest.mark.parametrize("sparse", [False, True])
def test_overflowing_sums_report_numerical(abip, sparse):
    lp = W.planted_dense(20, 45, seed=9)
    c = lp.c * 1e160                  # finite, but ||c||^2 and the Schur complement overflow FP64
    A = W.dense_to_csr(lp.A) if sparse else lp.A
    with pytest.raises(abip.AbipError) as ex:
        abip.Solver(A, lp.b, c).solve()
    assert ex.value.code == abip.ABIP_E_NUMERICAL
    _still_works(abip)
