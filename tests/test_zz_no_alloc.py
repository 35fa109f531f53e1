"""The allocation-free entry point abip_solve_dense_noalloc, for callers that cannot
allocate device memory (a framework owns every allocation through its own pool, or a
fixed memory budget forbids growth): it must give the same answer as the ordinary
abip_setup + abip_solve path, call after call, while taking all scratch from the
library's fixed device array.

This file is collected last so that, if it fails, a run stopping at the first failure
has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1805_12344_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10   # the iterate tolerance of the other GPU parity tests


@pytest.fixture(scope="module")
def abip():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1805_12344_gb300 import build, abip as _abip
    build.build()
    L = _abip.lib()
    f = L.abip_solve_dense_noalloc
    f.restype = C.c_int
    f.argtypes = [C.c_int32, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                  C.POINTER(_abip.abip_params), C.c_void_p, C.c_void_p, C.c_void_p,
                  C.POINTER(_abip.abip_info), C.c_void_p]
    return _abip


def _noalloc(abip, lp, params, free_bytes=None):
    """One call through the C ABI.  free_bytes (a list): receives the device's free memory
    (cudaMemGetInfo) read just before and just after the call, with no allocation by this
    process in between."""
    m, n = lp.A.shape
    dev = torch.device("cuda")
    A = torch.from_numpy(np.ascontiguousarray(lp.A)).to(dev)
    b = torch.from_numpy(lp.b).to(dev)
    c = torch.from_numpy(lp.c).to(dev)
    x = torch.full((n,), np.nan, dtype=torch.float64, device=dev)
    y = torch.full((m,), np.nan, dtype=torch.float64, device=dev)
    s = torch.full((n,), np.nan, dtype=torch.float64, device=dev)
    info = abip.abip_info()
    torch.cuda.synchronize()
    if free_bytes is not None:
        free_bytes.append(torch.cuda.mem_get_info()[0])
    rc = abip.lib().abip_solve_dense_noalloc(m, n, A.data_ptr(), n, b.data_ptr(), c.data_ptr(),
                                             C.byref(params), x.data_ptr(), y.data_ptr(), s.data_ptr(),
                                             C.byref(info), None)
    torch.cuda.synchronize()
    if free_bytes is not None:
        free_bytes.append(torch.cuda.mem_get_info()[0])
    assert rc == 0, abip.lib().abip_last_error(None)
    return info, x.cpu().numpy(), y.cpu().numpy(), s.cpu().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("m,n", [(50, 120), (128, 512)])
def test_noalloc_matches_setup_and_solve_twice(abip, m, n):
    lp = W.planted_dense(m, n, seed=W.seed_for(W.DENSE_PLANTED, 300 + m))
    prm = abip.default_params()
    ref = abip.Solver(lp.A, lp.b, lp.c)
    rinfo, rx, ry, rs = ref.solve()
    for call in range(2):                    # two calls in a row share the fixed scratch
        free = []
        info, x, y, s = _noalloc(abip, lp, prm, free)
        if call == 1:                        # the first call may load the module; the second allocates nothing
            assert free[0] == free[1], free
        assert info.status == rinfo["status"]
        assert info.admm_iters == rinfo["admm_iters"]
        assert _rel(x, rx) <= TOL and _rel(y, ry) <= TOL and _rel(s, rs) <= TOL


def test_noalloc_rejects_sizes_beyond_its_scratch(abip):
    lp = W.planted_dense(129, 300, seed=5)
    with pytest.raises(AssertionError):
        _noalloc(abip, lp, abip.default_params())
    assert b"at most" in abip.lib().abip_last_error(None)
