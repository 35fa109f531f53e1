"""C-ABI checks that need no GPU: the library builds and loads, exports every symbol
include/abip.h declares, and rejects bad arguments before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1805_12344_gb300 import build, abip
    build.build()
    return abip.lib()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "abip.h")).read()
    return sorted(set(re.findall(r"ABIP_API\s+[\w\s\*]+?\b(abip_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("abip_setup", "abip_solve", "abip_solve_batch", "abip_backward", "abip_default_params",
                 "abip_get_state", "abip_free", "abip_status_str", "abip_last_error"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_default_params(lib):
    from paper_1805_12344_gb300 import abip
    p = abip.default_params()
    assert p.beta == 1.0 and p.alpha == 1.8 and p.eps == 1e-6 and p.max_admm_iters == 10 ** 6
    assert 0 < p.gamma < 1
    assert lib.abip_default_params(None) == abip.ABIP_E_INVALID_ARG


def test_struct_layout_matches_header():
    """ctypes mirrors of the C structs have the sizes and field offsets the C compiler
    gives them (every field of every struct the boundary passes)."""
    from paper_1805_12344_gb300 import abip
    structs = [("abip_matrix", abip.abip_matrix), ("abip_params", abip.abip_params),
               ("abip_info", abip.abip_info), ("abip_presolve_info", abip.abip_presolve_info)]
    lines = []
    for cname, py in structs:
        lines.append('printf("%%zu\\n", sizeof(%s));' % cname)
        for f, _ in py._fields_:
            lines.append('printf("%%zu\\n", offsetof(%s, %s));' % (cname, f))
    code = ("#include <stdio.h>\n#include <stddef.h>\n#include \"abip.h\"\nint main(void){" + "".join(lines) +
            "return 0;}\n")
    import subprocess, tempfile
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.c")
        open(src, "w").write(code)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe])
        got = [int(v) for v in subprocess.check_output([exe]).split()]
    want = []
    for _, py in structs:
        want.append(C.sizeof(py))
        want += [getattr(py, f).offset for f, _ in py._fields_]
    assert got == want


def test_status_strings(lib):
    assert lib.abip_status_str(1) == b"optimal"
    assert lib.abip_status_str(2) == b"primal_infeasible"
    assert lib.abip_status_str(3) == b"dual_infeasible"
    assert lib.abip_status_str(4) == b"max_iter"
    assert lib.abip_version().startswith(b"abip")


def test_argument_errors_without_device(lib):
    from paper_1805_12344_gb300 import abip
    A = np.ones((2, 3))
    b = np.ones(2)
    c = np.ones(3)
    # NULL output handle
    M, keep = abip._matrix(A)
    assert lib.abip_setup(C.byref(M), b.ctypes.data, c.ctypes.data, None, None) == abip.ABIP_E_INVALID_ARG
    # n < m
    with pytest.raises(abip.AbipError) as e:
        abip.abip_setup(np.ones((3, 2)), np.ones(3), np.ones(2))
    assert e.value.code == abip.ABIP_E_DIM
    # non-finite data
    with pytest.raises(abip.AbipError) as e:
        abip.abip_setup(A, np.array([1.0, np.nan]), c)
    assert e.value.code == abip.ABIP_E_INVALID_ARG
    # bad parameters
    with pytest.raises(abip.AbipError) as e:
        abip.abip_setup(A, b, c, abip.default_params(gamma=1.5))
    assert e.value.code == abip.ABIP_E_INVALID_ARG
    with pytest.raises(abip.AbipError) as e:
        abip.abip_setup(A, b, c, abip.default_params(alpha=2.5))
    assert e.value.code == abip.ABIP_E_INVALID_ARG
    assert b"gamma" in lib.abip_last_error(None) or b"alpha" in lib.abip_last_error(None)
    # malformed CSR
    from paper_1805_12344_gb300 import workloads as W
    bad = W.CSR(m=2, n=3, row_ptr=np.array([0, 2, 1], np.int64), col_idx=np.array([0, 1], np.int32),
                val=np.ones(2))
    with pytest.raises(abip.AbipError) as e:
        abip.abip_setup(bad, b, c)
    assert e.value.code in (abip.ABIP_E_DIM, abip.ABIP_E_CUDA)
    # empty batch is a no-op
    assert lib.abip_solve_batch(0, None, None, None, None, None, None, None, None, None) == 0


def test_shared_and_backward_argument_errors_without_device(lib):
    """The shared-A batch and the batch backward refuse bad arguments before any device work."""
    from paper_1805_12344_gb300 import abip
    from paper_1805_12344_gb300 import workloads as W
    assert lib.abip_solve_batch_shared(0, None, None, None, None, None, None, None, None, None) == 0
    assert lib.abip_solve_batch_shared(1, None, None, None, None, None, None, None, None, None) == \
        abip.ABIP_E_INVALID_ARG
    assert lib.abip_backward(None, None, None, None, None) == abip.ABIP_E_INVALID_ARG
    assert lib.abip_backward_batch(0, None, None, None, None, None, None, None, None, None, None, None, None,
                                   None) == 0
    # a CSR matrix is not a shared dense A
    csr = W.dense_to_csr(np.eye(2, 3))
    with pytest.raises(abip.AbipError) as e:
        abip.abip_solve_batch_shared(csr, [np.ones(2)], [np.ones(3)])
    assert e.value.code == abip.ABIP_E_UNSUPPORTED
    # the tensor-core products hold A as bfloat16 terms of its FP32 value: beyond FP32's range
    A = np.full((2, 3), 0.1)
    A[1, 2] = 1e39
    with pytest.raises(abip.AbipError) as e:
        abip.abip_solve_batch_shared(A, [np.ones(2)], [np.ones(3)],
                                     abip.default_params(precision=abip.ABIP_PREC_MIXED_BF16))
    assert e.value.code == abip.ABIP_E_INVALID_ARG
    assert b"FP32 range" in lib.abip_last_error(None)
    # the Barzilai-Borwein selection is provided on the dense FP64 path only
    with pytest.raises(abip.AbipError) as e:
        abip.abip_solve_batch_shared(np.eye(2, 3), [np.ones(2)], [np.ones(3)], abip.default_params(bb_beta=1))
    assert e.value.code == abip.ABIP_E_UNSUPPORTED
    with pytest.raises(abip.AbipError) as e:
        abip.abip_solve_batch([np.eye(2, 3)], [np.ones(2)], [np.ones(3)],
                              abip.default_params(bb_beta=1, precision=abip.ABIP_PREC_MIXED))
    assert e.value.code == abip.ABIP_E_UNSUPPORTED
    for bad in (dict(bb_beta=2), dict(bb_beta=1, eps_cor=-1.0), dict(bb_beta=1, bb_max_redo=-1),
                dict(gamma_max=0.05), dict(gamma_max=1.0), dict(gamma_max=-0.5)):   # [gamma, 1) or 0
        with pytest.raises(abip.AbipError) as e:
            abip.abip_solve_batch([np.eye(2, 3)], [np.ones(2)], [np.ones(3)], abip.default_params(**bad))
        assert e.value.code == abip.ABIP_E_INVALID_ARG
    # no gradient at an infeasibility certificate (status from the forward's infos)
    with pytest.raises(abip.AbipError) as e:
        abip.abip_backward_batch([np.eye(2, 3)], [np.ones(2)], [np.ones(3)], [np.ones(3)], [np.ones(2)],
                                 [np.ones(3)], [dict(status=abip.ABIP_PRIMAL_INFEASIBLE, tau=1.0, kappa=1.0,
                                                     theta=1.0, mu=1e-3)], [np.ones(3)])
    assert e.value.code == abip.ABIP_E_INVALID_ARG
