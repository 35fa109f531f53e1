"""Thin ctypes binding of libabip (C ABI in include/abip.h).

Argument marshalling only: every step of the solve runs in the library's CUDA
kernels.  Arrays may be numpy arrays (host) or CUDA torch tensors (device); the
library detects which.  Functions keep the C names (`abip_setup`, `abip_solve`,
`abip_solve_batch`, `abip_backward`, ...); `Solver` wraps a handle.

The library is required: importing works without it, but any call raises
`AbipError` if libabip.so is missing (there is no fallback implementation).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from . import workloads as _W

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libabip.so")

ABIP_OK = 0
ABIP_E_INVALID_ARG = -1
ABIP_E_DIM = -2
ABIP_E_CUDA = -3
ABIP_E_OOM = -4
ABIP_E_NOT_SOLVED = -5
ABIP_E_NUMERICAL = -6
ABIP_E_UNSUPPORTED = -7
ABIP_E_TIMEOUT = -8

ABIP_DENSE_ROWMAJOR = 0
ABIP_CSR = 1
ABIP_F32 = 0
ABIP_F64 = 1
ABIP_UNSOLVED = 0
ABIP_OPTIMAL = 1
ABIP_PRIMAL_INFEASIBLE = 2
ABIP_DUAL_INFEASIBLE = 3
ABIP_MAX_ITER = 4
ABIP_PREC_F64 = 0
ABIP_PREC_MIXED = 1
ABIP_PREC_MIXED_BF16 = 2
ABIP_LINSYS_DENSE_CHOL = 0
ABIP_LINSYS_PCG = 1
ABIP_LINSYS_SPARSE_LDL = 2

STATUS_NAMES = {0: "unsolved", 1: "optimal", 2: "primal_infeasible", 3: "dual_infeasible", 4: "max_iter"}


class AbipError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"abip error {code}: {msg}")
        self.code = code


class abip_matrix(C.Structure):
    _fields_ = [("m", C.c_int32), ("n", C.c_int32), ("fmt", C.c_int32), ("dtype", C.c_int32),
                ("on_device", C.c_int32), ("val", C.c_void_p), ("ld", C.c_int64),
                ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("nnz", C.c_int64)]


class abip_params(C.Structure):
    _fields_ = [("beta", C.c_double), ("gamma", C.c_double), ("alpha", C.c_double), ("eps", C.c_double),
                ("max_admm_iters", C.c_int64), ("linsys", C.c_int32), ("cg_tol", C.c_double),
                ("cg_max_iter", C.c_int32), ("cg_rel", C.c_double), ("cg_warm", C.c_int32), ("precision", C.c_int32), ("warmstart", C.c_int32),
                ("stop_rule", C.c_int32), ("check_every", C.c_int32), ("grid_ctas", C.c_int32),
                ("barrier_limit_ns", C.c_int64), ("bb_beta", C.c_int32), ("bb_max_redo", C.c_int32),
                ("eps_cor", C.c_double), ("eps_penalty", C.c_double), ("autotune", C.c_int32),
                ("batch_order", C.c_int32), ("gamma_max", C.c_double),
                ("reserved", C.c_int32 * 4)]


class abip_presolve_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("m", C.c_int32), ("n", C.c_int32), ("nnz", C.c_int64),
                ("obj_offset", C.c_double), ("empty_rows", C.c_int32), ("singleton_rows", C.c_int32),
                ("dependent_rows", C.c_int32), ("fixed_cols", C.c_int32), ("empty_cols", C.c_int32),
                ("free_split", C.c_int32), ("upper_rows", C.c_int32), ("reserved", C.c_int32 * 5)]


class abip_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("outer_iters", C.c_int32), ("admm_iters", C.c_int64),
                ("cg_iters", C.c_int64), ("tau", C.c_double), ("kappa", C.c_double), ("theta", C.c_double),
                ("mu", C.c_double), ("obj", C.c_double), ("pres", C.c_double), ("dres", C.c_double),
                ("dgap", C.c_double), ("setup_s", C.c_double), ("solve_s", C.c_double),
                ("kernel_s", C.c_double), ("launches", C.c_int64), ("fp32_iters", C.c_int64),
                ("beta", C.c_double), ("ctas_per_sm", C.c_int32), ("tuned", C.c_int32)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["status_name"] = STATUS_NAMES.get(self.status, "unknown")
        return d


_lib = None

# every symbol include/abip.h declares, with its ctypes signature
_SIGS = {
    "abip_default_params": (C.c_int, [C.POINTER(abip_params)]),
    "abip_setup": (C.c_int, [C.POINTER(abip_matrix), C.c_void_p, C.c_void_p, C.POINTER(abip_params),
                             C.POINTER(C.c_void_p)]),
    "abip_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(abip_info), C.c_void_p]),
    "abip_solve_batch": (C.c_int, [C.c_int32, C.POINTER(abip_matrix), C.POINTER(C.c_void_p),
                                   C.POINTER(C.c_void_p), C.POINTER(abip_params), C.POINTER(C.c_void_p),
                                   C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(abip_info),
                                   C.c_void_p]),
    "abip_solve_batch_shared": (C.c_int, [C.c_int32, C.POINTER(abip_matrix), C.POINTER(C.c_void_p),
                                          C.POINTER(C.c_void_p), C.POINTER(abip_params), C.POINTER(C.c_void_p),
                                          C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(abip_info),
                                          C.c_void_p]),
    "abip_backward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "abip_backward_batch": (C.c_int, [C.c_int32, C.POINTER(abip_matrix), C.POINTER(C.c_void_p),
                                      C.POINTER(C.c_void_p), C.POINTER(abip_params), C.POINTER(C.c_void_p),
                                      C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(abip_info),
                                      C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                      C.POINTER(C.c_void_p), C.c_void_p]),
    "abip_get_state": (C.c_int, [C.c_void_p, C.c_void_p]),
    "abip_set_state": (C.c_int, [C.c_void_p, C.c_void_p]),
    "abip_state_size": (C.c_int64, [C.c_void_p]),
    "abip_free": (None, [C.c_void_p]),
    "abip_presolve": (C.c_int, [C.POINTER(abip_matrix), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_double, C.c_int32, C.POINTER(C.c_void_p), C.c_void_p]),
    "abip_presolved_lp": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "abip_postsolve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p]),
    "abip_presolve_free": (None, [C.c_void_p]),
    "abip_ldl_analyze": (C.c_int, [C.POINTER(abip_matrix), C.c_void_p, C.c_void_p, C.POINTER(C.c_int64)]),
    "abip_status_str": (C.c_char_p, [C.c_int32]),
    "abip_last_error": (C.c_char_p, [C.c_void_p]),
    "abip_version": (C.c_char_p, []),
}


def lib():
    """The loaded libabip (built in-tree by `paper_1805_12344_gb300.build`)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise AbipError(ABIP_E_UNSUPPORTED, f"{_LIB_PATH} not built: run paper_1805_12344_gb300.build.build()")
        L = C.CDLL(_LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, h=None):
    if rc != ABIP_OK:
        msg = lib().abip_last_error(h).decode()
        raise AbipError(rc, msg)


def default_params(**kw) -> abip_params:
    p = abip_params()
    _check(lib().abip_default_params(C.byref(p)))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


# --- array marshalling ------------------------------------------------------

def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a):
    """(address, keepalive, on_device) of a numpy array or torch tensor."""
    if a is None:
        return None, None, False
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), a, bool(a.is_cuda)
    arr = np.ascontiguousarray(a)
    return arr.ctypes.data, arr, False


def _matrix(A, dtype=None):
    """abip_matrix for a dense numpy/torch 2-D array or a workloads.CSR."""
    keep = []
    M = abip_matrix()
    if isinstance(A, _W.CSR):
        M.m, M.n, M.fmt = A.m, A.n, ABIP_CSR
        val = A.val if dtype is None else A.val.astype(dtype)
        M.dtype = ABIP_F32 if val.dtype == np.float32 else ABIP_F64
        rp = np.ascontiguousarray(A.row_ptr, dtype=np.int64)
        ci = np.ascontiguousarray(A.col_idx, dtype=np.int32)
        val = np.ascontiguousarray(val)
        keep += [rp, ci, val]
        M.row_ptr, M.col_idx, M.val = rp.ctypes.data, ci.ctypes.data, val.ctypes.data
        M.nnz = A.nnz
        M.on_device = 0
        return M, keep
    if _is_torch(A):
        t = A.contiguous()
        keep.append(t)
        M.m, M.n = t.shape
        M.fmt = ABIP_DENSE_ROWMAJOR
        M.dtype = ABIP_F32 if str(t.dtype) == "torch.float32" else ABIP_F64
        M.val = t.data_ptr()
        M.ld = t.shape[1]
        M.on_device = 1 if t.is_cuda else 0
        return M, keep
    a = np.ascontiguousarray(A, dtype=np.float64 if dtype is None else dtype)
    keep.append(a)
    M.m, M.n = a.shape
    M.fmt = ABIP_DENSE_ROWMAJOR
    M.dtype = ABIP_F32 if a.dtype == np.float32 else ABIP_F64
    M.val = a.ctypes.data
    M.ld = a.shape[1]
    M.on_device = 0
    return M, keep


# --- C-named entry points ---------------------------------------------------

def abip_setup(A, b, c, params: Optional[abip_params] = None) -> C.c_void_p:
    M, keep = _matrix(A)
    bp, kb, _ = _ptr(b if _is_torch(b) else np.asarray(b, dtype=np.float64))
    cp, kc, _ = _ptr(c if _is_torch(c) else np.asarray(c, dtype=np.float64))
    h = C.c_void_p()
    rc = lib().abip_setup(C.byref(M), bp, cp, C.byref(params) if params is not None else None, C.byref(h))
    _check(rc)
    return h


def abip_ldl_analyze(A):
    """(perm, col_counts, nnz_l) of the sparse direct projection's symbolic factor: the
    minimum-degree order of K = [I A^T; A -I] (node j < n: x_j, node n + i: row i of A)
    and the strictly-lower nonzeros of each column of L.  Host only."""
    M, keep = _matrix(A)
    N = M.m + M.n
    perm = np.zeros(N, dtype=np.int32)
    counts = np.zeros(N, dtype=np.int64)
    nnz = C.c_int64(0)
    _check(lib().abip_ldl_analyze(C.byref(M), perm.ctypes.data, counts.ctypes.data, C.byref(nnz)))
    return perm, counts, int(nnz.value)


def abip_solve(h, x=None, y=None, s=None, stream=None) -> dict:
    info = abip_info()
    xp, _, _ = _ptr(x)
    yp, _, _ = _ptr(y)
    sp_, _, _ = _ptr(s)
    st = None
    if stream is not None:
        st = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    _check(lib().abip_solve(h, xp, yp, sp_, C.byref(info), st), h)
    return info.as_dict()


def abip_get_state(h) -> np.ndarray:
    n = lib().abip_state_size(h)
    buf = np.zeros(n)
    _check(lib().abip_get_state(h, buf.ctypes.data), h)
    return buf


def abip_set_state(h, state):
    buf = np.ascontiguousarray(state, dtype=np.float64)
    _check(lib().abip_set_state(h, buf.ctypes.data), h)


def abip_free(h):
    lib().abip_free(h)


def abip_backward(h, dl_dx, dl_dc=None, dl_db=None, dl_dA=None):
    """Gradients of L(x*) w.r.t. c, b, A at the central point of the last solve's final mu,
    written into the caller's arrays (numpy or CUDA tensors, float64; None to skip)."""
    gp, _kg, _ = _ptr(dl_dx if _is_torch(dl_dx) else np.ascontiguousarray(dl_dx, dtype=np.float64))
    _check(lib().abip_backward(h, gp, _ptr(dl_dc)[0], _ptr(dl_db)[0], _ptr(dl_dA)[0]), h)


def _stream_arg(stream):
    if stream is None:
        return None
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _vec(a):
    return a if _is_torch(a) else np.ascontiguousarray(a, dtype=np.float64)


def _info_struct(d: dict) -> abip_info:
    f = abip_info()
    for k, _ in abip_info._fields_:
        if k in d:
            setattr(f, k, d[k])
    return f


def abip_backward_batch(As: Sequence, bs: Sequence, cs: Sequence, xs: Sequence, ys: Sequence, ss: Sequence,
                        infos: Sequence[dict], dl_dxs: Sequence, params: Optional[abip_params] = None,
                        want=("c", "b", "A"), device: bool = False, stream=None):
    """Gradients for the instances of one `abip_solve_batch` call (one launch).  xs, ys, ss,
    infos: what that call returned.  Returns lists (dcs, dbs, dAs) with None where not wanted;
    numpy arrays, or CUDA float64 tensors when `device`."""
    count = len(As)
    mats = (abip_matrix * count)()
    keep = []
    ptrs = {k: (C.c_void_p * count)() for k in ("b", "c", "x", "y", "s", "g", "dc", "db", "dA")}
    outs = {"c": [], "b": [], "A": []}
    finfo = (abip_info * count)()
    if device:
        import torch
    for k in range(count):
        M, kk = _matrix(As[k])
        keep += kk
        mats[k] = M
        for name, arr in (("b", bs[k]), ("c", cs[k]), ("x", xs[k]), ("y", ys[k]), ("s", ss[k]), ("g", dl_dxs[k])):
            a = _vec(arr)
            keep.append(a)
            ptrs[name][k] = _ptr(a)[0]
        finfo[k] = _info_struct(infos[k])
        for name, shape in (("c", (M.n,)), ("b", (M.m,)), ("A", (M.m, M.n))):
            if name in want:
                o = torch.empty(shape, dtype=torch.float64, device="cuda") if device else np.zeros(shape)
                outs[name].append(o)
                ptrs["d" + name][k] = _ptr(o)[0]
            else:
                outs[name].append(None)
    rc = lib().abip_backward_batch(count, mats, ptrs["b"], ptrs["c"],
                                   C.byref(params) if params is not None else None,
                                   ptrs["x"], ptrs["y"], ptrs["s"], finfo, ptrs["g"],
                                   ptrs["dc"] if "c" in want else None, ptrs["db"] if "b" in want else None,
                                   ptrs["dA"] if "A" in want else None, _stream_arg(stream))
    _check(rc)
    return outs["c"], outs["b"], outs["A"]


def abip_solve_batch(As: Sequence, bs: Sequence, cs: Sequence, params: Optional[abip_params] = None,
                     want_solution: bool = True, stream=None, device_out: bool = False):
    """Solve dense LPs (numpy arrays or torch tensors) in one persistent launch.
    Returns (infos, xs, ys, ss); the solutions are numpy arrays, or CUDA float64 tensors
    when `device_out`."""
    count = len(As)
    mats = (abip_matrix * count)()
    keep = []
    bptr = (C.c_void_p * count)()
    cptr = (C.c_void_p * count)()
    xs, ys, ss = [], [], []
    xptr = (C.c_void_p * count)()
    yptr = (C.c_void_p * count)()
    sptr = (C.c_void_p * count)()
    for k in range(count):
        M, kk = _matrix(As[k])
        keep += kk
        mats[k] = M
        b, c = _vec(bs[k]), _vec(cs[k])
        keep += [b, c]
        bptr[k] = _ptr(b)[0]
        cptr[k] = _ptr(c)[0]
        if want_solution:
            if device_out:
                import torch
                x, y, s = (torch.empty(k_, dtype=torch.float64, device="cuda") for k_ in (M.n, M.m, M.n))
            else:
                x, y, s = np.zeros(M.n), np.zeros(M.m), np.zeros(M.n)
            xs.append(x); ys.append(y); ss.append(s)
            xptr[k], yptr[k], sptr[k] = _ptr(x)[0], _ptr(y)[0], _ptr(s)[0]
    infos = (abip_info * count)()
    st = None
    if stream is not None:
        st = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    rc = lib().abip_solve_batch(count, mats, bptr, cptr, C.byref(params) if params is not None else None,
                                xptr if want_solution else None, yptr if want_solution else None,
                                sptr if want_solution else None, infos, st)
    _check(rc)
    return [infos[k].as_dict() for k in range(count)], xs, ys, ss


def abip_solve_batch_shared(A, bs: Sequence, cs: Sequence, params: Optional[abip_params] = None,
                            want_solution: bool = True, stream=None, device_out: bool = False):
    """Solve LPs that share the dense matrix A (numpy array or CUDA tensor) in lockstep.
    Returns (infos, xs, ys, ss) like `abip_solve_batch`."""
    count = len(bs)
    M, keep = _matrix(A)
    bptr = (C.c_void_p * count)()
    cptr = (C.c_void_p * count)()
    xptr = (C.c_void_p * count)()
    yptr = (C.c_void_p * count)()
    sptr = (C.c_void_p * count)()
    xs, ys, ss = [], [], []
    for k in range(count):
        b, c = _vec(bs[k]), _vec(cs[k])
        keep += [b, c]
        bptr[k] = _ptr(b)[0]
        cptr[k] = _ptr(c)[0]
        if want_solution:
            if device_out:
                import torch
                x, y, s = (torch.empty(k_, dtype=torch.float64, device="cuda") for k_ in (M.n, M.m, M.n))
            else:
                x, y, s = np.zeros(M.n), np.zeros(M.m), np.zeros(M.n)
            xs.append(x); ys.append(y); ss.append(s)
            xptr[k], yptr[k], sptr[k] = _ptr(x)[0], _ptr(y)[0], _ptr(s)[0]
    infos = (abip_info * count)()
    rc = lib().abip_solve_batch_shared(count, C.byref(M), bptr, cptr,
                                       C.byref(params) if params is not None else None,
                                       xptr if want_solution else None, yptr if want_solution else None,
                                       sptr if want_solution else None, infos, _stream_arg(stream))
    _check(rc)
    return [infos[k].as_dict() for k in range(count)], xs, ys, ss


class Presolved:
    """abip_presolve of  min c^T x, A x = b, l <= x <= w  (Sec. 4.5) on the host: `info` (dict),
    `lp()` the standard-form LP (a workloads.CSR, b, c), `postsolve(x, y)` the original
    (x, y, z = c - A^T y, objective).  l / w: use -inf / +inf for absent bounds."""

    def __init__(self, A, b, c, l, w, tol: float = 1e-9, ruiz: int = 10):
        M, keep = _matrix(A)
        arrs = [np.ascontiguousarray(v, dtype=np.float64) for v in (b, c, l, w)]
        self._h = C.c_void_p()
        inf = abip_presolve_info()
        rc = lib().abip_presolve(C.byref(M), *[a.ctypes.data for a in arrs], tol, ruiz, C.byref(self._h),
                                 C.byref(inf))
        _check(rc)
        self.info = {k: getattr(inf, k) for k, _ in abip_presolve_info._fields_ if k != "reserved"}
        self.status = inf.status
        self.why = lib().abip_last_error(None).decode() if inf.status not in (0, ABIP_OPTIMAL) else ""
        self.m0, self.n0 = M.m, M.n

    def lp(self):
        m, n, nnz = self.info["m"], self.info["n"], self.info["nnz"]
        rp = np.zeros(m + 1, dtype=np.int64)
        ci = np.zeros(nnz, dtype=np.int32)
        val = np.zeros(nnz, dtype=np.float64)
        b = np.zeros(m)
        c = np.zeros(n)
        _check(lib().abip_presolved_lp(self._h, rp.ctypes.data, ci.ctypes.data, val.ctypes.data,
                                       b.ctypes.data, c.ctypes.data))
        return _W.CSR(m=m, n=n, row_ptr=rp, col_idx=ci, val=val), b, c

    def postsolve(self, x, y):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        xo = np.zeros(self.n0)
        yo = np.zeros(self.m0)
        zo = np.zeros(self.n0)
        obj = C.c_double()
        _check(lib().abip_postsolve(self._h, x.ctypes.data, y.ctypes.data, None, xo.ctypes.data,
                                    yo.ctypes.data, zo.ctypes.data, C.byref(obj)))
        return xo, yo, zo, obj.value

    def close(self):
        if getattr(self, "_h", None):
            lib().abip_presolve_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """One LP on the GPU: setup once, solve, read the state."""

    def __init__(self, A, b, c, **params):
        self.params = default_params(**params)
        self.h = abip_setup(A, b, c, self.params)
        self.m, self.n = (A.m, A.n) if isinstance(A, _W.CSR) else tuple(A.shape)

    def solve(self, device_out: bool = False, stream=None):
        if device_out:
            import torch
            x = torch.empty(self.n, dtype=torch.float64, device="cuda")
            y = torch.empty(self.m, dtype=torch.float64, device="cuda")
            s = torch.empty(self.n, dtype=torch.float64, device="cuda")
        else:
            x, y, s = np.zeros(self.n), np.zeros(self.m), np.zeros(self.n)
        info = abip_solve(self.h, x, y, s, stream=stream)
        return info, x, y, s

    def backward(self, dl_dx, want=("c", "b", "A")) -> dict:
        """dL/dc, dL/db, dL/dA (numpy) at the central point of the last solve's final mu."""
        out = {"c": np.zeros(self.n) if "c" in want else None,
               "b": np.zeros(self.m) if "b" in want else None,
               "A": np.zeros((self.m, self.n)) if "A" in want else None}
        abip_backward(self.h, dl_dx, out["c"], out["b"], out["A"])
        return out

    def state(self) -> np.ndarray:
        return abip_get_state(self.h)

    def set_state(self, state) -> None:
        abip_set_state(self.h, state)

    def stacked_state(self) -> np.ndarray:
        """(y, x, tau, theta, s, kappa): the iterate ordering of the parity tests."""
        st = self.state()
        return st[:-1]

    def close(self):
        if self.h:
            abip_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
