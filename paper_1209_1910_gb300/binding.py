"""Thin ctypes binding of libtinv (C ABI in include/tinv.h).

Argument marshalling only: every step of the computation runs in the CUDA library.  Host
(numpy) arrays go through the synchronous host-pointer mode; torch CUDA tensors go through
the device-pointer mode on the tensor's current stream.  There is no fallback: if the library
is missing or the device is unusable, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtinv.so")
_lock = threading.Lock()
_lib = None

TINV_CWY, TINV_MGS = 0, 1
METHODS = {"cwy": TINV_CWY, "mgs": TINV_MGS}
ERRORS = {-101: "ENOMEM", -102: "ECUDA", -103: "ETIMEDOUT", -104: "EAGAIN", -105: "ECANCELED",
          -106: "ENOTSUP", -107: "ENODEV", -108: "EWORKSPACE"}

# every function include/tinv.h declares
EXPORTS = ["tinv_opts_default", "tinv_strerror", "tinv_version", "tinv", "tinv_ex",
           "tinv_workspace_size", "tinv_plan", "tinv_lu", "tinv_solve", "tinv_solve_noalloc",
           "tinv_orth"]


class TinvError(RuntimeError):
    def __init__(self, code: int, fn: str):
        self.code = code
        msg = load().tinv_strerror(code).decode()
        super().__init__("%s returned %d (%s)" % (fn, code, msg))


class Opts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int32), ("device_ptrs", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("seed", ctypes.c_uint64), ("j0", ctypes.c_int64),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t),
                ("iters", ctypes.c_void_p), ("info", ctypes.c_void_p),
                ("max_team", ctypes.c_int32), ("grid_ctas", ctypes.c_int32),
                ("phase_ms", ctypes.c_void_p), ("reserved", ctypes.c_int32 * 8)]


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libtinv.so (built by paper_1209_1910_gb300.build); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError("libtinv.so not found at %s: build it with "
                                   "`python -m paper_1209_1910_gb300.build`" % p)
            lib = ctypes.CDLL(p)
            P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
            lib.tinv_opts_default.argtypes = [ctypes.POINTER(Opts)]
            lib.tinv_opts_default.restype = None
            lib.tinv_strerror.argtypes = [ctypes.c_int]
            lib.tinv_strerror.restype = ctypes.c_char_p
            lib.tinv_version.restype = ctypes.c_char_p
            lib.tinv.argtypes = [I64, P, P, P, P]
            lib.tinv.restype = ctypes.c_int
            lib.tinv_ex.argtypes = [I64, P, P, I64, P, P, I64, ctypes.POINTER(Opts), P]
            lib.tinv_ex.restype = ctypes.c_int
            lib.tinv_workspace_size.argtypes = [I64, I64, ctypes.POINTER(Opts)]
            lib.tinv_workspace_size.restype = ctypes.c_size_t
            lib.tinv_plan.argtypes = [I64, P, P, I64, P, P, P, P, ctypes.POINTER(Opts)]
            lib.tinv_plan.restype = ctypes.c_int
            lib.tinv_lu.argtypes = [I64, P, P, I64, P, P, P, P, P, P, ctypes.POINTER(Opts)]
            lib.tinv_lu.restype = ctypes.c_int
            lib.tinv_solve.argtypes = [I64, P, P, I64, P, P, I64, I32, ctypes.POINTER(Opts)]
            lib.tinv_solve.restype = ctypes.c_int
            lib.tinv_solve_noalloc.argtypes = [I64, P, P, I64, P, P, I64, I32, P]
            lib.tinv_solve_noalloc.restype = ctypes.c_int
            lib.tinv_orth.argtypes = [I64, I64, P, I64, P, I64, P, P, ctypes.POINTER(Opts)]
            lib.tinv_orth.restype = ctypes.c_int
            _lib = lib
    return _lib


def _opts(method="cwy", seed=0, j0=0, device=False, stream=None, **kw) -> Opts:
    o = Opts()
    load().tinv_opts_default(ctypes.byref(o))
    o.method = METHODS[method] if isinstance(method, str) else int(method)
    o.seed = seed
    o.j0 = j0
    o.device_ptrs = 1 if device else 0
    o.stream = stream
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr() or None
    return a.ctypes.data_as(ctypes.c_void_p) if a.size else None


def _check(rc: int, fn: str) -> int:
    if rc < 0:
        raise TinvError(rc, fn)
    return rc


def _stream_of(t):
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


# ------------------------------------------------------------------------------------------
# host-pointer API (numpy)
# ------------------------------------------------------------------------------------------
def tinv(d, e, w, method="cwy", seed=0, j0=0, return_info=False, out=None, **kw):
    """Eigenvectors for all approximations w (host arrays).  Returns Z (n x m, Fortran order),
    or (Z, info, ifail, iters) with return_info.  `out` may supply Z (e.g. pinned memory)."""
    d, e, w = _f64(d), _f64(e), _f64(w)
    n, m = len(d), len(w)
    Z = np.zeros((n, m), order="F") if out is None else out
    assert Z.shape == (n, m) and Z.flags.f_contiguous and Z.dtype == np.float64
    ifail = np.zeros(max(m, 1), dtype=np.int64)
    iters = np.zeros(max(m, 1), dtype=np.int32)
    o = _opts(method, seed, j0, iters=iters.ctypes.data, **kw)
    rc = _check(load().tinv_ex(n, _ptr(d), _ptr(e), m, _ptr(w), _ptr(Z), max(n, 1),
                               ctypes.byref(o), ifail.ctypes.data), "tinv_ex")
    if return_info:
        return Z, rc, ifail[:rc], iters[:m]
    return Z


def plan(d, e, w, **kw):
    """Returns (wp, head, scal) of the cluster plan."""
    d, e, w = _f64(d), _f64(e), _f64(w)
    n, m = len(d), len(w)
    wp = np.zeros(m)
    head = np.zeros(m, dtype=np.int32)
    scal = np.zeros(3)
    o = _opts(**kw)
    _check(load().tinv_plan(n, _ptr(d), _ptr(e), m, _ptr(w), _ptr(wp), _ptr(head), _ptr(scal),
                            ctypes.byref(o)), "tinv_plan")
    return wp, head, scal


def lu(d, e, s, **kw):
    """LU factors of T - s_j I for each shift: (l, u0, u1, u2, piv), each m x n."""
    d, e, s = _f64(d), _f64(e), _f64(s)
    n, m = len(d), len(s)
    outs = [np.zeros((m, n)) for _ in range(4)]
    piv = np.zeros((m, n), dtype=np.uint8)
    o = _opts(**kw)
    _check(load().tinv_lu(n, _ptr(d), _ptr(e), m, _ptr(s), *[_ptr(x) for x in outs], _ptr(piv),
                          ctypes.byref(o)), "tinv_lu")
    return (*outs, piv)


def solve(d, e, s, X, scale=False, **kw):
    """x_j <- (T - s_j I)^{-1} x_j (optionally DSTEIN-scaled first); X is n x m."""
    d, e, s = _f64(d), _f64(e), _f64(s)
    X = np.asfortranarray(X, dtype=np.float64).copy(order="F")
    n, m = X.shape
    o = _opts(**kw)
    _check(load().tinv_solve(n, _ptr(d), _ptr(e), m, _ptr(s), _ptr(X), n, int(bool(scale)),
                             ctypes.byref(o)), "tinv_solve")
    return X


def orth(V, method="cwy", want_yt=False, **kw):
    """GPU incremental orthogonalization of the columns of V (n x m)."""
    V = np.asfortranarray(V, dtype=np.float64)
    n, m = V.shape
    Q = np.zeros((n, m), order="F")
    Y = np.zeros((n, m), order="F") if want_yt else None
    T = np.zeros((m, m), order="F") if want_yt else None
    o = _opts(method, **kw)
    _check(load().tinv_orth(n, m, _ptr(V), n, _ptr(Q), n, _ptr(Y), _ptr(T), ctypes.byref(o)),
           "tinv_orth")
    return (Q, Y, T) if want_yt else Q


# ------------------------------------------------------------------------------------------
# device-pointer API (torch CUDA tensors, asynchronous on the current stream)
# ------------------------------------------------------------------------------------------
def workspace_size(n: int, m: int, **kw) -> int:
    return int(load().tinv_workspace_size(n, m, ctypes.byref(_opts(**kw))))


def tinv_device(d, e, w, Z, method="cwy", seed=0, j0=0, workspace=None, iters=None, info=None,
                **kw):
    """Enqueue inverse iteration on torch CUDA tensors (float64 d[n], e[n-1], w[m], Z[m, n]
    whose rows are the eigenvectors, i.e. column-major n x m).  Returns immediately."""
    n, m = d.numel(), w.numel()
    o = _opts(method, seed, j0, device=True, stream=_stream_of(d),
              workspace=_ptr(workspace),
              workspace_bytes=(workspace.numel() * workspace.element_size()) if workspace is not None else 0,
              iters=_ptr(iters), info=_ptr(info), **kw)
    return _check(load().tinv_ex(n, _ptr(d), _ptr(e), m, _ptr(w), _ptr(Z), n, ctypes.byref(o),
                                 None), "tinv_ex")
