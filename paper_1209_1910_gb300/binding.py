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
           "tinv_workspace_size", "tinv_batch", "tinv_batch_workspace_size", "tinv_bisect",
           "tinv_bisect_batch", "tinv_split", "tinv_eig", "tinv_bdsvd",
           "tinv_plan", "tinv_tune", "tinv_tune_auto", "tinv_tune_batch", "tinv_tune_clear",
           "tinv_tune_save", "tinv_tune_load",
           "tinv_lu", "tinv_solve", "tinv_solve_noalloc", "tinv_orth",
           "tinv_server_cfg_default", "tinv_server_create", "tinv_submit", "tinv_poll",
           "tinv_wait", "tinv_cancel", "tinv_server_stats", "tinv_server_destroy"]


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
                ("phase_ms", ctypes.c_void_p), ("counters", ctypes.c_void_p),
                ("table_ready", ctypes.c_int32), ("spin_limit", ctypes.c_int32),
                ("block", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class Tuning(ctypes.Structure):
    _fields_ = [("max_team", ctypes.c_int32), ("block", ctypes.c_int32), ("ms", ctypes.c_float),
                ("cached", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


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
            SP = ctypes.POINTER(ctypes.c_void_p)
            lib.tinv_server_cfg_default.argtypes = [ctypes.POINTER(ServerCfg)]
            lib.tinv_server_cfg_default.restype = None
            lib.tinv_server_create.argtypes = [ctypes.POINTER(ServerCfg), SP]
            lib.tinv_server_create.restype = ctypes.c_int
            lib.tinv_submit.argtypes = [P, I64, P, P, P, P, ctypes.c_uint64,
                                        ctypes.POINTER(ctypes.c_uint64)]
            lib.tinv_submit.restype = ctypes.c_int
            lib.tinv_poll.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32)]
            lib.tinv_poll.restype = ctypes.c_int
            lib.tinv_wait.argtypes = [P, ctypes.c_uint64, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)]
            lib.tinv_wait.restype = ctypes.c_int
            lib.tinv_cancel.argtypes = [P, ctypes.c_uint64]
            lib.tinv_cancel.restype = ctypes.c_int
            lib.tinv_server_stats.argtypes = [P, ctypes.POINTER(Stats)]
            lib.tinv_server_stats.restype = ctypes.c_int
            lib.tinv_server_destroy.argtypes = [P]
            lib.tinv_server_destroy.restype = ctypes.c_int
            lib.tinv_bisect.argtypes = [I64, P, P, P, ctypes.POINTER(Opts)]
            lib.tinv_bisect.restype = ctypes.c_int
            lib.tinv_bisect_batch.argtypes = [I64, P, P, P, P, P, ctypes.POINTER(Opts)]
            lib.tinv_bisect_batch.restype = ctypes.c_int
            lib.tinv_batch.argtypes = [I64, P, P, P, P, P, P, P, P, ctypes.POINTER(Opts)]
            lib.tinv_batch.restype = ctypes.c_int
            lib.tinv_batch_workspace_size.argtypes = [I64, P, ctypes.POINTER(Opts)]
            lib.tinv_batch_workspace_size.restype = ctypes.c_size_t
            lib.tinv_solve_noalloc.argtypes = [I64, P, P, I64, P, P, I64, I32, P]
            lib.tinv_solve_noalloc.restype = ctypes.c_int
            lib.tinv_orth.argtypes = [I64, I64, P, I64, P, I64, P, P, ctypes.POINTER(Opts)]
            lib.tinv_orth.restype = ctypes.c_int
            lib.tinv_split.argtypes = [I64, P, P, P, P, ctypes.POINTER(Opts)]
            lib.tinv_split.restype = ctypes.c_int
            lib.tinv_eig.argtypes = [I64, P, P, P, P, I64, P, P, P, ctypes.POINTER(Opts)]
            lib.tinv_eig.restype = ctypes.c_int
            lib.tinv_bdsvd.argtypes = [I64, P, P, P, P, I64, P, I64, ctypes.POINTER(Opts)]
            lib.tinv_bdsvd.restype = ctypes.c_int
            lib.tinv_tune.argtypes = [I64, P, P, I64, P, ctypes.POINTER(Opts), I32,
                                      ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float),
                                      ctypes.POINTER(ctypes.c_int32)]
            lib.tinv_tune.restype = ctypes.c_int
            lib.tinv_tune_auto.argtypes = [I64, P, P, I64, P, ctypes.POINTER(Opts), I32,
                                           ctypes.POINTER(Tuning)]
            lib.tinv_tune_auto.restype = ctypes.c_int
            lib.tinv_tune_batch.argtypes = [I64, P, P, P, P, P, P, ctypes.POINTER(Opts), I32,
                                            ctypes.POINTER(Tuning)]
            lib.tinv_tune_batch.restype = ctypes.c_int
            lib.tinv_tune_clear.argtypes = []
            lib.tinv_tune_clear.restype = None
            lib.tinv_tune_save.argtypes = [ctypes.c_char_p]
            lib.tinv_tune_save.restype = ctypes.c_int
            lib.tinv_tune_load.argtypes = [ctypes.c_char_p]
            lib.tinv_tune_load.restype = ctypes.c_int
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


def tune(d, e, w, reps=2, **kw):
    """tinv_tune: (max_team, ms, cached) for this problem; pass max_team to later calls."""
    dev = kw.get("device", False)
    if not dev:
        d, e, w = _f64(d), _f64(e), _f64(w)
    n, m = len(d), len(w)
    mt, ms, cached = ctypes.c_int32(0), ctypes.c_float(0.0), ctypes.c_int32(0)
    o = _opts(**kw)
    _check(load().tinv_tune(n, _ptr(d), _ptr(e), m, _ptr(w), ctypes.byref(o), reps,
                            ctypes.byref(mt), ctypes.byref(ms), ctypes.byref(cached)), "tinv_tune")
    return int(mt.value), float(ms.value), bool(cached.value)


def tune_auto(d, e, w, reps=2, **kw):
    """tinv_tune_auto: (max_team, block, ms, cached) for this problem."""
    d, e, w = _f64(d), _f64(e), _f64(w)
    t = Tuning()
    _check(load().tinv_tune_auto(len(d), _ptr(d), _ptr(e), len(w), _ptr(w), ctypes.byref(_opts(**kw)),
                                 reps, ctypes.byref(t)), "tinv_tune_auto")
    return int(t.max_team), int(t.block), float(t.ms), bool(t.cached)


def tune_batch(ds, es, ws, reps=1, **kw):
    """tinv_tune_batch on host arrays of the problems: (max_team, block, ms, cached)."""
    ns, off_de, off_z = pack_offsets([len(d) for d in ds])
    M = int(ns.sum())
    D, E, W = np.zeros(max(M, 1)), np.zeros(max(M, 1)), np.zeros(max(M, 1))
    for q, (d, e, w) in enumerate(zip(ds, es, ws)):
        a, n = int(off_de[q]), int(ns[q])
        D[a:a + n], W[a:a + n] = d, w
        if n > 1:
            E[a:a + n - 1] = e
    t = Tuning()
    _check(load().tinv_tune_batch(len(ns), _ptr(ns), _ptr(off_de), _ptr(off_z), _ptr(D), _ptr(E), _ptr(W),
                                  ctypes.byref(_opts(**kw)), reps, ctypes.byref(t)), "tinv_tune_batch")
    return int(t.max_team), int(t.block), float(t.ms), bool(t.cached)


def tune_clear():
    load().tinv_tune_clear()


def tune_save(path: str) -> None:
    _check(load().tinv_tune_save(os.fsencode(path)), "tinv_tune_save")


def tune_load(path: str) -> int:
    """Merge a saved tune cache; returns the number of entries read."""
    return _check(load().tinv_tune_load(os.fsencode(path)), "tinv_tune_load")


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


# ------------------------------------------------------------------------------------------
# batched API: many independent problems of uneven order in one launch sequence
# ------------------------------------------------------------------------------------------
def pack_offsets(ns):
    """Packed offsets of d/e/w (sum of n) and of Z (sum of n^2) for problem orders ns."""
    ns = np.asarray(ns, dtype=np.int64)
    off_de = np.zeros(len(ns), dtype=np.int64)
    off_z = np.zeros(len(ns), dtype=np.int64)
    if len(ns):
        off_de[1:] = np.cumsum(ns)[:-1]
        off_z[1:] = np.cumsum(ns * ns)[:-1]
    return ns, off_de, off_z


def batch_workspace_size(ns, **kw) -> int:
    ns = np.ascontiguousarray(ns, dtype=np.int64)
    return int(load().tinv_batch_workspace_size(len(ns), _ptr(ns), ctypes.byref(_opts(**kw))))


def tinv_batch(ds, es, ws, method="cwy", seed=0, j0=0, return_info=False, **kw):
    """All eigenvectors of each problem (host arrays; lists of d, e, w).  Returns the list of
    Z_q (n_q x n_q, Fortran order), or (Zs, rc, info, iters) with return_info."""
    ns, off_de, off_z = pack_offsets([len(d) for d in ds])
    tot = int(ns.sum())
    d = np.zeros(max(tot, 1))
    e = np.zeros(max(tot, 1))
    w = np.zeros(max(tot, 1))
    for q in range(len(ns)):
        a, k = int(off_de[q]), int(ns[q])
        d[a:a + k] = ds[q]
        e[a:a + max(k - 1, 0)] = es[q][:max(k - 1, 0)]
        w[a:a + k] = ws[q]
    Z = np.zeros(max(int((ns * ns).sum()), 1))
    info = np.zeros(max(len(ns), 1), dtype=np.int64)
    iters = np.zeros(max(tot, 1), dtype=np.int32)
    o = _opts(method, seed, j0, iters=iters.ctypes.data, **kw)
    rc = _check(load().tinv_batch(len(ns), _ptr(ns), _ptr(off_de), _ptr(off_z), _ptr(d), _ptr(e),
                                  _ptr(w), _ptr(Z), _ptr(info), ctypes.byref(o)), "tinv_batch")
    Zs = [Z[int(off_z[q]):int(off_z[q] + ns[q] * ns[q])].reshape((int(ns[q]), int(ns[q])), order="F")
          for q in range(len(ns))]
    if return_info:
        return Zs, rc, info[:len(ns)], iters[:tot]
    return Zs


def tinv_batch_device(ns, off_de, off_z, d, e, w, Z, method="cwy", seed=0, j0=0, info=None,
                      workspace=None, iters=None, **kw):
    """Enqueue a batch on torch CUDA tensors (packed float64 d, e, w, Z; int64 info[nprob]);
    ns, off_de and off_z are host int64 arrays.  Returns immediately."""
    ns = np.ascontiguousarray(ns, dtype=np.int64)
    off_de = np.ascontiguousarray(off_de, dtype=np.int64)
    off_z = np.ascontiguousarray(off_z, dtype=np.int64)
    o = _opts(method, seed, j0, device=True, stream=_stream_of(d),
              workspace=_ptr(workspace),
              workspace_bytes=(workspace.numel() * workspace.element_size()) if workspace is not None else 0,
              iters=_ptr(iters), **kw)
    return _check(load().tinv_batch(len(ns), _ptr(ns), _ptr(off_de), _ptr(off_z), _ptr(d), _ptr(e),
                                    _ptr(w), _ptr(Z), _ptr(info), ctypes.byref(o)), "tinv_batch")


def bisect(d, e, **kw):
    """All eigenvalues of T (host arrays), ascending, by GPU Sturm bisection."""
    d, e = _f64(d), _f64(e)
    n = len(d)
    w = np.zeros(max(n, 1))
    _check(load().tinv_bisect(n, _ptr(d), _ptr(e), _ptr(w), ctypes.byref(_opts(**kw))), "tinv_bisect")
    return w[:n]


def bisect_batch_device(ns, off_de, d, e, w, **kw):
    """Enqueue bisection of packed problems on torch CUDA tensors (w receives the eigenvalues in
    the layout tinv_batch expects); ns and off_de are host int64 arrays.  Returns immediately."""
    ns = np.ascontiguousarray(ns, dtype=np.int64)
    off_de = np.ascontiguousarray(off_de, dtype=np.int64)
    o = _opts(device=True, stream=_stream_of(d), **kw)
    return _check(load().tinv_bisect_batch(len(ns), _ptr(ns), _ptr(off_de), _ptr(d), _ptr(e),
                                           _ptr(w), ctypes.byref(o)), "tinv_bisect_batch")


def split(d, e, **kw):
    """Unreduced blocks of T (host arrays): one past the last row of each block."""
    d, e = _f64(d), _f64(e)
    n = len(d)
    isplit = np.zeros(max(n, 1), dtype=np.int64)
    nb = ctypes.c_int64(0)
    _check(load().tinv_split(n, _ptr(d), _ptr(e), _ptr(isplit), ctypes.byref(nb),
                             ctypes.byref(_opts(**kw))), "tinv_split")
    return isplit[:nb.value].copy()


def split_device(d, e, **kw):
    """tinv_split on torch CUDA tensors d[n], e[n-1] (synchronizes their stream); returns the
    block ends (host int64 array)."""
    n = d.numel()
    isplit = np.zeros(max(n, 1), dtype=np.int64)
    nb = ctypes.c_int64(0)
    _check(load().tinv_split(n, _ptr(d), _ptr(e), _ptr(isplit), ctypes.byref(nb),
                             ctypes.byref(_opts(device=True, stream=_stream_of(d), **kw))),
           "tinv_split")
    return isplit[:nb.value].copy()


def eig(d, e, method="cwy", seed=0, j0=0, ldz=None, iters=None, **kw):
    """All eigenpairs of T split into unreduced blocks (host arrays).  Returns
    (w, Z, iblock, isplit, info): Z is n x n (column j the eigenvector of w[j])."""
    d, e = _f64(d), _f64(e)
    n = len(d)
    ldz = n if ldz is None else ldz
    w = np.zeros(max(n, 1))
    Zf = np.empty((max(ldz, 1), max(n, 1)), order="F")  # column-major, leading dimension ldz
    iblock = np.zeros(max(n, 1), dtype=np.int64)
    isplit = np.zeros(max(n, 1), dtype=np.int64)
    nb = ctypes.c_int64(0)
    o = _opts(method, seed, j0, iters=_ptr(iters), **kw)
    info = _check(load().tinv_eig(n, _ptr(d), _ptr(e), _ptr(w), _ptr(Zf), ldz, _ptr(iblock),
                                  _ptr(isplit), ctypes.byref(nb), ctypes.byref(o)), "tinv_eig")
    Z = Zf[:n, :n] if n else np.zeros((0, 0))
    return w[:n], Z, iblock[:n], isplit[:nb.value].copy(), info


def eig_device(d, e, w, Z, iblock=None, method="cwy", seed=0, j0=0, iters=None, **kw):
    """tinv_eig on torch CUDA tensors (float64 d[n], e[n-1], w[n], Z[n, n] whose rows are the
    eigenvectors, int64 iblock[n]).  Synchronizes the tensors' stream.  Returns
    (info, isplit)."""
    n = d.numel()
    isplit = np.zeros(max(n, 1), dtype=np.int64)
    nb = ctypes.c_int64(0)
    o = _opts(method, seed, j0, device=True, stream=_stream_of(d), iters=_ptr(iters), **kw)
    info = _check(load().tinv_eig(n, _ptr(d), _ptr(e), _ptr(w), _ptr(Z), n, _ptr(iblock),
                                  _ptr(isplit), ctypes.byref(nb), ctypes.byref(o)), "tinv_eig")
    return info, isplit[:nb.value].copy()


def bdsvd(a, b, method="cwy", seed=0, j0=0, iters=None, **kw):
    """Singular triplets of the upper bidiagonal B (host arrays: diagonal a[n], superdiagonal
    b[n-1]).  Returns (s, U, V, info) with s ascending and B V = U diag(s)."""
    a, b = _f64(a), _f64(b)
    n = len(a)
    s = np.zeros(max(n, 1))
    U = np.empty((max(n, 1), max(n, 1)), order="F")  # column-major, leading dimension n
    V = np.empty((max(n, 1), max(n, 1)), order="F")
    o = _opts(method, seed, j0, iters=_ptr(iters), **kw)
    info = _check(load().tinv_bdsvd(n, _ptr(a), _ptr(b), _ptr(s), _ptr(U), n, _ptr(V), n,
                                    ctypes.byref(o)), "tinv_bdsvd")
    if n == 0:
        return np.zeros(0), np.zeros((0, 0)), np.zeros((0, 0)), info
    return s[:n], U, V, info


def bdsvd_device(a, b, s, U, V, method="cwy", seed=0, j0=0, **kw):
    """tinv_bdsvd on torch CUDA tensors (float64 a[n], b[n-1], s[n], U[n, n] and V[n, n] whose
    rows are the singular vectors).  Synchronizes the tensors' stream.  Returns info."""
    n = a.numel()
    o = _opts(method, seed, j0, device=True, stream=_stream_of(a), **kw)
    return _check(load().tinv_bdsvd(n, _ptr(a), _ptr(b), _ptr(s), _ptr(U), n, _ptr(V), n,
                                    ctypes.byref(o)), "tinv_bdsvd")


# ------------------------------------------------------------------------------------------
# serving: request queue with continuous batching
# ------------------------------------------------------------------------------------------
class ServerCfg(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int32), ("max_inflight", ctypes.c_int32),
                ("hbm_fraction", ctypes.c_double), ("method", ctypes.c_int32),
                ("max_team", ctypes.c_int32), ("max_pending", ctypes.c_int32),
                ("device", ctypes.c_int32), ("wave_ctas", ctypes.c_int32),
                ("block", ctypes.c_int32), ("reserved", ctypes.c_int32 * 6)]


class Stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in
                ("submitted", "completed", "cancelled", "failed", "rejected", "waves",
                 "max_inflight_seen", "pending", "inflight_waves")] + \
               [(k, ctypes.c_double) for k in
                ("mean_wave_problems", "p50_ms", "p99_ms", "mean_ms", "problems_per_s",
                 "eigvecs_per_s")] + [("reserved", ctypes.c_double * 8)]


REQ_STATES = {0: "pending", 1: "running", 2: "done", 3: "cancelled", 4: "failed"}


class Server:
    """Request-queue server (tinv_server_*): submit problems at any time, wait for results."""

    def __init__(self, method="cwy", **cfg):
        lib = load()
        c = ServerCfg()
        lib.tinv_server_cfg_default(ctypes.byref(c))
        c.method = METHODS[method] if isinstance(method, str) else int(method)
        for k, v in cfg.items():
            setattr(c, k, v)
        h = ctypes.c_void_p()
        _check(lib.tinv_server_create(ctypes.byref(c), ctypes.byref(h)), "tinv_server_create")
        self._h = h
        self._bufs = {}  # ticket -> (Z, inputs kept alive until final)

    def submit(self, d, e, w=None, seed=0, out=None):
        d, e = _f64(d), _f64(e)
        w = None if w is None else _f64(w)
        n = len(d)
        Z = np.zeros((n, n), order="F") if out is None else out
        t = ctypes.c_uint64()
        rc = load().tinv_submit(self._h, n, _ptr(d), _ptr(e), _ptr(w), _ptr(Z), seed, ctypes.byref(t))
        _check(rc, "tinv_submit")
        self._bufs[t.value] = Z
        return t.value

    def poll(self, ticket):
        s = ctypes.c_int32()
        _check(load().tinv_poll(self._h, ticket, ctypes.byref(s)), "tinv_poll")
        return REQ_STATES[s.value]

    def wait(self, ticket, timeout_ms=-1):
        """Returns (Z, info); raises TinvError for a cancelled or failed request or a timeout."""
        info = ctypes.c_int64()
        rc = load().tinv_wait(self._h, ticket, timeout_ms, ctypes.byref(info))
        if rc == -103:  # timed out: the request stays queued
            raise TinvError(rc, "tinv_wait")
        Z = self._bufs.pop(ticket, None)
        _check(rc, "tinv_wait")
        return Z, info.value

    def cancel(self, ticket):
        return load().tinv_cancel(self._h, ticket)

    def stats(self):
        st = Stats()
        _check(load().tinv_server_stats(self._h, ctypes.byref(st)), "tinv_server_stats")
        return {k: getattr(st, k) for k, _ in Stats._fields_ if k != "reserved"}

    def close(self):
        if self._h:
            load().tinv_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
