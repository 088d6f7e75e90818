"""CPU FP64 oracle for inverse iteration with MGS / Householder / compact-WY reorthogonalization
(Ishigami, Kimura, Nakamura, arXiv:1209.1910).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The product path (the CUDA
library and its binding) never imports it, and it shares no code with that path.

The arithmetic lives in ``tinv_oracle.c`` (plain C, built with ``-ffp-contract=off``); this
module only compiles it and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tinv_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MGS, CWY, HOUSE = 0, 1, 2
METHODS = {"mgs": MGS, "cwy": CWY, "house": HOUSE}


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, -O2, no FP contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "tinv_oracle.h"))
    ):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Stats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int64), ("breakdowns", ctypes.c_int64),
                ("orth_flops", ctypes.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            D = ctypes.c_double
            lib.orc_sm64_mix.restype = ctypes.c_uint64
            lib.orc_sm64_mix.argtypes = [ctypes.c_uint64]
            lib.orc_start_value.restype = D
            lib.orc_start_value.argtypes = [ctypes.c_uint64, I64, ctypes.c_int, I64]
            lib.orc_onenorm.restype = D
            lib.orc_onenorm.argtypes = [I64, P, P]
            lib.orc_split.restype = I64
            lib.orc_split.argtypes = [I64, P, P, P]
            lib.orc_sturm_count.restype = I64
            lib.orc_sturm_count.argtypes = [I64, P, P, D, D]
            lib.orc_bisect.restype = None
            lib.orc_bisect.argtypes = [I64, P, P, P]
            lib.orc_plan.restype = None
            lib.orc_plan.argtypes = [I64, P, P, I64, P, P, P, P, P, P]
            lib.orc_lagtf.restype = None
            lib.orc_lagtf.argtypes = [I64, P, P, D, P, P, P, P, P]
            lib.orc_lagts.restype = D
            lib.orc_lagts.argtypes = [I64, P, P, P, P, P, P]
            for name in ("orc_orth_mgs",):
                getattr(lib, name).restype = D
                getattr(lib, name).argtypes = [I64, I64, P, I64, P, I64]
            for name in ("orc_orth_house", "orc_orth_cwy_ordinary", "orc_orth_cwy_new"):
                getattr(lib, name).restype = D
                getattr(lib, name).argtypes = [I64, I64, P, I64, P, I64, P, P]
            lib.orc_orth_cwy_block.restype = D
            lib.orc_orth_cwy_block.argtypes = [I64, I64, P, I64, I64, P, I64, P, P]
            lib.orc_tinv_blocked.restype = I64
            lib.orc_tinv_blocked.argtypes = [I64, P, P, I64, P, I64, P, I64, I64,
                                             ctypes.c_uint64, P, P, ctypes.POINTER(_Stats)]
            lib.orc_tinv.restype = I64
            lib.orc_tinv.argtypes = [I64, P, P, I64, P, I64, P, I64, ctypes.c_int,
                                     ctypes.c_uint64, P, P, ctypes.POINTER(_Stats)]
            lib.orc_jacobi.restype = None
            lib.orc_jacobi.argtypes = [I64, P, P, P]
            _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None and a.size else None


# ----------------------------------------------------------------------------------------
def sm64_mix(z: int) -> int:
    return int(_load().orc_sm64_mix(ctypes.c_uint64(z & 0xFFFFFFFFFFFFFFFF)))


def start_vector(seed: int, j: int, n: int, attempt: int = 0) -> np.ndarray:
    lib = _load()
    return np.array([lib.orc_start_value(seed, j, attempt, i) for i in range(n)])


def onenorm(d, e) -> float:
    d, e = _f64(d), _f64(e)
    return float(_load().orc_onenorm(len(d), _p(d), _p(e)))


def split(d, e) -> np.ndarray:
    """One past the last row of each unreduced block (row i ends a block iff
    |e_i| <= eps ||T||_1)."""
    d, e = _f64(d), _f64(e)
    n = len(d)
    isplit = np.zeros(max(n, 1), dtype=np.int64)
    nb = int(_load().orc_split(n, _p(d), _p(e), _p(isplit)))
    return isplit[:nb].copy()


def sturm_count(d, e, x: float, pivmin: float) -> int:
    d, e = _f64(d), _f64(e)
    return int(_load().orc_sturm_count(len(d), _p(d), _p(e), x, pivmin))


def bisect(d, e) -> np.ndarray:
    d, e = _f64(d), _f64(e)
    w = np.empty(len(d))
    _load().orc_bisect(len(d), _p(d), _p(e), _p(w))
    return w


def plan(d, e, w):
    """Returns (wp, head, onenrm, ortol, dtpcrt)."""
    d, e, w = _f64(d), _f64(e), _f64(w)
    m = len(w)
    wp = np.empty(m)
    head = np.empty(m, dtype=np.int64)
    o = (ctypes.c_double * 3)()
    _load().orc_plan(len(d), _p(d), _p(e), m, _p(w), _p(wp), _p(head),
                     ctypes.byref(o, 0), ctypes.byref(o, 8), ctypes.byref(o, 16))
    return wp, head, o[0], o[1], o[2]


def lagtf(d, e, lam: float):
    """Returns (u0, u1, u2, l, piv) of T - lam*I = P L U."""
    d, e = _f64(d), _f64(e)
    n = len(d)
    u0, u1, u2, l = (np.zeros(n) for _ in range(4))
    piv = np.zeros(n, dtype=np.uint8)
    _load().orc_lagtf(n, _p(d), _p(e), lam, _p(u0), _p(u1), _p(u2), _p(l), _p(piv))
    return u0, u1, u2, l, piv


def lagts(factors, y):
    u0, u1, u2, l, piv = factors
    x = _f64(y).copy()
    tol = _load().orc_lagts(len(u0), _p(u0), _p(u1), _p(u2), _p(l), _p(piv), _p(x))
    return x, tol


def orth(V, method: str, block: int = 0):
    """Stand-alone orthogonalization of the columns of V (n x m).  Returns (Q, Y, T, flops);
    Y/T are None for MGS, T is the vector of t_j for Householder.  method "cwy_block" takes
    the columns `block` at a time (Sec. 3.2)."""
    V = np.asfortranarray(V, dtype=np.float64)
    n, m = V.shape
    Q = np.zeros((n, m), order="F")
    lib = _load()
    if method == "cwy_block":
        Y = np.zeros((n, m), order="F")
        T = np.zeros((m, m), order="F")
        fl = lib.orc_orth_cwy_block(n, m, _p(V), n, max(1, block), _p(Q), n, _p(Y), _p(T))
        return Q, Y, T, fl
    if method == "mgs":
        fl = lib.orc_orth_mgs(n, m, _p(V), n, _p(Q), n)
        return Q, None, None, fl
    Y = np.zeros((n, m), order="F")
    if method == "house":
        tv = np.zeros(m)
        fl = lib.orc_orth_house(n, m, _p(V), n, _p(Q), n, _p(Y), _p(tv))
        return Q, Y, tv, fl
    T = np.zeros((m, m), order="F")
    fn = {"cwy_ordinary": lib.orc_orth_cwy_ordinary, "cwy_new": lib.orc_orth_cwy_new}[method]
    fl = fn(n, m, _p(V), n, _p(Q), n, _p(Y), _p(T))
    return Q, Y, T, fl


def tinv(d, e, w, method: str = "cwy", seed: int = 0, j0: int = 0, block: int = 0):
    """Inverse iteration for the eigenvectors of w.  Returns (Z, info, ifail, iters, stats).
    block >= 1 (method "cwy"): each cluster's members orthogonalized `block` at a time."""
    d, e, w = _f64(d), _f64(e), _f64(w)
    n, m = len(d), len(w)
    Z = np.zeros((n, m), order="F")
    ifail = np.zeros(max(m, 1), dtype=np.int64)
    iters = np.zeros(max(m, 1), dtype=np.int32)
    st = _Stats()
    if block >= 1:
        if method != "cwy":
            raise ValueError("blocked orthogonalization is compact WY")
        info = _load().orc_tinv_blocked(n, _p(d), _p(e), m, _p(w), j0, _p(Z), n, block,
                                        ctypes.c_uint64(seed), _p(ifail), _p(iters),
                                        ctypes.byref(st))
    else:
        info = _load().orc_tinv(n, _p(d), _p(e), m, _p(w), j0, _p(Z), n, METHODS[method],
                                ctypes.c_uint64(seed), _p(ifail), _p(iters), ctypes.byref(st))
    return Z, int(info), ifail[:info], iters[:m], {
        "sweeps": st.sweeps, "breakdowns": st.breakdowns, "orth_flops": st.orth_flops}


def eig_split(d, e, method: str = "cwy", seed: int = 0, j0: int = 0):
    """All eigenpairs of T split into unreduced blocks: each block's eigenvalues by bisection
    and its eigenvectors by `tinv` (the same method, seed and j0 for every block), merged into
    ascending order by a stable sort over the blocks' values in block order (ties keep the
    lower block first).  Returns (w, Z, iblock, isplit, info); Z is n x n with each column zero
    outside its block."""
    d, e = _f64(d), _f64(e)
    n = len(d)
    isplit = split(d, e)
    vals, blk, cols = [], [], []
    info = 0
    b0 = 0
    for b, b1 in enumerate(isplit):
        db, eb = d[b0:b1], e[b0:b1 - 1]
        wb = bisect(db, eb)
        Zb, ib, _, _, _ = tinv(db, eb, wb, method=method, seed=seed, j0=j0)
        info += ib
        for l in range(b1 - b0):
            col = np.zeros(n)
            col[b0:b1] = Zb[:, l]
            vals.append(wb[l])
            blk.append(b)
            cols.append(col)
        b0 = b1
    order = np.argsort(np.asarray(vals), kind="stable")
    w = np.asarray(vals)[order] if n else np.zeros(0)
    Z = np.zeros((n, n), order="F")
    for j, src in enumerate(order):
        Z[:, j] = cols[src]
    iblock = np.asarray(blk, dtype=np.int64)[order] if n else np.zeros(0, dtype=np.int64)
    return w, Z, iblock, isplit, info


def golub_kahan(a, b):
    """The Golub-Kahan form of the upper bidiagonal B (diagonal a[n], superdiagonal b[n-1]):
    the symmetric tridiagonal T_GK of order 2n with zero diagonal and off-diagonal
    (a_1, b_1, a_2, b_2, ..., a_n).  Its eigenvalues are +-sigma_i; for +sigma the eigenvector
    is (v_1, u_1, v_2, u_2, ..., v_n, u_n) / sqrt(2) with B v = sigma u, B^T u = sigma v."""
    a, b = _f64(a), _f64(b)
    n = len(a)
    e2 = np.zeros(max(2 * n - 1, 0))
    e2[0::2] = a
    e2[1::2] = b
    return np.zeros(2 * n), e2


def bdsvd(a, b, method: str = "cwy", seed: int = 0, j0: int = 0):
    """Singular triplets of the upper bidiagonal B by inverse iteration on T_GK (the paper's
    Sec. 6 names singular vectors of a bidiagonal matrix as a further use of the method):
    s = the n largest eigenvalues of T_GK by bisection (ascending), z_j the eigenvector of s_j
    from `tinv` with the given method, seed and j0; v_j = the even entries of z_j and u_j = the
    odd ones, each scaled to unit 2-norm (left as zeros if they are all zero).  Returns
    (s, U, V, info)."""
    n = len(a)
    d2, e2 = golub_kahan(a, b)
    if n == 0:
        return np.zeros(0), np.zeros((0, 0)), np.zeros((0, 0)), 0
    w2 = bisect(d2, e2)
    s = w2[n:].copy()
    Z, info, _, _, _ = tinv(d2, e2, s, method=method, seed=seed, j0=j0)
    V = np.array(Z[0::2, :], order="F")
    U = np.array(Z[1::2, :], order="F")
    for j in range(n):
        nv = np.sqrt(np.sum(V[:, j] * V[:, j]))
        nu = np.sqrt(np.sum(U[:, j] * U[:, j]))
        if nv > 0:
            V[:, j] = V[:, j] / nv
        if nu > 0:
            U[:, j] = U[:, j] / nu
    return s, U, V, info


def jacobi(A):
    """Cyclic Jacobi: returns (ascending eigenvalues, eigenvectors as columns)."""
    A = np.asfortranarray(A, dtype=np.float64).copy(order="F")
    n = A.shape[0]
    lam = np.zeros(n)
    V = np.zeros((n, n), order="F")
    _load().orc_jacobi(n, _p(A), _p(lam), _p(V))
    return lam, V
